"""Error norms of Section 3 ("Error and notations", Eq. meanErr) and moments.

kappa selects the central 2^-kappa part of the d x d solution matrix.  The
printed index set I^kappa = {floor(d/2 - d/2^(kappa+1)), ..., floor(d/2 +
d/2^(kappa+1))} has floor(d/2^kappa) + 1 members while the stated size is
floor(d/2^kappa); this oracle reads it as the half-open 0-based range
    [lo, lo + floor(d/2^kappa)),  lo = floor(d/2 - d/2^(kappa+1)),
so kappa = 0 is the whole grid.

    ME    = (1/M) sum_m |U_ref,m - U_app,m|          (matrix over I x I)
    AME   = mean of ME over I x I
    Err   = (1/M) sum_m ||U_ref,m - U_app,m||_F / ||U_ref,m||_F
Arrays are (paths, n_v, n_x); the region is applied to both axes.
"""
from __future__ import annotations

import math

import numpy as np


def kappa_range(d: int, kappa: int):
    lo = math.floor(d / 2 - d / 2 ** (kappa + 1))
    return lo, lo + math.floor(d / 2 ** kappa)


def _region(U, kappa):
    U = np.asarray(U, dtype=np.float64)
    lo, hi = kappa_range(U.shape[-1], kappa)
    lov, hiv = kappa_range(U.shape[-2], kappa)
    return U[..., lov:hiv, lo:hi]


def rel_err_per_path(U_app, U_ref, kappa: int = 0):
    a, r = _region(U_app, kappa), _region(U_ref, kappa)
    num = np.sqrt(np.sum((r - a) ** 2, axis=(-2, -1)))
    den = np.sqrt(np.sum(r ** 2, axis=(-2, -1)))
    return num / den


def Err(U_app, U_ref, kappa: int = 0):
    return float(np.mean(rel_err_per_path(U_app, U_ref, kappa)))


def ME(U_app, U_ref, kappa: int = 0):
    return np.mean(np.abs(_region(U_ref, kappa) - _region(U_app, kappa)), axis=0)


def AME(U_app, U_ref, kappa: int = 0):
    return float(np.mean(ME(U_app, U_ref, kappa)))


def moments(U, xs, vs, dx, dv):
    """Per path: mass, mean x, mean v, cov xx, xv, vv of the grid function.

    U is (paths, n_v, n_x); mass = sum u dx dv, moments normalised by mass.
    """
    U = np.asarray(U, dtype=np.float64)
    X, V = np.meshgrid(xs, vs, indexing="xy")          # (n_v, n_x)
    m = U.sum(axis=(-2, -1)) * dx * dv
    ex = (U * X).sum(axis=(-2, -1)) * dx * dv / m
    ev = (U * V).sum(axis=(-2, -1)) * dx * dv / m
    cxx = (U * X * X).sum(axis=(-2, -1)) * dx * dv / m - ex * ex
    cxv = (U * X * V).sum(axis=(-2, -1)) * dx * dv / m - ex * ev
    cvv = (U * V * V).sum(axis=(-2, -1)) * dx * dv / m - ev * ev
    return np.stack([m, ex, ev, cxx, cxv, cvv], axis=-1)

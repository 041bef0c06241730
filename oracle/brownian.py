"""Brownian paths on the fine ("Lebesgue") grid and the per-step functionals.

Section 3 ("Implementation", "Error and notations") computes the Lebesgue
integrals of the Magnus formulas by simple Riemann sums on a fine grid of
mesh Delta^Leb (1e-4 in all experiments).  The rule is not stated; this
oracle reads every functional as the exact integral of the piecewise-linear
interpolant of W through the fine nodes, so that for a fine cell
[s_k, s_k+1] with end values w0, w1 and width delta
    int W ds    = delta (w0 + w1) / 2
    int W^2 ds  = delta (w0^2 + w0 w1 + w1^2) / 3
    int s W ds  = delta (s_k (2 w0 + w1) + s_k+1 (w0 + 2 w1)) / 6.
Under that reading dW = (dW_k / delta) ds on each cell, so a stochastic
integral of a deterministic weight f becomes sum_k f(s_k+1/2) dW_k (midpoint of
the cell) and a Lebesgue integral of a product f(s) omega(s) with omega known
at the nodes is the trapezoid sum.  For constant coefficients this reduces
exactly to the integrals above (summation by parts).

Functionals of Magnus step n use the step-local Brownian motion
W~(s) = W(t_n + s) - W(t_n), 0 <= s <= h (the iterated scheme restarts the
expansion at each sub-interval, Section 2 "Iterated Magnus expansion").
"""
from __future__ import annotations

import numpy as np

from .coefficients import Coefficients
from .philox import standard_normals


def fine_increments(w, path_local: int) -> np.ndarray:
    """dW_k, k = 0..n_fine-1, of local path `path_local` (global index path_offset + p)."""
    z = standard_normals(w.seed, w.path_offset + path_local, w.n_fine)
    return np.sqrt(w.T / w.n_fine) * z


def _cells(w, K: int):
    if w.n_fine % K:
        raise ValueError("n_fine must be a multiple of the number of steps")
    return w.n_fine // K


def interval_functionals(w, path_local: int, c0: int, c1: int, dw_all=None) -> dict:
    """Functionals of the fine cells c0 .. c1-1, i.e. of [t0, t0 + h] with t0 = c0 delta and
    h = (c1 - c0) delta, with the Brownian motion restarted at t0 (W~(s) = W(t0 + s) - W(t0)):
      dW  = W~(h)                       I1 = int_0^h W~ ds
      I2  = int_0^h W~^2 ds             I3 = int_0^h s W~ ds
      om  = omega~(h) = int_0^h sigma dW
      Jom = int_0^h omega~ ds
      G1  = int omega~ ds - int s sigma dW
      G2  = int alpha omega~ ds - int alpha_bar sigma dW
    where sigma, alpha are evaluated at absolute time t0 + s.  A Magnus step is one
    such interval; an output time inside a step is another (Section 3, "Implementation":
    the expansion of a sub-interval evaluated at any time inside it)."""
    if not 0 <= c0 < c1 <= w.n_fine:
        raise ValueError("need 0 <= c0 < c1 <= n_fine")
    coef = Coefficients.of(w)
    delta = w.T / w.n_fine
    if dw_all is None:
        dw_all = fine_increments(w, path_local)
    dw = dw_all[c0:c1]
    L = c1 - c0
    tn = c0 * delta
    s_nodes = delta * np.arange(L + 1)
    s_mid = delta * (np.arange(L) + 0.5)
    wn = np.concatenate(([0.0], np.cumsum(dw)))            # W~ at the fine nodes
    w0, w1 = wn[:-1], wn[1:]
    out = {"dW": wn[-1],
           "I1": np.sum(delta * (w0 + w1) / 2.0),
           "I2": np.sum(delta * (w0 * w0 + w0 * w1 + w1 * w1) / 3.0),
           "I3": np.sum(delta * (s_nodes[:-1] * (2 * w0 + w1) + s_nodes[1:] * (w0 + 2 * w1)) / 6.0)}
    sig_mid = coef.sigma(tn + s_mid)
    om = np.concatenate(([0.0], np.cumsum(sig_mid * dw)))   # omega~ at the nodes
    alp = coef.alpha(tn + s_nodes)
    abar_mid = coef.alpha_bar(tn, s_mid)
    jom = np.sum(delta * (om[:-1] + om[1:]) / 2.0)
    out["om"] = om[-1]
    out["Jom"] = jom
    out["G1"] = jom - np.sum(s_mid * sig_mid * dw)
    out["G2"] = (np.sum(delta * (alp[:-1] * om[:-1] + alp[1:] * om[1:]) / 2.0)
                 - np.sum(abar_mid * sig_mid * dw))
    return out


def step_functionals(w, path_local: int, K: int) -> dict:
    """Per-step functionals of one path for an iterated scheme with K steps: the
    interval functionals of the cells n L .. (n+1) L - 1, n = 0..K-1 (arrays of length K)."""
    L = _cells(w, K)
    dw_all = fine_increments(w, path_local)
    per = [interval_functionals(w, path_local, n * L, (n + 1) * L, dw_all) for n in range(K)]
    return {k: np.array([f[k] for f in per]) for k in ("dW", "I1", "I2", "I3", "om", "Jom", "G1", "G2")}


def terminal_functionals(w, path_local: int) -> dict:
    """Whole-interval functionals used by the explicit solution.

    omega_T = int_0^T sigma dW and int_0^T omega_t dt, with the same fine-grid
    reading as step_functionals (midpoint weights, trapezoid in time).
    """
    coef = Coefficients.of(w)
    delta = w.T / w.n_fine
    dw = fine_increments(w, path_local)
    s_mid = delta * (np.arange(w.n_fine) + 0.5)
    om = np.concatenate(([0.0], np.cumsum(coef.sigma(s_mid) * dw)))
    return {"omega_T": om[-1], "int_omega": np.sum(delta * (om[:-1] + om[1:]) / 2.0),
            "W_T": np.sum(dw)}


def coarse_increments(w, path_local: int, n_steps: int) -> np.ndarray:
    """Brownian increments over n_steps equal steps (sums of fine increments)."""
    L = _cells(w, n_steps)
    return fine_increments(w, path_local).reshape(n_steps, L).sum(axis=1)

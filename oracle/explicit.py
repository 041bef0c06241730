"""Closed-form solution of the Langevin SPDE for a Gaussian initial datum.

Section 3.1 states the fundamental solution for constant 0 < sigma^2 < a: a
Kolmogorov kernel Gamma_0 shifted along m_t(zeta), and leaves the solution for
a Gaussian datum to the authors' code.  Re-derived here by Fourier transform
in (x, v): with k = (xi, eta), d u^ = (-a/2 eta^2 - kappa xi d_eta) u^ dt
+ i sigma eta u^ dW, integrated along the characteristics eta_t = eta_T -
kappa xi (T - t).  For u0 = c0 N(m0, S0) this gives

    u_T(z) = c0 N(z; M_T m0 + c_T, M_T S0 M_T^T + C_T)
    M_T = [[1, -kappa T], [0, 1]]
    C_T = int_0^T (a(t) - sigma(t)^2) m(T-t) m(T-t)^T dt,   m(tau) = (-kappa tau, 1)
    c_T = (kappa int_0^T omega_t dt, -omega_T),              omega_t = int_0^t sigma dW.

For kappa = -1 and constant coefficients the mean shift is the paper's
m_t(zeta) = (xi + t eta - sigma int W ds, eta - sigma W_t) and C_T is the
covariance of Gamma_0, (a - sigma^2) [[T^3/3, T^2/2], [T^2/2, T]].
The Brownian functionals use the same fine-grid reading as brownian.py.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import quad

from workloads import COEF_CONST
from .brownian import terminal_functionals
from .coefficients import Coefficients
from .discretization import gaussian_density, grid


def drift_matrix(kappa: float, T: float):
    return np.array([[1.0, -kappa * T], [0.0, 1.0]])


def diffusion_cov(w):
    """C_T as (xx, xv, vv)."""
    k, T = float(w.drift_sign), w.T
    coef = Coefficients.of(w)
    if w.kind == COEF_CONST:
        g = coef.a0 - coef.s0 ** 2
        return g * k * k * T ** 3 / 3.0, -g * k * T ** 2 / 2.0, g * T

    def gam(t):
        return float(coef.a(t)) - float(coef.sigma(t)) ** 2

    opts = dict(epsabs=1e-15, epsrel=1e-13, limit=200)
    cxx = quad(lambda t: gam(t) * (k * (T - t)) ** 2, 0.0, T, **opts)[0]
    cxv = quad(lambda t: gam(t) * (-k * (T - t)), 0.0, T, **opts)[0]
    cvv = quad(gam, 0.0, T, **opts)[0]
    return cxx, cxv, cvv


def terminal_gaussian(w, path_local: int):
    """Mean (x, v) and covariance (xx, xv, vv) of u_T / c0 for one path."""
    if getattr(w, "x_profile", 0) != 0:
        raise ValueError("no closed form with x-dependent coefficients (Section 3.2)")
    k = float(w.drift_sign)
    M = drift_matrix(k, w.T)
    m0 = np.asarray(w.u0_mean, float)
    S0 = np.array([[w.u0_cov[0], w.u0_cov[1]], [w.u0_cov[1], w.u0_cov[2]]])
    f = terminal_functionals(w, path_local)
    cT = np.array([k * f["int_omega"], -f["omega_T"]])
    mean = M @ m0 + cT
    cxx, cxv, cvv = diffusion_cov(w)
    S = M @ S0 @ M.T + np.array([[cxx, cxv], [cxv, cvv]])
    return mean, (S[0, 0], S[0, 1], S[1, 1])


def solution(w, path_local: int):
    """u_T on the interior grid, [v][x] layout."""
    xs, _ = grid(w.d, w.ax, w.bx)
    vs, _ = grid(w.d, w.av, w.bv)
    X, V = np.meshgrid(xs, vs, indexing="ij")
    mean, cov = terminal_gaussian(w, path_local)
    return gaussian_density(X, V, mean, cov, w.u0_scale).T.copy()


def solutions(w, paths=None):
    paths = range(w.paths) if paths is None else paths
    return np.stack([solution(w, p) for p in paths]) if len(paths) else np.zeros((0, w.d, w.d))

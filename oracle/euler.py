"""Euler-Maruyama comparator in matrix form (Eq. EulerMaruyama), oracle side.

The paper does not vectorise for Euler: with u the n_x x n_v solution matrix,
an x derivative multiplies from the left and a v derivative from the right by
the transposed matrix, and coefficient grids act by Hadamard products.  For
the Langevin coefficients (f^x = kappa v, g^vv = a psi(x), sigma^v = sigma
sqrt(psi(x)); psi = 1 for constant coefficients) one step is
    u_{k+1} = u_k + ( F^x . (D^x u_k) + 1/2 G^vv . (u_k (D^vv)^T) ) dt
                  + ( Sigma^v . (u_k (D^v)^T) ) dW_k,
with time-dependent a, sigma taken at the left end t_k of the step and dW_k
the sum of the fine increments inside the step.
"""
from __future__ import annotations

import numpy as np

from .brownian import coarse_increments
from .coefficients import Coefficients
from .discretization import coefficient_grid, d_first, d_second, gaussian_initial, grid, x_profile


def solve_path(w, n_steps: int, path_local: int):
    xs, dx = grid(w.d, w.ax, w.bx)
    vs, dv = grid(w.d, w.av, w.bv)
    Dx, Dv, Dvv = d_first(w.d, dx), d_first(w.d, dv), d_second(w.d, dv)
    Fx = coefficient_grid(lambda x, v: w.drift_sign * v, xs, vs)
    Psi = coefficient_grid(lambda x, v: x_profile(w, x), xs, vs)      # (n_x, n_v)
    coef = Coefficients.of(w)
    dt = w.T / n_steps
    dW = coarse_increments(w, path_local, n_steps)
    u = gaussian_initial(w, xs, vs)                    # (n_x, n_v)
    for k in range(n_steps):
        tk = k * dt
        a_k, s_k = float(coef.a(tk)), float(coef.sigma(tk))
        u_DvvT = (Dvv @ u.T).T                         # u (D^vv)^T
        u_DvT = (Dv @ u.T).T                           # u (D^v)^T
        drift = Fx * (Dx @ u) + 0.5 * a_k * Psi * u_DvvT
        noise = s_k * np.sqrt(Psi) * u_DvT
        u = u + drift * dt + noise * dW[k]
    return u.T.copy()                                  # [v][x]


def solve(w, n_steps: int, paths=None):
    paths = range(w.paths) if paths is None else paths
    return np.stack([solve_path(w, n_steps, p) for p in paths]) if len(paths) else \
        np.zeros((0, w.d, w.d))

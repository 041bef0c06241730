"""Iterated Ito-stochastic Magnus scheme (orders 1, 2, 3), oracle side.

Constant coefficients: the truncated Magnus logarithms of Eq. MagnusFormulas,
    Y1 = B t + A W_t
    Y2 = Y1 - 1/2 A^2 t + [B,A] int_0^t W ds - 1/2 [B,A] t W_t
    Y3 = Y2 + [[B,A],A] (1/2 int W^2 ds - 1/2 W_t int W ds + t W_t^2 / 12)
            + [[B,A],B] (int s W ds - 1/2 t int W ds - t^2 W_t / 12),
with [X,Y] = XY - YX formed by sparse matrix products.

Time-dependent coefficients (beyond the paper, which treats constant A, B and
says the extension is straightforward, Section 2 and Remark piecewise): with
B_t = Bx + alpha(t) Bvv and A_t = sigma(t) A0, repeating the Appendix's
order-2 Picard step (sigma_2, mu_2 of Eq. sigmaMagnusCut / muMagnusCut with
Y1_t = t Bx + alpha_bar_t Bvv + omega_t A0) gives, on a step of length h,
    Y2 = h Bx + alpha_bar_h Bvv + omega_h A0 - 1/2 (int sigma^2) A0^2
         + 1/2 [Bx,A0] G1 + 1/2 [Bvv,A0] G2 - 1/2 [Bx,Bvv] G3
    G1 = int omega ds - int s sigma dW
    G2 = int alpha omega ds - int alpha_bar sigma dW
    G3 = int (s alpha - alpha_bar) ds,
which reduces exactly to the constant Y2.  Order 3 adds the two third-order
terms of Eq. MagnusFormulas with B, A frozen at the step midpoint.

The iterated scheme (Section 2, "Iterated Magnus expansion") applies
U <- exp(Y) U on each of K equal sub-intervals.  exp(Y) U is computed with
scipy's expm_multiply (Al-Mohy & Higham's truncated-Taylor action), a library
primitive; the dense exponential is never formed.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import expm_multiply

from workloads import COEF_CONST
from .brownian import fine_increments, interval_functionals, step_functionals
from .coefficients import Coefficients
from .discretization import LangevinOperators, gaussian_initial, vec


def comm(X, Y):
    """Matrix commutator [X, Y] = XY - YX."""
    return (X @ Y - Y @ X).tocsr()


def omega_const(B, A, h, dW, I1, I2, I3, order):
    """Truncated Magnus logarithm of Eq. MagnusFormulas on one step."""
    Y = B * h + A * dW
    if order >= 2:
        BA = comm(B, A)
        Y = Y - 0.5 * h * (A @ A) + BA * I1 - 0.5 * h * dW * BA
        if order >= 3:
            Y = (Y + comm(BA, A) * (0.5 * I2 - 0.5 * dW * I1 + h * dW * dW / 12.0)
                 + comm(BA, B) * (I3 - 0.5 * h * I1 - h * h * dW / 12.0))
    return Y.tocsr()


def omega_timedep(ops, coef, tn, h, f, order):
    """Order-1/2/3 logarithm for B_t = Bx + alpha(t) Bvv, A_t = sigma(t) A0."""
    Bx, Bvv, A0 = ops.Bx, ops.Bvv, ops.A0
    Y = h * Bx + float(coef.alpha_bar(tn, h)) * Bvv + f["om"] * A0
    if order >= 2:
        Y = (Y - 0.5 * coef.sigma_sq_integral(tn, h) * (A0 @ A0)
             + 0.5 * f["G1"] * comm(Bx, A0) + 0.5 * f["G2"] * comm(Bvv, A0)
             - 0.5 * coef.g3(tn, h) * comm(Bx, Bvv))
        if order >= 3:
            tm = tn + 0.5 * h
            Bm = Bx + float(coef.alpha(tm)) * Bvv
            Am = float(coef.sigma(tm)) * A0
            BA = comm(Bm, Am)
            dW, I1, I2, I3 = f["dW"], f["I1"], f["I2"], f["I3"]
            Y = (Y + comm(BA, Am) * (0.5 * I2 - 0.5 * dW * I1 + h * dW * dW / 12.0)
                 + comm(BA, Bm) * (I3 - 0.5 * h * I1 - h * h * dW / 12.0))
    return Y.tocsr()


def expm_action(Y, U):
    """exp(Y) U (library primitive)."""
    return expm_multiply(Y, U)


def solve_path(w, order: int, K: int, path_local: int, ops=None, u0=None):
    """U_T of one path after K iterated Magnus steps; returns the (n_v, n_x) array."""
    if order not in (1, 2, 3):
        raise ValueError("order must be 1, 2 or 3")
    ops = ops or LangevinOperators(w)
    coef = Coefficients.of(w)
    U = vec(gaussian_initial(w, ops.xs, ops.vs)) if u0 is None else np.asarray(u0, float).ravel()
    h = w.T / K
    f = step_functionals(w, path_local, K)
    if w.kind == COEF_CONST:
        B, A = ops.B(coef.a0), ops.A(coef.s0)
    for n in range(K):
        fn = {k: v[n] for k, v in f.items()}
        if w.kind == COEF_CONST:
            Y = omega_const(B, A, h, fn["dW"], fn["I1"], fn["I2"], fn["I3"], order)
        else:
            Y = omega_timedep(ops, coef, n * h, h, fn, order)
        U = expm_action(Y, U)
    return U.reshape(w.d, w.d)          # vec index j*nx + i -> [v][x]


def solve_times(w, order: int, K: int, path_local: int, cells, ops=None):
    """Solutions at several output times (Section 3, "Implementation": within each
    sub-interval the Magnus expansion is evaluated at every requested time).  Output
    time t = T c / n_fine (c in `cells`, 1 <= c <= n_fine) lies in the sub-interval
    n = (c - 1) // L of the K-step scheme (L = n_fine / K cells); the solution there is
    exp(Y(t_n, t)) U(t_n), Y over the cells n L .. c - 1 and U(t_n) the iterated solution
    after n full steps.  Returns shape (len(cells), n_v, n_x)."""
    if order not in (1, 2, 3):
        raise ValueError("order must be 1, 2 or 3")
    ops = ops or LangevinOperators(w)
    coef = Coefficients.of(w)
    L = w.n_fine // K
    if L * K != w.n_fine:
        raise ValueError("n_fine must be a multiple of K")
    delta = w.T / w.n_fine
    dw_all = fine_increments(w, path_local)
    U = vec(gaussian_initial(w, ops.xs, ops.vs))
    if w.kind == COEF_CONST:
        B, A = ops.B(coef.a0), ops.A(coef.s0)

    def log_of(c0, c1):
        f = interval_functionals(w, path_local, c0, c1, dw_all)
        h = (c1 - c0) * delta
        if w.kind == COEF_CONST:
            return omega_const(B, A, h, f["dW"], f["I1"], f["I2"], f["I3"], order)
        return omega_timedep(ops, coef, c0 * delta, h, f, order)

    out, n_done = [], 0
    for c in cells:
        if not 1 <= c <= w.n_fine:
            raise ValueError("output cells must lie in 1 .. n_fine")
        n = (c - 1) // L
        while n_done < n:                                   # advance U to t_n
            U = expm_action(log_of(n_done * L, (n_done + 1) * L), U)
            n_done += 1
        out.append(expm_action(log_of(n * L, c), U).reshape(w.d, w.d))
    return np.stack(out)


def solve(w, order: int, K: int, paths=None):
    """U_T for a list of local path indices (default: all w.paths); shape (P, n_v, n_x)."""
    ops = LangevinOperators(w)
    paths = range(w.paths) if paths is None else paths
    return np.stack([solve_path(w, order, K, p, ops) for p in paths]) if len(paths) else \
        np.zeros((0, w.d, w.d))


def omega_matrix(w, order: int, K: int, path_local: int, step: int):
    """The step-`step` Magnus logarithm of one path (for operator-level checks)."""
    ops = LangevinOperators(w)
    coef = Coefficients.of(w)
    h = w.T / K
    f = {k: v[step] for k, v in step_functionals(w, path_local, K).items()}
    if w.kind == COEF_CONST:
        return omega_const(ops.B(coef.a0), ops.A(coef.s0), h, f["dW"], f["I1"], f["I2"], f["I3"], order)
    return omega_timedep(ops, coef, step * h, h, f, order)


__all__ = ["comm", "omega_const", "omega_timedep", "expm_action", "solve_path", "solve", "solve_times",
           "omega_matrix", "sp"]

"""Space discretisation of Section 2: grids, finite differences, Kronecker assembly.

Grids (Eq. xGrid, vGrid): n + 2 equispaced points on [a, b] with
Delta = (b - a)/(n + 1); the unknowns live on the n interior points
x_i = a + i Delta, i = 1..n (0-based here: a + (i+1) Delta).

vec stacks the columns of the n_x x n_v matrix u_{ij} = u(x_i, v_j), so the
x index runs fastest: vec index = i + n_x j.

Finite differences with zero Dirichlet boundary (Section 2, "Computation of
A and B"):
    D^x  = tridiag(-1, 0, 1) / (2 Delta x)     D^xx = tridiag(1, -2, 1) / Delta x^2
and likewise in v.  Multiplication by a coefficient grid F is diag(vec F), an
x derivative is I_v (x) D^x and a v derivative is D^v (x) I_x, giving

  B = diag(vec H) + diag(vec F^x)(I (x) D^x) + diag(vec F^v)(D^v (x) I)
      + 1/2 diag(vec G^xx)(I (x) D^xx) + diag(vec G^xv)(D^v (x) D^x)
      + 1/2 diag(vec G^vv)(D^vv (x) I)
  A = diag(vec Sigma) + diag(vec Sigma^x)(I (x) D^x) + diag(vec Sigma^v)(D^v (x) I).

Matrices are scipy.sparse CSR in float64.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def grid(n: int, a: float, b: float):
    """Interior points and mesh of Eq. xGrid / vGrid."""
    delta = (b - a) / (n + 1)
    return a + delta * np.arange(1, n + 1), delta


def tridiag(n: int, lo: float, mid: float, up: float):
    return sp.diags([np.full(n - 1, lo), np.full(n, mid), np.full(n - 1, up)], [-1, 0, 1],
                    shape=(n, n), format="csr", dtype=np.float64)


def d_first(n: int, delta: float):
    return tridiag(n, -1.0, 0.0, 1.0) / (2.0 * delta)


def d_second(n: int, delta: float):
    return tridiag(n, 1.0, -2.0, 1.0) / (delta * delta)


def vec(u_xv: np.ndarray) -> np.ndarray:
    """Column stacking of an (n_x, n_v) matrix: x index fastest."""
    return np.asarray(u_xv).reshape(-1, order="F")


def unvec(U: np.ndarray, nx: int, nv: int) -> np.ndarray:
    return np.asarray(U).reshape((nx, nv), order="F")


def coefficient_grid(f, xs, vs):
    """Z^w = (f(x_i, v_j))_{ij} as an (n_x, n_v) matrix; f may be None (zero)."""
    X, V = np.meshgrid(xs, vs, indexing="ij")
    if f is None:
        return np.zeros_like(X)
    return np.broadcast_to(np.asarray(f(X, V), dtype=np.float64), X.shape).copy()


def assemble(nx, ax, bx, nv, av, bv, *, h=None, fx=None, fv=None, gxx=None, gxv=None,
             gvv=None, s=None, sx=None, sv=None):
    """B and A of Eq. SPDEvec for the general SPDE (Eq. generalSPDE)."""
    xs, dx = grid(nx, ax, bx)
    vs, dv = grid(nv, av, bv)
    Ix, Iv = sp.identity(nx, format="csr"), sp.identity(nv, format="csr")
    Dx, Dxx = d_first(nx, dx), d_second(nx, dx)
    Dv, Dvv = d_first(nv, dv), d_second(nv, dv)

    def dg(f):
        return sp.diags(vec(coefficient_grid(f, xs, vs)), 0, format="csr")

    B = (dg(h)
         + dg(fx) @ sp.kron(Iv, Dx)
         + dg(fv) @ sp.kron(Dv, Ix)
         + 0.5 * dg(gxx) @ sp.kron(Iv, Dxx)
         + dg(gxv) @ sp.kron(Dv, Dx)
         + 0.5 * dg(gvv) @ sp.kron(Dvv, Ix))
    A = (dg(s)
         + dg(sx) @ sp.kron(Iv, Dx)
         + dg(sv) @ sp.kron(Dv, Ix))
    return B.tocsr(), A.tocsr()


def x_profile(w, x):
    """psi(x) of the variable coefficients (Eq. coeffsLangevinVar).

    The paper's variable-coefficient Langevin SPDE has g^vv(x, v) = a (1 + 1/(x^2+1))
    and sigma^v(x, v) = sigma sqrt(1 + 1/(x^2+1)); with psi(x) = 1 + c/(1 + x^2)
    (c = 1 there) these are a psi and sigma sqrt(psi).  Without a profile psi = 1.
    """
    from workloads import XPROF_NONE, XPROF_RATIONAL
    x = np.asarray(x, dtype=np.float64)
    kind = getattr(w, "x_profile", XPROF_NONE)
    if kind == XPROF_NONE:
        return np.ones_like(x)
    if kind == XPROF_RATIONAL:
        return 1.0 + w.x_profile_c / (1.0 + x * x)
    raise ValueError("unknown x profile")


class LangevinOperators:
    """Unit operators of the Langevin SPDE on one grid.

    With f^x = kappa v, g^vv = a psi(x), sigma^v = sigma sqrt(psi(x)) and all
    other coefficients zero (Eq. coeffsLangevinConst with psi = 1, Eq.
    coeffsLangevinVar with the paper's psi; kappa = -1 there):
        B = Bx + (a/2) Bvv,   A = sigma A0,
        Bx  = diag(vec F^x)(I (x) D^x),  F^x_ij = kappa v_j
        Bvv = diag(vec Psi)(D^vv (x) I)
        A0  = diag(vec Psi^(1/2))(D^v (x) I)
    Each is assembled through the general formula of `assemble` with unit
    coefficients, so time-dependent a(t), sigma(t) only rescale Bvv and A0.
    """

    def __init__(self, w):
        d, k = w.d, float(w.drift_sign)
        self.d = d
        self.xs, self.dx = grid(d, w.ax, w.bx)
        self.vs, self.dv = grid(d, w.av, w.bv)
        args = (d, w.ax, w.bx, d, w.av, w.bv)
        psi = lambda x, v: x_profile(w, x)
        self.Bx, _ = assemble(*args, fx=lambda x, v: k * v)
        self.Bvv, _ = assemble(*args, gvv=lambda x, v: 2.0 * psi(x, v))   # 1/2 * 2 psi
        _, self.A0 = assemble(*args, sv=lambda x, v: np.sqrt(psi(x, v)))

    def B(self, a: float):
        return (self.Bx + (0.5 * a) * self.Bvv).tocsr()

    def A(self, sigma: float):
        return (sigma * self.A0).tocsr()


def gaussian_initial(w, xs=None, vs=None):
    """u0 on the interior grid as an (n_x, n_v) matrix.

    u0(z) = c0 N(z; m0, S0) with c0 = w.u0_scale (Eq. initialdatum is the
    unnormalised standard case c0 = 2 pi, m0 = 0, S0 = I).
    """
    if xs is None:
        xs, _ = grid(w.d, w.ax, w.bx)
    if vs is None:
        vs, _ = grid(w.d, w.av, w.bv)
    X, V = np.meshgrid(xs, vs, indexing="ij")
    return gaussian_density(X, V, w.u0_mean, w.u0_cov, w.u0_scale)


def gaussian_density(X, V, mean, cov, scale=1.0):
    mx, mv = mean
    cxx, cxv, cvv = cov
    det = cxx * cvv - cxv * cxv
    ex, ev = X - mx, V - mv
    q = (cvv * ex * ex - 2.0 * cxv * ex * ev + cxx * ev * ev) / det
    return scale * np.exp(-0.5 * q) / (2.0 * np.pi * np.sqrt(det))

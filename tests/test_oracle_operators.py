"""Pins of the oracle's space discretisation (Section 2) and commutators."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import discretization as disc
from oracle.magnus import comm
from workloads import LANGEVIN_32


def test_grid_definition():
    xs, dx = disc.grid(3, -1.0, 1.0)
    assert dx == 0.5
    np.testing.assert_array_equal(xs, [-0.5, 0.0, 0.5])


def test_fd_matrices_are_exact_on_low_degree_polynomials():
    n, a, b = 9, -2.0, 3.0
    xs, dx = disc.grid(n, a, b)
    D1, D2 = disc.d_first(n, dx).toarray(), disc.d_second(n, dx).toarray()
    # interior rows see both neighbours: central differences are exact on quadratics
    p = lambda x: 3 + 2 * x - x * x
    np.testing.assert_allclose((D1 @ p(xs))[1:-1], (2 - 2 * xs)[1:-1], atol=1e-9)
    q = lambda x: 1 - x + 4 * x ** 2 + x ** 3
    np.testing.assert_allclose((D2 @ q(xs))[1:-1], (8 + 6 * xs)[1:-1], atol=1e-9)
    # zero Dirichlet boundary: the first row drops the left neighbour
    assert D1[0, 0] == 0 and D1[0, 1] == 1 / (2 * dx) and D2[0, 0] == -2 / dx ** 2


def _bruteforce(nx, ax, bx, nv, av, bv, c):
    """B and A by looping over grid points with the finite-difference formulas of
    Section 2 written pointwise (zero outside the interior), independent of vec/kron."""
    xs, dx = disc.grid(nx, ax, bx)
    vs, dv = disc.grid(nv, av, bv)
    n = nx * nv
    B = np.zeros((n, n))
    A = np.zeros((n, n))
    idx = lambda i, j: i + nx * j
    for j in range(nv):
        for i in range(nx):
            r = idx(i, j)
            x, v = xs[i], vs[j]

            def add(M, di, dj, val):
                ii, jj = i + di, j + dj
                if 0 <= ii < nx and 0 <= jj < nv:
                    M[r, idx(ii, jj)] += val

            add(B, 0, 0, c["h"](x, v))
            add(B, 1, 0, c["fx"](x, v) / (2 * dx)); add(B, -1, 0, -c["fx"](x, v) / (2 * dx))
            add(B, 0, 1, c["fv"](x, v) / (2 * dv)); add(B, 0, -1, -c["fv"](x, v) / (2 * dv))
            g = 0.5 * c["gxx"](x, v) / dx ** 2
            add(B, 1, 0, g); add(B, -1, 0, g); add(B, 0, 0, -2 * g)
            g = c["gxv"](x, v) / (4 * dx * dv)
            add(B, 1, 1, g); add(B, -1, -1, g); add(B, 1, -1, -g); add(B, -1, 1, -g)
            g = 0.5 * c["gvv"](x, v) / dv ** 2
            add(B, 0, 1, g); add(B, 0, -1, g); add(B, 0, 0, -2 * g)
            add(A, 0, 0, c["s"](x, v))
            add(A, 1, 0, c["sx"](x, v) / (2 * dx)); add(A, -1, 0, -c["sx"](x, v) / (2 * dx))
            add(A, 0, 1, c["sv"](x, v) / (2 * dv)); add(A, 0, -1, -c["sv"](x, v) / (2 * dv))
    return B, A


def test_kronecker_assembly_matches_pointwise_stencils():
    rng = np.random.default_rng(0)
    names = ["h", "fx", "fv", "gxx", "gxv", "gvv", "s", "sx", "sv"]
    co = {}
    for k in names:
        p = rng.normal(size=3)
        co[k] = (lambda p: (lambda x, v: p[0] + p[1] * x + p[2] * v * v))(p)
    args = (5, -1.0, 2.0, 4, -3.0, 1.0)
    B, A = disc.assemble(*args, **co)
    Bb, Ab = _bruteforce(*args, co)
    np.testing.assert_allclose(B.toarray(), Bb, atol=1e-12)
    np.testing.assert_allclose(A.toarray(), Ab, atol=1e-12)


def test_vec_kronecker_identity():
    rng = np.random.default_rng(1)
    U = rng.normal(size=(4, 3))
    D1, D2 = rng.normal(size=(4, 4)), rng.normal(size=(3, 3))
    np.testing.assert_allclose(disc.vec(D1 @ U @ D2), np.kron(D2.T, D1) @ disc.vec(U), atol=1e-12)
    np.testing.assert_array_equal(disc.unvec(disc.vec(U), 4, 3), U)


def _ops(d=7, kappa=1, a=1.3, sigma=0.6):
    w = LANGEVIN_32.with_(d=d, drift_sign=kappa, a0=a, s0=sigma, ax=-2.0, bx=2.0, av=-3.0, bv=3.0)
    ops = disc.LangevinOperators(w)
    return w, ops, ops.B(a), ops.A(sigma)


@pytest.mark.parametrize("kappa", [1, -1])
def test_commutator_closed_forms(kappa):
    """Closed forms of the truncated-matrix commutators (Kronecker factors v (x) x):
        [B,A]     = -(kappa sigma/2) S (x) D^x + (a sigma / (2 dv^3)) E (x) I
        [[B,A],A] = -(kappa sigma^2 / (2 dv)) E (x) D^x - (a sigma^2 / (4 dv^4)) F (x) I
    with S = tridiag(1,0,1), E = diag(-1,0,...,0,1) and F the four corner
    couplings (1,2),(2,1),(d-1,d),(d,d-1).  Derived from
    [diag v, D^v] = -S/2, [D^vv, D^v] = E/dv^3, [S, D^v] = E/dv, [E, D^v] = -F/(2 dv)."""
    a, sigma = 1.3, 0.6
    w, ops, B, A = _ops(kappa=kappa, a=a, sigma=sigma)
    d, dv = w.d, ops.dv
    S = disc.tridiag(d, 1.0, 0.0, 1.0)
    E = sp.diags([np.r_[-1.0, np.zeros(d - 2), 1.0]], [0])
    F = sp.lil_matrix((d, d))
    F[0, 1] = F[1, 0] = F[d - 2, d - 1] = F[d - 1, d - 2] = 1.0
    Dx = disc.d_first(d, ops.dx)
    Ix = sp.identity(d)
    BA = comm(B, A)
    want = -(kappa * sigma / 2) * sp.kron(S, Dx) + (a * sigma / (2 * dv ** 3)) * sp.kron(E, Ix)
    np.testing.assert_allclose(BA.toarray(), want.toarray(), atol=1e-12 * abs(BA).max())
    BAA = comm(BA, A)
    want = (-(kappa * sigma ** 2 / (2 * dv)) * sp.kron(E, Dx)
            - (a * sigma ** 2 / (4 * dv ** 4)) * sp.kron(F.tocsr(), Ix))
    np.testing.assert_allclose(BAA.toarray(), want.toarray(), atol=1e-12 * abs(BAA).max())


def _diagonals(M, rel):
    M = M.tocoo()
    thr = rel * np.abs(M.data).max()
    keep = np.abs(M.data) > thr
    return len(set((M.col[keep] - M.row[keep]).tolist()))


def test_sparsity_pattern_of_the_paper_figure():
    """Fig. sparsity / Remark sparsity (d = 50, constant coefficients): A and B
    have 2 and 5 non-zero diagonals and [B,A] has 5.  Exactly, [[B,A],A] has 4
    and [[B,A],B] 6; the figure's 8 and 10 include diagonals that are zero up
    to rounding (every entry below 1e-12 of the largest)."""
    w = LANGEVIN_32.with_(d=50, ax=-4.0, bx=4.0, av=-4.0, bv=4.0, drift_sign=-1, a0=1.1,
                          s0=10 ** -0.5)
    ops = disc.LangevinOperators(w)
    B, A = ops.B(w.a0), ops.A(w.s0)
    BA = comm(B, A)
    counts = [_diagonals(M, 1e-12) for M in (A, B, BA, comm(BA, A), comm(BA, B))]
    assert counts == [2, 5, 5, 4, 6]


def test_langevin_operators_match_general_assembly():
    w, ops, B, A = _ops(kappa=-1, a=0.8, sigma=0.3)
    args = (w.d, w.ax, w.bx, w.d, w.av, w.bv)
    Bg, Ag = disc.assemble(*args, fx=lambda x, v: -v, gvv=lambda x, v: 0.8, sv=lambda x, v: 0.3)
    np.testing.assert_allclose(B.toarray(), Bg.toarray(), atol=1e-12)
    np.testing.assert_allclose(A.toarray(), Ag.toarray(), atol=1e-12)


def test_gaussian_initial_is_a_density():
    w = LANGEVIN_32.with_(d=200, ax=-12.0, bx=12.0, av=-12.0, bv=12.0, u0_mean=(0.3, -0.2),
                          u0_cov=(0.7, 0.2, 1.1))
    xs, dx = disc.grid(w.d, w.ax, w.bx)
    vs, dv = disc.grid(w.d, w.av, w.bv)
    u = disc.gaussian_initial(w)
    assert u.sum() * dx * dv == pytest.approx(1.0, rel=1e-6)
    X, V = np.meshgrid(xs, vs, indexing="ij")
    assert (u * X).sum() * dx * dv == pytest.approx(0.3, abs=1e-6)
    assert (u * X * V).sum() * dx * dv - 0.3 * -0.2 == pytest.approx(0.2, abs=1e-6)


# ---------------------------------------------------------------- variable coefficients
def _var_case(d=7, c=1.0, a=1.1, s=0.3, kappa=-1):
    from workloads import PAPER_VAR
    return PAPER_VAR[0].with_(d=d, x_profile_c=c, a0=a, s0=s, drift_sign=kappa)


def test_paper_profile_values():
    w = _var_case()
    # psi(0) = 2, psi(+-1) = 3/2, psi -> 1 far out (Eq. coeffsLangevinVar)
    np.testing.assert_allclose(disc.x_profile(w, [0.0, 1.0, -1.0, 1e8]), [2.0, 1.5, 1.5, 1.0], rtol=1e-15)
    # g^vv - (sigma^v)^2 = (a - sigma^2) psi: equals 1 everywhere only where psi = 1
    # for the paper's a = 1.1, sigma^2 = 0.1 the difference is a psi - sigma^2 psi = psi
    ws = _var_case(a=1.1, s=10 ** -0.5)
    x = np.linspace(-4, 4, 9)
    psi = disc.x_profile(ws, x)
    np.testing.assert_allclose(ws.a0 * psi - (ws.s0 * np.sqrt(psi)) ** 2, psi, rtol=1e-14)


@pytest.mark.parametrize("kappa", [1, -1])
def test_variable_coefficient_operators_match_pointwise_stencils(kappa):
    """B, A of the x-profile case against the pointwise finite-difference loops."""
    w = _var_case(d=6, c=0.7, a=1.3, s=0.4, kappa=kappa).with_(ax=-3.0, bx=2.0, av=-2.5, bv=3.5)
    ops = disc.LangevinOperators(w)
    psi = lambda x: 1.0 + 0.7 / (1.0 + x * x)
    zero = lambda x, v: 0.0 * x
    c = dict(h=zero, fx=lambda x, v: kappa * v + 0 * x, fv=zero, gxx=zero, gxv=zero,
             gvv=lambda x, v: 1.3 * psi(x), s=zero, sx=zero, sv=lambda x, v: 0.4 * np.sqrt(psi(x)))
    Bb, Ab = _bruteforce(6, -3.0, 2.0, 6, -2.5, 3.5, c)
    np.testing.assert_allclose(ops.B(1.3).toarray(), Bb, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(ops.A(0.4).toarray(), Ab, rtol=1e-13, atol=1e-12)


def test_variable_coefficient_operators_have_kronecker_form():
    """Bvv = D^vv (x) Psi and A0 = D^v (x) Psi^(1/2): the profile acts on the x index only."""
    w = _var_case(d=9)
    ops = disc.LangevinOperators(w)
    xs, dx = disc.grid(9, w.ax, w.bx)
    vs, dv = disc.grid(9, w.av, w.bv)
    Psi = sp.diags(disc.x_profile(w, xs))
    np.testing.assert_allclose(ops.Bvv.toarray(), sp.kron(disc.d_second(9, dv), Psi).toarray(), rtol=1e-14)
    np.testing.assert_allclose(ops.A0.toarray(), sp.kron(disc.d_first(9, dv), Psi.sqrt()).toarray(), rtol=1e-14)
    # the profile does not commute with D^x, so [Bx, A0] picks up the x-derivative of sqrt(psi)
    C = comm(ops.Bx, ops.A0).toarray()
    w1 = w.with_(x_profile=0)
    C1 = comm(disc.LangevinOperators(w1).Bx, disc.LangevinOperators(w1).A0).toarray()
    assert np.abs(C - C1).max() > 1e-3


def test_no_closed_form_with_a_profile():
    from oracle import explicit
    with pytest.raises(ValueError):
        explicit.solution(_var_case(), 0)

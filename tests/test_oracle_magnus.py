"""Pins of the oracle's Magnus scheme, Euler-Maruyama, explicit solution and norms."""
import math
import os

import mpmath
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import brownian, discretization as disc, errors, euler, explicit, magnus
from workloads import COEF_TRIG, LANGEVIN_32, LANGEVIN_TRIG_128

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _worked():
    vals, rows = {}, {}
    with open(os.path.join(GOLDEN, "magnus_sl2_worked.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            if t[0].isdigit():
                rows[int(t[0])] = np.array([float(x) for x in t[1:]]).reshape(2, 2)
            else:
                vals[t[0]] = float(t[1])
    return vals, rows


@pytest.mark.parametrize("order", [1, 2, 3])
def test_magnus_formulas_worked_example(order):
    v, rows = _worked()
    B = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    A = sp.csr_matrix(np.array([[0.0, 0.0], [1.0, 0.0]]))
    Y = magnus.omega_const(B, A, v["h"], v["dW"], v["I1"], v["I2"], v["I3"], order)
    np.testing.assert_allclose(Y.toarray(), rows[order], atol=1e-15)


def _tiny(d=4, sigma=0.0, kappa=1):
    return LANGEVIN_32.with_(d=d, ax=-2.0, bx=2.0, av=-2.0, bv=2.0, s0=sigma, drift_sign=kappa,
                             n_fine=64, paths=2)


def _expm_taylor_mp(M, u, digits=40, terms=400):
    """exp(M) u by a plain Taylor series in 40-digit arithmetic with scaling 2^-s."""
    mpmath.mp.dps = digits
    Mm = mpmath.matrix(M.tolist())
    nrm = max(sum(abs(Mm[i, j]) for j in range(Mm.cols)) for i in range(Mm.rows))
    s = max(0, int(math.ceil(math.log2(float(nrm) + 1e-30))) + 1)
    Ms = Mm / (2 ** s)
    x = mpmath.matrix(u.tolist())
    for _ in range(2 ** s):
        term, acc = x, x
        for k in range(1, terms):
            term = Ms * term / k
            acc = acc + term
            if mpmath.norm(term) < mpmath.mpf(10) ** (-digits + 2):
                break
        x = acc
    return np.array([float(t) for t in x])


def test_expm_action_against_padé_and_high_precision_taylor():
    w = _tiny(d=3, sigma=0.7)
    Y = magnus.omega_matrix(w, 3, 1, 0, 0)
    u = disc.vec(disc.gaussian_initial(w))
    got = magnus.expm_action(Y, u)
    pade = sla.expm(Y.toarray()) @ u
    mp = _expm_taylor_mp(Y.toarray(), u)
    np.testing.assert_allclose(got, mp, rtol=1e-12, atol=1e-14 * np.abs(mp).max())
    np.testing.assert_allclose(pade, mp, rtol=1e-12, atol=1e-14 * np.abs(mp).max())


def test_deterministic_case_is_exact_at_order_one():
    """Remark determLangevin: with A = 0 the order-1 scheme is exact up to the
    space discretisation, so any number of steps gives exp(T B) u0."""
    w = _tiny(d=6, sigma=0.0)
    ops = disc.LangevinOperators(w)
    u0 = disc.vec(disc.gaussian_initial(w))
    exact = sla.expm(w.T * ops.B(w.a0).toarray()) @ u0
    for K in (1, 4, 16):
        U = magnus.solve_path(w, 1, K, 0).ravel()
        np.testing.assert_allclose(U, exact, rtol=1e-11, atol=1e-13 * np.abs(exact).max())
    # orders 2 and 3 add only A-terms, which vanish
    for order in (2, 3):
        np.testing.assert_allclose(magnus.solve_path(w, order, 4, 1).ravel(), exact, rtol=1e-11,
                                   atol=1e-13 * np.abs(exact).max())


def test_higher_orders_add_vanishing_corrections():
    """||Y3 - Y2|| and ||Y2 - Y1|| shrink as the step h -> 0 (orders h and h^1.5
    in mean square for the Brownian weights of Eq. MagnusFormulas)."""
    w = LANGEVIN_32.with_(d=8, n_fine=2 ** 12)
    d21, d32 = [], []
    for K in (4, 64):
        diff21 = diff32 = 0.0
        for p in range(20):
            Y = [magnus.omega_matrix(w, o, K, p, 0) for o in (1, 2, 3)]
            diff21 += abs(Y[1] - Y[0]).sum()
            diff32 += abs(Y[2] - Y[1]).sum()
        d21.append(diff21)
        d32.append(diff32)
    assert d21[1] < d21[0] / 4       # ~ 16x smaller for h/16 at order h
    assert d32[1] < d32[0] / 8       # ~ 64x smaller at order h^1.5


def test_timedep_formulas_reduce_to_constant_ones():
    wc = LANGEVIN_32.with_(d=6, n_fine=120, ax=-3.0, bx=3.0, av=-3.0, bv=3.0, a0=1.2, s0=0.4)
    wt = wc.with_(kind=COEF_TRIG, a1=0.0, s1=0.0)
    for order in (1, 2, 3):
        Uc = magnus.solve_path(wc, order, 5, 3)
        Ut = magnus.solve_path(wt, order, 5, 3)
        np.testing.assert_allclose(Ut, Uc, rtol=1e-12, atol=1e-14)


def test_magnus_converges_to_the_explicit_solution_in_space():
    """Orders 2 and 3 approach the closed form as the grid is refined (the
    spatial error of central differences is O(Delta^2))."""
    errs = []
    for d in (20, 40):
        w = LANGEVIN_32.with_(d=d, paths=2)
        ref = explicit.solutions(w, [0, 1])
        errs.append([errors.Err(magnus.solve(w, o, 4, [0, 1]), ref) for o in (2, 3)])
    assert errs[0][0] > 3.0 * errs[1][0] and errs[0][1] > 3.0 * errs[1][1]
    assert errs[1][1] < 0.015


def test_order_one_is_consistent_with_the_stratonovich_equation():
    """Y1 = B t + A W_t has no Ito correction: the iterated m1 scheme converges
    to the solution with diffusion a + sigma^2 rather than a."""
    w = LANGEVIN_32.with_(d=40, paths=2)
    U = magnus.solve(w, 1, 50, [0, 1])
    e_strat = errors.Err(U, explicit.solutions(w.with_(a0=w.a0 + w.s0 ** 2), [0, 1]))
    e_ito = errors.Err(U, explicit.solutions(w, [0, 1]))
    assert e_strat < 0.02 < 0.04 < e_ito


def test_timedep_magnus_converges_in_time_and_space():
    w = LANGEVIN_TRIG_128.with_(d=40, n_fine=1024, paths=2)
    ref = explicit.solutions(w, [0, 1])
    fine = magnus.solve(w, 3, 128, [0, 1])
    assert errors.Err(fine, ref) < 0.04
    e8 = errors.Err(magnus.solve(w, 2, 8, [0, 1]), fine)
    e32 = errors.Err(magnus.solve(w, 2, 32, [0, 1]), fine)
    assert e32 < e8 / 4


def test_explicit_kernel_is_the_printed_gamma0():
    """Section 3.1: for kappa = -1, constant 0 < sigma^2 < a and a point datum,
    u_T(z) = Gamma_0(T, z - m_T(zeta)) with
    Gamma_0(t,(x,v)) = sqrt(3)/(pi t^2 (a - s^2)) exp(-2/(a-s^2) (v^2/t - 3vx/t^2 + 3x^2/t^3))."""
    a, s, T = 1.1, 10 ** -0.5, 0.7
    w = LANGEVIN_32.with_(d=30, drift_sign=-1, a0=a, s0=s, T=T, u0_mean=(0.4, -0.3),
                          u0_cov=(0.0, 0.0, 0.0), n_fine=700)
    mean, cov = explicit.terminal_gaussian(w, 5)
    f = brownian.terminal_functionals(w, 5)
    xi, eta = w.u0_mean
    m = np.array([xi + T * eta - f["int_omega"], eta - f["omega_T"]])   # omega = sigma W
    np.testing.assert_allclose(mean, m, atol=1e-14)
    g = a - s * s
    rng = np.random.default_rng(3)
    for _ in range(5):
        x, v = rng.normal(size=2)
        gam0 = math.sqrt(3) / (math.pi * T ** 2 * g) * math.exp(
            -2 / g * (v * v / T - 3 * v * x / T ** 2 + 3 * x * x / T ** 3))
        ours = disc.gaussian_density(np.array(x + m[0]), np.array(v + m[1]), mean, cov, 1.0)
        assert float(ours) == pytest.approx(gam0, rel=1e-12)


def test_explicit_solution_solves_the_kolmogorov_equation_when_sigma_is_zero():
    w = LANGEVIN_32.with_(s0=0.0, a0=0.9, drift_sign=1, u0_mean=(0.2, 0.1), u0_cov=(0.6, 0.1, 0.8))

    def u(t, x, v):
        ww = w.with_(T=t)
        mean, cov = explicit.terminal_gaussian(ww, 0)
        return disc.gaussian_density(np.array(x), np.array(v), mean, cov, 1.0)

    t, x, v, e = 0.6, 0.3, -0.4, 1e-4
    ut = (u(t + e, x, v) - u(t - e, x, v)) / (2 * e)
    ux = (u(t, x + e, v) - u(t, x - e, v)) / (2 * e)
    uvv = (u(t, x, v + e) - 2 * u(t, x, v) + u(t, x, v - e)) / e ** 2
    rhs = 0.5 * 0.9 * uvv + 1.0 * v * ux
    assert ut == pytest.approx(rhs, rel=1e-5, abs=1e-7)


def test_euler_step_matches_pointwise_formula():
    w = LANGEVIN_32.with_(d=5, ax=-2.0, bx=2.0, av=-2.0, bv=2.0, n_fine=10, drift_sign=-1)
    xs, dx = disc.grid(w.d, w.ax, w.bx)
    vs, dv = disc.grid(w.d, w.av, w.bv)
    u = disc.gaussian_initial(w)                         # (x, v)
    dW = brownian.coarse_increments(w, 0, 1)[0]
    new = np.zeros_like(u)
    g = lambda i, j: u[i, j] if (0 <= i < w.d and 0 <= j < w.d) else 0.0
    for i in range(w.d):
        for j in range(w.d):
            ux = (g(i + 1, j) - g(i - 1, j)) / (2 * dx)
            uv = (g(i, j + 1) - g(i, j - 1)) / (2 * dv)
            uvv = (g(i, j + 1) - 2 * g(i, j) + g(i, j - 1)) / dv ** 2
            new[i, j] = u[i, j] + (-vs[j] * ux + 0.5 * w.a0 * uvv) * w.T + w.s0 * uv * dW
    np.testing.assert_allclose(euler.solve_path(w, 1, 0), new.T, atol=1e-14)


def test_euler_converges_to_the_fine_magnus_solution():
    w = LANGEVIN_32.with_(d=16, n_fine=4000, paths=2)
    ref = magnus.solve(w, 3, 100, [0, 1])
    e = [errors.Err(euler.solve(w, n, [0, 1]), ref) for n in (250, 4000)]
    assert e[1] < e[0] / 2


def test_error_norms():
    assert errors.kappa_range(32, 0) == (0, 32)
    assert errors.kappa_range(32, 1) == (8, 24)
    assert errors.kappa_range(200, 4) == (93, 105)
    rng = np.random.default_rng(0)
    R = rng.uniform(1, 2, size=(3, 8, 8))
    assert errors.Err(1.1 * R, R) == pytest.approx(0.1, rel=1e-13)
    D = R.copy()
    D[:, 2:6, 2:6] += 0.5
    assert errors.AME(D, R, 1) == pytest.approx(0.5, rel=1e-13)
    assert errors.AME(D, R, 0) == pytest.approx(0.5 * 16 / 64, rel=1e-13)
    np.testing.assert_allclose(errors.ME(D, R, 1), 0.5)


def test_moments_of_a_gaussian_grid_function():
    w = LANGEVIN_32.with_(d=160, ax=-10.0, bx=10.0, av=-10.0, bv=10.0, u0_mean=(0.5, -1.0),
                          u0_cov=(1.5, -0.3, 0.8), u0_scale=3.0)
    xs, dx = disc.grid(w.d, w.ax, w.bx)
    vs, dv = disc.grid(w.d, w.av, w.bv)
    U = disc.gaussian_initial(w).T[None]
    m = errors.moments(U, xs, vs, dx, dv)[0]
    np.testing.assert_allclose(m, [3.0, 0.5, -1.0, 1.5, -0.3, 0.8], atol=1e-8)


# ---------------------------------------------------------------- variable coefficients
def _var(d=6, sigma=10 ** -0.5, n_fine=120, c=1.0):
    from workloads import PAPER_VAR
    return PAPER_VAR[0].with_(d=d, s0=sigma, n_fine=n_fine, paths=4, x_profile_c=c, ax=-3.0, bx=3.0,
                              av=-3.0, bv=3.0)


def test_variable_coefficient_deterministic_case_is_exact():
    """sigma = 0 with the x profile: Omega = h B at every order, so K steps give exp(T B) u0."""
    w = _var(d=6, sigma=0.0)
    ops = disc.LangevinOperators(w)
    u0 = disc.vec(disc.gaussian_initial(w))
    exact = sla.expm(w.T * ops.B(w.a0).toarray()) @ u0
    for order, K in ((1, 1), (2, 3), (3, 5)):
        np.testing.assert_allclose(magnus.solve_path(w, order, K, 0).ravel(), exact, rtol=1e-11,
                                   atol=1e-13 * np.abs(exact).max())


def test_variable_coefficient_euler_step_matches_pointwise_formula():
    w = _var(d=5, n_fine=10).with_(ax=-2.0, bx=2.0, av=-2.0, bv=2.0)
    xs, dx = disc.grid(w.d, w.ax, w.bx)
    vs, dv = disc.grid(w.d, w.av, w.bv)
    u = disc.gaussian_initial(w)                         # (x, v)
    dW = brownian.coarse_increments(w, 0, 1)[0]
    new = np.zeros_like(u)
    g = lambda i, j: u[i, j] if (0 <= i < w.d and 0 <= j < w.d) else 0.0
    for i in range(w.d):
        psi = 1.0 + 1.0 / (xs[i] ** 2 + 1.0)             # Eq. coeffsLangevinVar
        for j in range(w.d):
            ux = (g(i + 1, j) - g(i - 1, j)) / (2 * dx)
            uv = (g(i, j + 1) - g(i, j - 1)) / (2 * dv)
            uvv = (g(i, j + 1) - 2 * g(i, j) + g(i, j - 1)) / dv ** 2
            new[i, j] = (u[i, j] + (-vs[j] * ux + 0.5 * w.a0 * psi * uvv) * w.T
                         + w.s0 * math.sqrt(psi) * uv * dW)
    np.testing.assert_allclose(euler.solve_path(w, 1, 0), new.T, atol=1e-14)


def test_variable_coefficient_magnus_and_euler_meet():
    """Two different schemes for the same SPDE: the fine Euler solution approaches the
    order-3 Magnus solution as its step shrinks (Table errorsVar uses fine Euler as reference)."""
    w = _var(d=12, n_fine=4000).with_(ax=-4.0, bx=4.0, av=-4.0, bv=4.0)
    ref = magnus.solve(w, 3, 50, [0, 1])
    e = [errors.Err(euler.solve(w, n, [0, 1]), ref) for n in (250, 4000)]
    assert e[1] < e[0] / 2 and e[1] < 2e-3
    # and the profile matters: the constant-coefficient solution is far away
    ref0 = magnus.solve(w.with_(x_profile=0), 3, 50, [0, 1])
    assert errors.Err(ref0, ref) > 10 * e[1]

"""Pins of the oracle's time-dependent arithmetic against quadrature, the Kolmogorov
equation, the Ito isometry, an ODE solver and a frozen-coefficient fine-step
reference -- none of which shares a formula with the code it checks.

* The closed-form integrals of `oracle/coefficients.py` (alpha_bar, the integral of
  sigma^2, the integral of s alpha, G3) against adaptive quadrature of the
  pointwise profiles a(t) = a0 + a1 sin 2 pi t, sigma(t) = s0 (1 + s1 cos 2 pi t).
* The covariance C_T of the closed-form solution with time-dependent coefficients
  (derived solution of Section 3.1): its a(t) part by the residual of the
  Kolmogorov equation u_t = a(t)/2 u_vv + kappa v u_x at sigma = 0; its sigma(t)^2
  part by the Ito isometry (the mean of the closed form over Brownian paths is the
  sigma = 0 solution with the same a(t)), the covariance of the random shift c_T
  being taken exactly from the fine-grid functionals by linearity.
* The time-dependent order-2 logarithm (the Appendix's Picard step with
  B_t = Bx + alpha(t) Bvv): at sigma = 0 it is the deterministic Magnus expansion
  truncated after its commutator term, fourth order in the step against a
  high-accuracy ODE solver; a wrong G3 weight drops it to second order.
* The stochastic weights G1, G2 and the midpoint-frozen third-order terms: the
  order-3 scheme against the paper's constant-coefficient order-3 formula iterated
  over every fine Brownian cell with the coefficients frozen at the cell midpoint
  (the fine-grid reading of the stochastic integrals), strong order ~2; a wrong G1
  or G2 leaves an O(h) error."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.integrate import quad, solve_ivp

import oracle.brownian as obrownian
from oracle import discretization as disc, explicit, magnus
from oracle.coefficients import Coefficients
from workloads import COEF_TRIG, LANGEVIN_32, LANGEVIN_TRIG_128

QOPTS = dict(epsabs=1e-15, epsrel=1e-14, limit=400)
COEFS = [(1.0, 0.5, 0.5, 0.3), (1.3, -0.7, 0.8, 0.6), (0.6, 0.45, 0.2, -0.9)]
INTERVALS = [(0.0, 0.125), (0.3, 0.05), (0.77, 0.2), (0.9, 1.0), (0.0, 1.0 / 1024)]


@pytest.mark.parametrize("cf", COEFS)
def test_coefficient_integrals_match_adaptive_quadrature(cf):
    c = Coefficients(COEF_TRIG, *cf)
    alpha = lambda t: float(c.alpha(t))
    sig2 = lambda t: float(c.sigma(t)) ** 2
    for t0, h in INTERVALS:
        tol = lambda ref: 1e-13 * max(abs(ref), h)
        ab = quad(alpha, t0, t0 + h, **QOPTS)[0]
        assert abs(float(c.alpha_bar(t0, h)) - ab) <= tol(ab)
        ss = quad(sig2, t0, t0 + h, **QOPTS)[0]
        assert abs(c.sigma_sq_integral(t0, h) - ss) <= tol(ss)
        sa = quad(lambda s: s * alpha(t0 + s), 0.0, h, **QOPTS)[0]
        assert abs(c.s_alpha_integral(t0, h) - sa) <= tol(sa) * h
        # G3 = int_0^h (s alpha(t0 + s) - int_0^s alpha(t0 + r) dr) ds, inner integral by quadrature too
        g3 = quad(lambda s: s * alpha(t0 + s) - quad(alpha, t0, t0 + s, **QOPTS)[0], 0.0, h, **QOPTS)[0]
        # the closed form 2 int s alpha - h alpha_bar cancels terms of size h^2: rounding ~ eps h^2
        assert abs(c.g3(t0, h) - g3) <= 1e-13 * max(abs(g3), h * h)


def test_constant_profiles_reduce_to_products():
    c = Coefficients(COEF_TRIG, 1.2, 0.0, 0.7, 0.0)
    for t0, h in INTERVALS:
        assert float(c.alpha_bar(t0, h)) == pytest.approx(0.6 * h, rel=1e-14)
        assert c.sigma_sq_integral(t0, h) == pytest.approx(0.49 * h, rel=1e-14)
        assert c.g3(t0, h) == pytest.approx(0.0, abs=1e-15)        # s alpha - alpha_bar vanishes


def _trig(**kw):
    base = dict(d=40, kind=COEF_TRIG, a0=1.0, a1=0.6, s0=0.0, s1=0.0, drift_sign=1, u0_mean=(0.2, 0.1),
                u0_cov=(0.6, 0.1, 0.8), n_fine=1024)
    base.update(kw)
    return LANGEVIN_32.with_(**base)


@pytest.mark.parametrize("kappa", [1, -1])
def test_closed_form_with_a_of_t_solves_the_kolmogorov_equation(kappa):
    """sigma = 0: u_t = a(t)/2 u_vv + kappa v u_x, checked at several (t, x, v) by
    central differences of the closed form (its C_T by quadrature of a(t))."""
    w0 = _trig(drift_sign=kappa)
    coef = Coefficients.of(w0)

    def u(t, x, v):
        mean, cov = explicit.terminal_gaussian(w0.with_(T=t), 0)
        return float(disc.gaussian_density(np.array(x), np.array(v), mean, cov, 1.0))

    e = 1e-4
    for t, x, v in ((0.6, 0.3, -0.4), (0.25, -0.2, 0.5), (0.9, 0.1, 0.2)):
        ut = (u(t + e, x, v) - u(t - e, x, v)) / (2 * e)
        ux = (u(t, x + e, v) - u(t, x - e, v)) / (2 * e)
        uvv = (u(t, x, v + e) - 2 * u(t, x, v) + u(t, x, v - e)) / e ** 2
        rhs = 0.5 * float(coef.a(t)) * uvv + kappa * v * ux
        assert ut == pytest.approx(rhs, rel=1e-5, abs=1e-7)
        # and the profile matters: the residual with the mean diffusion a0 is far off
        assert abs(ut - (0.5 * w0.a0 * uvv + kappa * v * ux)) > 100 * abs(ut - rhs)


def _shift_map(w):
    """The random shift c_T = (kappa int omega dt, -omega_T) of the closed form is linear
    in the fine increments; its coefficient rows come from unit increments."""
    rows = np.zeros((w.n_fine, 2))
    orig = obrownian.fine_increments
    try:
        for k in range(w.n_fine):
            e = np.zeros(w.n_fine)
            e[k] = 1.0
            obrownian.fine_increments = lambda ww, p, e=e: e
            f = obrownian.terminal_functionals(w, 0)
            rows[k] = (w.drift_sign * f["int_omega"], -f["omega_T"])
    finally:
        obrownian.fine_increments = orig
    return rows


@pytest.mark.parametrize("kappa", [1, -1])
def test_closed_form_covariance_obeys_the_ito_isometry(kappa):
    """E over paths of N(M m0 + c_T, S + C_T(sigma)) is N(M m0, S + C_T(sigma) + Cov c_T),
    and it must equal the sigma = 0 solution with the same a(t): C_T(sigma) + Cov c_T
    = C_T(0).  Cov c_T = delta sum_k r_k r_k^T exactly for the fine-grid functionals
    (midpoint rule of int sigma^2 m m^T, error O(delta^2))."""
    w = _trig(drift_sign=kappa, s0=0.5, s1=0.3, n_fine=2048)
    R = _shift_map(w)
    cov_shift = (w.T / w.n_fine) * R.T @ R
    cxx, cxv, cvv = explicit.diffusion_cov(w)
    z = explicit.diffusion_cov(w.with_(s0=0.0))
    got = np.array([cxx + cov_shift[0, 0], cxv + cov_shift[0, 1], cvv + cov_shift[1, 1]])
    # (a dropped s1^2 term of sigma(t)^2 would move C_T(sigma)_vv by s0^2 s1^2 T / 2 ~ 1e-2)
    np.testing.assert_allclose(got, z, rtol=1e-6)


def _order_sigma0(g3_scale=1.0):
    w = LANGEVIN_32.with_(d=6, ax=-2.0, bx=2.0, av=-2.0, bv=2.0, kind=COEF_TRIG, a0=1.0, a1=0.8, s0=0.0,
                          s1=0.0, n_fine=64, paths=1)
    ops = disc.LangevinOperators(w)
    coef = Coefficients.of(w)
    Bx, Bvv = ops.Bx.toarray(), ops.Bvv.toarray()
    u0 = disc.vec(disc.gaussian_initial(w, ops.xs, ops.vs))
    sol = solve_ivp(lambda t, u: (Bx + float(coef.alpha(t)) * Bvv) @ u, (0.0, w.T), u0, method="DOP853",
                    rtol=1e-13, atol=1e-16)
    ref = sol.y[:, -1]
    orig = Coefficients.g3
    Coefficients.g3 = lambda self, t0, h: g3_scale * orig(self, t0, h)
    try:
        errs = [np.linalg.norm(magnus.solve_path(w, 2, K, 0).ravel() - ref) / np.linalg.norm(ref)
                for K in (4, 8, 16, 32)]
    finally:
        Coefficients.g3 = orig
    return np.array(errs)


def test_timedep_order2_at_sigma_zero_is_fourth_order():
    """sigma = 0: Y2 = h Bx + alpha_bar Bvv - G3/2 [Bx,Bvv] is the Magnus expansion of
    u' = (Bx + alpha(t) Bvv) u truncated after its commutator term, whose remainder is
    O(h^5) per step: global order 4 against a DOP853 solve at rtol 1e-13."""
    e = _order_sigma0()
    orders = np.log2(e[:-1] / e[1:])
    assert orders[-2:].min() >= 3.5, orders
    assert e[-1] < 1e-7


@pytest.mark.parametrize("scale", [0.0, 2.0])
def test_a_wrong_g3_drops_the_order(scale):
    e = _order_sigma0(scale)
    orders = np.log2(e[:-1] / e[1:])
    assert orders[-1] < 2.5 and e[-1] > 1e-6, orders


NF_STRONG = 1024


_STRONG_CACHE = {}


def _strong_case():
    """The 4 x 4 time-dependent problem and its frozen-coefficient fine reference (cached)."""
    if "case" in _STRONG_CACHE:
        return _STRONG_CACHE["case"]
    w = LANGEVIN_32.with_(d=4, ax=-2.0, bx=2.0, av=-2.0, bv=2.0, kind=COEF_TRIG, a0=1.0, a1=0.5, s0=0.6,
                          s1=0.6, n_fine=NF_STRONG, paths=6)
    ops = disc.LangevinOperators(w)
    coef = Coefficients.of(w)
    Bx, Bvv, A0 = ops.Bx.toarray(), ops.Bvv.toarray(), ops.A0.toarray()
    u0 = disc.vec(disc.gaussian_initial(w, ops.xs, ops.vs))
    delta = w.T / w.n_fine
    refs = []
    for p in range(w.paths):
        dw = obrownian.fine_increments(w, p)
        U = u0.copy()
        for k in range(w.n_fine):
            tm = (k + 0.5) * delta
            B = sp.csr_matrix(Bx + float(coef.alpha(tm)) * Bvv)
            A = sp.csr_matrix(float(coef.sigma(tm)) * A0)
            x = dw[k]      # on one cell W~(s) = x s / delta
            Y = magnus.omega_const(B, A, delta, x, delta * x / 2, delta * x * x / 3, delta * delta * x / 3, 3)
            U = sla.expm(Y.toarray()) @ U
        refs.append(U)
    _STRONG_CACHE["case"] = (w, refs)
    return w, refs


def _strong(order, plant=None):
    """RMS over 6 paths of the relative error of the time-dependent scheme at K = 16, 32, 64
    against the constant-coefficient order-3 formula iterated over all NF_STRONG fine cells
    with a, sigma frozen at each cell's midpoint (cell functionals of the linear path)."""
    w, refs = _strong_case()
    orig = obrownian.interval_functionals
    if plant:
        key, scale = plant

        def planted(*a, **k):
            r = dict(orig(*a, **k))
            r[key] = scale * r[key]
            return r
        obrownian.interval_functionals = planted
        magnus.interval_functionals = planted
    try:
        out = []
        for K in (16, 32, 64):
            e = [np.linalg.norm(magnus.solve_path(w, order, K, p).ravel() - refs[p]) / np.linalg.norm(refs[p])
                 for p in range(w.paths)]
            out.append(math.sqrt(np.mean(np.square(e))))
    finally:
        obrownian.interval_functionals = orig
        magnus.interval_functionals = orig
    return np.array(out)


def test_timedep_order3_converges_fast_to_the_frozen_coefficient_fine_solution():
    e3 = _strong(3)
    assert e3[0] / e3[-1] >= 8.0, e3           # measured ~17 (strong order ~2)
    assert e3[-1] < 2e-5, e3
    e2 = _strong(2)
    assert e2[-1] > 10 * e3[-1]                # order 2 lags (strong order ~1)


@pytest.mark.parametrize("plant", [("G1", 0.0), ("G2", 0.0), ("G1", 1.2), ("G2", 1.2)])
def test_a_wrong_stochastic_weight_is_caught(plant):
    e3 = _strong(3, plant)
    assert e3[0] / e3[-1] < 8.0 or e3[-1] >= 2e-5, e3


def test_bench_coefficient_set_is_covered():
    """The time-dependent benchmark coefficients (a1 = 0.5, s1 = 0.3) are among the sets above."""
    w = LANGEVIN_TRIG_128
    assert (w.a0, w.a1, w.s0, w.s1) == COEFS[0]

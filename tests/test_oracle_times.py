"""Pins of the oracle's interval functionals and of its solutions at several output
times inside the Magnus sub-intervals (Section 3, "Implementation")."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import brownian, discretization as disc, magnus
from workloads import COEF_TRIG, LANGEVIN_32


def _w(**kw):
    base = dict(d=6, ax=-3.0, bx=3.0, av=-3.0, bv=3.0, n_fine=240, paths=2)
    base.update(kw)
    return LANGEVIN_32.with_(**base)


@pytest.mark.parametrize("kind", [0, COEF_TRIG])
def test_interval_functionals_compose_across_a_split(kind):
    """Splitting [c0, c2) at c1 with the Brownian motion restarted at c1: the increments add,
    and the integrals pick up the closed-form shift terms of the restart."""
    w = _w(kind=kind, a1=0.4, s1=0.3)
    delta = w.T / w.n_fine
    c0, c1, c2 = 17, 70, 131
    F = brownian.interval_functionals(w, 1, c0, c2)
    a = brownian.interval_functionals(w, 1, c0, c1)
    b = brownian.interval_functionals(w, 1, c1, c2)
    t1, h2 = (c1 - c0) * delta, (c2 - c1) * delta          # offset of the split, length of part two
    W1 = a["dW"]
    np.testing.assert_allclose(F["dW"], W1 + b["dW"], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(F["om"], a["om"] + b["om"], rtol=1e-13, atol=1e-15)
    # int_0^h W = int_0^t1 W + int_t1^h (W1 + W') = I1a + W1 h2 + I1b
    np.testing.assert_allclose(F["I1"], a["I1"] + W1 * h2 + b["I1"], rtol=1e-12, atol=1e-15)
    # int W^2 = I2a + int (W1 + W')^2 = I2a + W1^2 h2 + 2 W1 I1b + I2b
    np.testing.assert_allclose(F["I2"], a["I2"] + W1 * W1 * h2 + 2 * W1 * b["I1"] + b["I2"], rtol=1e-12,
                               atol=1e-15)
    # int s W with s = t1 + s': I3a + W1 (t1 h2 + h2^2/2) + t1 I1b + I3b
    np.testing.assert_allclose(F["I3"], a["I3"] + W1 * (t1 * h2 + 0.5 * h2 * h2) + t1 * b["I1"] + b["I3"],
                               rtol=1e-12, atol=1e-15)
    # int omega ds = Jom_a + om_a h2 + Jom_b
    np.testing.assert_allclose(F["Jom"], a["Jom"] + a["om"] * h2 + b["Jom"], rtol=1e-12, atol=1e-15)


def test_outputs_at_step_boundaries_equal_shorter_solves():
    """Output time t_n (a sub-interval end) equals the iterated solution of the same path on
    [0, t_n] (same fine increments, n steps)."""
    w = _w(s0=0.6)
    K, L = 4, 60
    got = magnus.solve_times(w, 3, K, 0, [L, 2 * L, 4 * L])
    for n, g in zip((1, 2, 4), got):
        wn = w.with_(T=w.T * n / K, n_fine=n * L)
        np.testing.assert_allclose(g, magnus.solve_path(wn, 3, n, 0), rtol=1e-11, atol=1e-13)


def test_outputs_inside_steps_are_exact_when_sigma_is_zero():
    """sigma = 0: every output time t has u(t) = exp(t B) u0 exactly."""
    w = _w(s0=0.0)
    ops = disc.LangevinOperators(w)
    u0 = disc.vec(disc.gaussian_initial(w))
    cells = [7, 60, 61, 100, 239, 240]
    got = magnus.solve_times(w, 2, 4, 1, cells)
    for c, g in zip(cells, got):
        ref = sla.expm(c * w.T / w.n_fine * ops.B(w.a0).toarray()) @ u0
        np.testing.assert_allclose(g.ravel(), ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def test_output_times_must_be_on_the_grid():
    with pytest.raises(ValueError):
        magnus.solve_times(_w(), 2, 4, 0, [0])
    with pytest.raises(ValueError):
        magnus.solve_times(_w(), 2, 4, 0, [241])

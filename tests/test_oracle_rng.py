"""Pins of the oracle's Philox4x32-10 generator and Brownian functionals."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import brownian, philox
from workloads import COEF_TRIG, LANGEVIN_32, LANGEVIN_TRIG_128

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    got = philox.philox4x32(tuple(np.uint64(c) for c in ctr), tuple(np.uint64(k) for k in key))
    assert [int(g) for g in got] == out


def test_philox_is_a_vectorised_pure_function():
    j = np.arange(7)
    a = philox.brownian_words(123, 5, j)
    b = [philox.brownian_words(123, 5, [i]) for i in j]
    for w in range(4):
        assert [int(x) for x in a[w]] == [int(bb[w][0]) for bb in b]
    # path and seed enter the counter and key: changing either changes the words
    assert int(philox.brownian_words(124, 5, [0])[0][0]) != int(a[0][0])
    assert int(philox.brownian_words(123, 6, [0])[0][0]) != int(a[0][0])
    # the high half of a 64-bit path index lands in counter word 2
    hi = philox.brownian_words(1, (1 << 32) + 3, [0])
    lo = philox.brownian_words(1, 3, [0])
    assert int(hi[0][0]) != int(lo[0][0])


def test_uniform52_endpoints():
    assert philox.uniform52(0, 0) == 0.5 * 2.0 ** -52
    top = philox.uniform52(0xFFFFFFFF, 0xFFFFFFFF)
    assert top < 1.0 and top == 1.0 - 0.5 * 2.0 ** -52
    # bits 12..63 of hi:lo are used, the low 12 bits of lo are dropped
    assert philox.uniform52(0xFFF, 0) == philox.uniform52(0, 0)
    assert philox.uniform52(0x1000, 0) == 1.5 * 2.0 ** -52
    assert philox.uniform52(0, 1) == (2.0 ** 20 + 0.5) * 2.0 ** -52


def test_normals_are_standard_normal():
    z = np.concatenate([philox.standard_normals(99, p, 20000) for p in range(5)])
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(z)) < 5 * math.sqrt(24.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # Box-Muller pairs: z_{2j}^2 + z_{2j+1}^2 = -2 log u1 ~ Exp(1/2)
    r2 = z[0::2] ** 2 + z[1::2] ** 2
    assert stats.kstest(r2, "expon", args=(0, 2.0)).pvalue > 1e-4


def _cell_integrals_bruteforce(wn, delta, sub=2000):
    """int W, int W^2, int s W of the piecewise-linear interpolant by fine midpoint sums."""
    L = len(wn) - 1
    t = (np.arange(L * sub) + 0.5) / sub                     # cell units
    k = np.floor(t).astype(int)
    frac = t - k
    W = wn[k] * (1 - frac) + wn[k + 1] * frac
    s = t * delta
    ds = delta / sub
    return np.sum(W) * ds, np.sum(W * W) * ds, np.sum(s * W) * ds


def test_step_functionals_match_the_interpolant_integrals():
    w = LANGEVIN_32.with_(n_fine=64)
    K = 4
    f = brownian.step_functionals(w, 3, K)
    dw = brownian.fine_increments(w, 3).reshape(K, -1)
    delta = w.T / w.n_fine
    for n in range(K):
        wn = np.concatenate(([0.0], np.cumsum(dw[n])))
        i1, i2, i3 = _cell_integrals_bruteforce(wn, delta)
        assert f["dW"][n] == pytest.approx(wn[-1], abs=1e-15)
        assert f["I1"][n] == pytest.approx(i1, rel=1e-6, abs=1e-12)
        assert f["I2"][n] == pytest.approx(i2, rel=1e-6, abs=1e-12)
        assert f["I3"][n] == pytest.approx(i3, rel=1e-6, abs=1e-12)


def test_ito_integration_by_parts_and_constant_reduction():
    """Lemma Ito1 (Eq. Ito1a, p = 1, q = 0): int_0^h s dW = h W_h - int_0^h W ds.

    With constant sigma and alpha the time-dependent functionals must reduce to
    omega = sigma W, G1 = sigma (2 I1 - h dW), G2 = alpha sigma (2 I1 - h dW)."""
    w = LANGEVIN_32.with_(n_fine=800, s0=0.7, a0=1.3)
    K = 8
    h = w.T / K
    f = brownian.step_functionals(w, 11, K)
    dw = brownian.fine_increments(w, 11).reshape(K, -1)
    delta = w.T / w.n_fine
    s_mid = delta * (np.arange(dw.shape[1]) + 0.5)
    for n in range(K):
        lhs = np.sum(s_mid * dw[n])
        assert lhs == pytest.approx(h * f["dW"][n] - f["I1"][n], abs=1e-14)
    np.testing.assert_allclose(f["om"], 0.7 * f["dW"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(f["Jom"], 0.7 * f["I1"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(f["G1"], 0.7 * (2 * f["I1"] - h * f["dW"]), rtol=0, atol=1e-14)
    np.testing.assert_allclose(f["G2"], 0.65 * 0.7 * (2 * f["I1"] - h * f["dW"]), rtol=0, atol=1e-14)


def test_functional_moments():
    """E dW^2 = h, E I1 dW = h^2/2, E I1^2 = h^3/3, E I2 = h^2/2, E I3 dW = h^3/3."""
    w = LANGEVIN_32.with_(n_fine=40, T=1.0)
    K = 4
    h = w.T / K
    F = [brownian.step_functionals(w, p, K) for p in range(1500)]
    dW = np.concatenate([f["dW"] for f in F])
    I1 = np.concatenate([f["I1"] for f in F])
    I2 = np.concatenate([f["I2"] for f in F])
    I3 = np.concatenate([f["I3"] for f in F])
    n = dW.size

    def close(x, target, tol_sd=5):
        assert abs(x.mean() - target) < tol_sd * x.std() / math.sqrt(n), (x.mean(), target)

    close(dW, 0.0)
    close(dW * dW, h)
    close(I1 * dW, h * h / 2)
    # The interpolant misses an independent Brownian bridge on each fine cell,
    # which removes delta^3/12 (resp. delta^2/6) per cell from E I1^2 (resp. E I2).
    delta = w.T / w.n_fine
    close(I1 * I1, h ** 3 / 3 - h * delta ** 2 / 12)
    close(I2, h * h / 2 - h * delta / 6)
    close(I3 * dW, h ** 3 / 3)


def test_steps_tile_the_path():
    w = LANGEVIN_TRIG_128.with_(n_fine=256, d=8)
    assert w.kind == COEF_TRIG
    f4 = brownian.step_functionals(w, 2, 4)
    term = brownian.terminal_functionals(w, 2)
    assert np.sum(f4["dW"]) == pytest.approx(term["W_T"], abs=1e-14)
    assert np.sum(f4["om"]) == pytest.approx(term["omega_T"], abs=1e-14)
    # int_0^T omega dt = sum_n (h omega(t_n) + int_step omega~)
    h = w.T / 4
    om_start = np.concatenate(([0.0], np.cumsum(f4["om"])[:-1]))
    assert np.sum(h * om_start + f4["Jom"]) == pytest.approx(term["int_omega"], abs=1e-14)
    with pytest.raises(ValueError):
        brownian.step_functionals(w, 0, 3)

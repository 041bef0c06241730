"""Pins of the surrogate oracle (MLP, bfloat16 rounding, Adam, POD, features)."""
import math

import numpy as np
import pytest
import torch

from oracle import brownian, surrogate as sg
from workloads import LANGEVIN_TRIG_128


def test_bf16_rounding_matches_torch_and_ties_to_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-20, 20, size=2000),
                        [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, 65504.0, -3.3e38]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(sg.to_bf16(x), want)
    assert sg.to_bf16(1 + 2 ** -8) == 1.0                  # tie -> even
    assert sg.to_bf16(1 + 3 * 2 ** -9) == 1 + 2 ** -7


def test_gelu_identities():
    x = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(sg.gelu(x) - sg.gelu(-x), x, atol=1e-14)
    assert sg.gelu(0.0) == 0.0
    e = 1e-6
    np.testing.assert_allclose(sg.gelu_prime(x), (sg.gelu(x + e) - sg.gelu(x - e)) / (2 * e), atol=1e-8)


def test_backprop_against_finite_differences():
    rng = np.random.default_rng(1)
    params = sg.init_params([5, 7, 6, 3], seed=2)
    params = [(W, rng.normal(size=b.shape) * 0.1) for W, b in params]
    X = rng.normal(size=(9, 5))
    C = rng.normal(size=(9, 3))
    loss, grads = sg.loss_and_grads(params, X, C)
    e = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for idx in list(np.ndindex(arr.shape))[:12]:
                old = arr[idx]
                arr[idx] = old + e
                lp, _ = sg.loss_and_grads(params, X, C)
                arr[idx] = old - e
                lm, _ = sg.loss_and_grads(params, X, C)
                arr[idx] = old
                assert g[idx] == pytest.approx((lp - lm) / (2 * e), rel=1e-6, abs=1e-9)


def test_bf16_mode_only_rounds_the_stored_operands():
    rng = np.random.default_rng(3)
    params = [(sg.to_bf16(W), b) for W, b in sg.init_params([6, 8, 4], seed=4)]
    X = sg.to_bf16(rng.normal(size=(5, 6)))
    C = rng.normal(size=(5, 4))
    l64, g64 = sg.loss_and_grads(params, X, C, bf16=False)
    l16, g16 = sg.loss_and_grads(params, X, C, bf16=True)
    assert l16 == pytest.approx(l64, rel=2e-2)
    for (a, b), (c, d) in zip(g64, g16):
        assert np.linalg.norm(a - c) <= 3e-2 * np.linalg.norm(a)


def test_adam_first_step_is_a_normalised_step():
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -4.0]]), np.array([1e-3]))]
    st = sg.adam_state(params)
    new = sg.adam_step(params, grads, st, lr=0.01, t=1)
    # t = 1: mhat = g, vhat = g^2 -> w - lr g / (|g| + eps)
    np.testing.assert_allclose(new[0][0], [[1.0 - 0.01 * 0.3 / (0.3 + 1e-8), -2.0 + 0.01 * 4.0 / (4.0 + 1e-8)]])
    np.testing.assert_allclose(new[0][1], [0.5 - 0.01 * 1e-3 / (1e-3 + 1e-8)])


def test_pod_reproduces_low_rank_data():
    rng = np.random.default_rng(5)
    U, V = rng.normal(size=(40, 3)), rng.normal(size=(3, 25))
    mean = rng.normal(size=25)
    S = U @ V + mean
    m, Phi, sv = sg.pod(S, 3)
    np.testing.assert_allclose(Phi.T @ Phi, np.eye(3), atol=1e-12)
    c = sg.pod_coefficients(S, m, Phi)
    np.testing.assert_allclose(m + c @ Phi.T, S, atol=1e-10)
    assert sv[3] < 1e-10 * sv[0]


def test_features_are_the_scaled_step_functionals():
    w = LANGEVIN_TRIG_128.with_(n_fine=512, paths=3)
    K = 16
    h = w.T / K
    X = sg.features(w, K, [0, 1, 2])
    assert X.shape == (3, 48)
    dw = brownian.fine_increments(w, 1).reshape(K, -1)
    delta = w.T / w.n_fine
    s_mid = delta * (np.arange(dw.shape[1]) + 0.5)
    s1, s3 = math.sqrt(h), h ** 1.5 / math.sqrt(3)
    np.testing.assert_allclose(X[1, 0::3], dw.sum(axis=1) / s1, atol=1e-12)
    np.testing.assert_allclose(X[1, 2::3], (dw * s_mid).sum(axis=1) / s3, atol=1e-9)   # int s dW

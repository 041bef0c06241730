"""Surrogate oracle: POD of terminal solutions and an MLP from Brownian functionals.

Not part of the paper: a learned stand-in for the Magnus solver maps the
per-step Brownian functionals of a path to the POD coefficients of its
terminal solution u_T.  This module is the plain CPU reference of every
computation the GPU surrogate performs:

  features   x = [dW_k / sqrt(h), I1_k / s3, (h dW_k - I1_k) / s3]_k,  s3 = h^1.5/sqrt(3)
             (dW, int W ds and int s dW of each of K steps, each scaled to unit
             variance; int s dW = h dW - int W ds by Ito integration by parts)
  POD        mean m and the leading r right singular vectors Phi of S - m
             (S: snapshots x grid points); coefficients c = (u - m) Phi
  MLP        z_l = h_{l-1} W_l^T + b_l, h_l = GELU(z_l) for hidden layers, output z_L;
             GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2
  loss       L = (1/B) sum_b sum_j (zhat_bj - c_bj)^2
  Adam       m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, w -= lr mhat / (sqrt(vhat) + eps)

With bf16=True the forward/backward passes round to bfloat16 (round to
nearest even) exactly where the GPU stores bfloat16: the inputs, the weights,
the hidden activations h_l and the backward GEMM operands dz_l; all other
arithmetic is float64 (the GPU accumulates in float32).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from .brownian import step_functionals


# ---------------------------------------------------------------- bfloat16 rounding

def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


# ---------------------------------------------------------------- features

def feature_scales(h):
    return math.sqrt(h), h ** 1.5 / math.sqrt(3.0)


def features(w, K: int, paths):
    """(len(paths), 3K) feature matrix of the given local path indices."""
    h = w.T / K
    s1, s3 = feature_scales(h)
    rows = []
    for p in paths:
        f = step_functionals(w, p, K)
        dW, I1 = f["dW"], f["I1"]
        rows.append(np.stack([dW / s1, I1 / s3, (h * dW - I1) / s3], axis=1).ravel())
    return np.array(rows)


# ---------------------------------------------------------------- POD

def pod(S, r):
    """Mean and the leading r right singular vectors (columns) of S - mean."""
    S = np.asarray(S, dtype=np.float64)
    m = S.mean(axis=0)
    _, sv, Vt = np.linalg.svd(S - m, full_matrices=False)
    return m, Vt[:r].T, sv


def pod_coefficients(S, m, Phi):
    return (np.asarray(S, dtype=np.float64) - m) @ Phi


# ---------------------------------------------------------------- MLP

def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_prime(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def init_params(sizes, seed=0):
    """He-style initialisation; params = [(W_l (out x in), b_l), ...]."""
    rng = np.random.default_rng(seed)
    return [(rng.normal(size=(o, i)) * math.sqrt(2.0 / i), np.zeros(o)) for i, o in zip(sizes[:-1], sizes[1:])]


def forward(params, X, bf16=False):
    """Returns the output and the cache (inputs of each layer, pre-activations)."""
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    h = r(X)
    cache = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ r(W).T + b
        cache.append((h, z))
        h = r(gelu(z)) if l < L - 1 else z
    return h, cache


def loss_and_grads(params, X, C, bf16=False):
    """L = mean_b sum_j (out - C)^2 and its gradients [(dW_l, db_l), ...]."""
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    out, cache = forward(params, X, bf16)
    B = X.shape[0]
    diff = out - C
    loss = float(np.sum(diff * diff) / B)
    g = 2.0 * diff / B                         # dL/dz of the output layer
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        h, z = cache[l]
        W = r(params[l][0])
        if l < len(params) - 1:
            g = g * gelu_prime(z)              # dL/dz_l from dL/dh_l
        gq = r(g)
        grads[l] = (gq.T @ h, g.sum(axis=0))
        if l > 0:
            g = gq @ W                         # dL/dh_{l-1}
    return loss, grads


def adam_step(params, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t = 1, 2, ...); state = [(mW, vW, mb, vb), ...] updated in place."""
    new = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        mW, vW, mb, vb = state[l]
        mW[:] = b1 * mW + (1 - b1) * gW
        vW[:] = b2 * vW + (1 - b2) * gW * gW
        mb[:] = b1 * mb + (1 - b1) * gb
        vb[:] = b2 * vb + (1 - b2) * gb * gb
        c1, c2 = 1 - b1 ** t, 1 - b2 ** t
        new.append((W - lr * (mW / c1) / (np.sqrt(vW / c2) + eps), b - lr * (mb / c1) / (np.sqrt(vb / c2) + eps)))
    return new


def adam_state(params):
    return [(np.zeros_like(W), np.zeros_like(W), np.zeros_like(b), np.zeros_like(b)) for W, b in params]

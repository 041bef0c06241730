"""Learned surrogate: features, BF16 MLP forward/backward and Adam against the
CPU oracle, the randomized POD against an exact SVD, training, and serving
with the Magnus audit and fallback."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from oracle import surrogate as sg  # noqa: E402
from workloads import LANGEVIN_TRIG_128  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2207_09776_b300 import build
    build.build()
    msk.load_library()


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def bf16_tensor(x):
    return torch.tensor(np.asarray(x, np.float32), device="cuda").to(torch.bfloat16)


def np64(t):
    return t.float().cpu().numpy().astype(np.float64)


def set_random_params(s, dims, seed, bias_scale=0.1):
    """Random weights/biases written through the flat layout; returns them as float64 lists."""
    rng = np.random.default_rng(seed)
    layout = msk.msk_surrogate_param_layout(s, len(dims) - 2)
    flat = np.zeros(msk.msk_surrogate_num_params(s), np.float32)
    params = []
    for l, (ow, ob) in enumerate(layout):
        fin, fout = dims[l], dims[l + 1]
        W = (rng.normal(size=(fout, fin)) * math.sqrt(2.0 / fin)).astype(np.float32)
        b = (rng.normal(size=fout) * bias_scale).astype(np.float32)
        flat[ow:ow + W.size] = W.ravel()
        flat[ob:ob + fout] = b
        params.append((W.astype(np.float64), b.astype(np.float64)))
    msk.msk_surrogate_set_params(s, torch.tensor(flat, device="cuda"))
    return params, layout


def unflatten(flat, layout, dims):
    out = []
    for l, (ow, ob) in enumerate(layout):
        fin, fout = dims[l], dims[l + 1]
        out.append((flat[ow:ow + fin * fout].reshape(fout, fin).astype(np.float64),
                    flat[ob:ob + fout].astype(np.float64)))
    return out


def make(w, **cfg):
    solver = msk.Solver(w)
    s = msk.msk_surrogate_create(solver.ctx, **cfg)
    return solver, s


# ------------------------------------------------------------------ features

@pytest.mark.parametrize("n_fine,path0", [(720, 3), (16384, 0)])
def test_features_match_the_oracle(n_fine, path0):
    """K = 16 substeps; 720 fine cells give 45 per substep (Philox pairs straddle substeps)."""
    w = LANGEVIN_TRIG_128.with_(d=64, n_fine=n_fine)
    solver, s = make(w, steps=16, rank=4, hidden=64, layers=1, train_batch=64, infer_batch=64)
    P = 5
    X = torch.empty(P, 48, dtype=torch.bfloat16, device="cuda")
    msk.msk_surrogate_features(s, path0, P, X)
    got = np64(X)
    want = sg.to_bf16(sg.features(w, 16, range(path0, path0 + P)))
    # single-precision normals and sums: at most one bf16 rounding step apart
    assert np.all(np.abs(got - want) <= 2.0 ** -7 * np.abs(want) + 1e-30)
    assert np.mean(got == want) >= 0.97
    msk.msk_surrogate_destroy(s)
    solver.close()


# ------------------------------------------------------------------ MLP forward / backward / Adam

@pytest.mark.parametrize("dims,B", [([48, 64, 64, 8], 300), ([48, 512, 512, 512, 512, 64], 4096)])
def test_forward_and_gradients_match_the_bf16_oracle(dims, B):
    """Gradients of L = (1/B) sum (out - C)^2 against the oracle with the same
    bfloat16 rounding points (inputs, weights, hidden activations, dz)."""
    w = LANGEVIN_TRIG_128.with_(d=32, n_fine=1024)
    solver, s = make(w, steps=16, rank=dims[-1], hidden=dims[1], layers=len(dims) - 2, train_batch=B,
                     infer_batch=1000)
    params, layout = set_random_params(s, dims, seed=11)
    rng = np.random.default_rng(12)
    X = sg.to_bf16(rng.normal(size=(B, dims[0])))
    C = rng.normal(size=(B, dims[-1])).astype(np.float32).astype(np.float64)
    Xd, Cd = bf16_tensor(X), torch.tensor(C, dtype=torch.float32, device="cuda")
    out = torch.empty(B, dims[-1], device="cuda")
    msk.msk_surrogate_forward(s, Xd, B, out)
    loss = torch.empty(1, device="cuda")
    grads = torch.empty(msk.msk_surrogate_num_params(s), device="cuda")
    msk.msk_surrogate_loss_grads(s, Xd, Cd, B, loss, grads)
    torch.cuda.synchronize()
    want_out, _ = sg.forward(params, X, bf16=True)
    want_loss, want_grads = sg.loss_and_grads(params, X, C, bf16=True)
    assert rel(out.cpu().numpy(), want_out) <= 1e-3
    assert float(loss) == pytest.approx(want_loss, rel=1e-4)
    got = unflatten(grads.cpu().numpy(), layout, dims)
    for (gW, gb), (wW, wb) in zip(got, want_grads):
        assert rel(gW, wW) <= 3e-3
        assert rel(gb, wb) <= 3e-3
    # the bf16 rounding points matter: the unrounded float64 gradients are further away
    _, g64 = sg.loss_and_grads(params, X, C, bf16=False)
    assert rel(got[0][0], g64[0][0]) > 2 * rel(got[0][0], want_grads[0][0])
    msk.msk_surrogate_sync_status(s)
    msk.msk_surrogate_destroy(s)
    solver.close()


@pytest.mark.parametrize("B", [6000, 40000])
def test_forward_on_large_batches_matches_the_oracle(B):
    """Large batches run the 128- and 256-column tensor-core tiles; sampled rows
    (including the ragged last tile) against the bf16 oracle."""
    dims = [48, 512, 512, 64]
    w = LANGEVIN_TRIG_128.with_(d=32, n_fine=1024)
    solver, s = make(w, steps=16, rank=64, hidden=512, layers=2, train_batch=64, infer_batch=B)
    params, _ = set_random_params(s, dims, seed=13)
    rng = np.random.default_rng(14)
    X = sg.to_bf16(rng.normal(size=(B, 48)))
    out = torch.empty(B, 64, device="cuda")
    msk.msk_surrogate_forward(s, bf16_tensor(X), B, out)
    torch.cuda.synchronize()
    rows = np.concatenate([rng.choice(B - 200, 56, replace=False), np.arange(B - 8, B)])
    want, _ = sg.forward(params, X[rows], bf16=True)
    assert rel(out.cpu().numpy()[rows], want) <= 1e-3
    msk.msk_surrogate_sync_status(s)
    msk.msk_surrogate_destroy(s)
    solver.close()


def test_adam_steps_match_the_oracle():
    dims = [48, 64, 64, 8]
    B = 200
    w = LANGEVIN_TRIG_128.with_(d=32, n_fine=1024)
    solver, s = make(w, steps=16, rank=8, hidden=64, layers=2, train_batch=B, infer_batch=256)
    params, layout = set_random_params(s, dims, seed=21)
    rng = np.random.default_rng(22)
    Xd = bf16_tensor(rng.normal(size=(B, 48)))
    Cd = torch.tensor(rng.normal(size=(B, 8)), dtype=torch.float32, device="cuda")
    state = sg.adam_state(params)
    n = msk.msk_surrogate_num_params(s)
    grads, flat = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    cur = params
    for t in (1, 2):
        msk.msk_surrogate_loss_grads(s, Xd, Cd, B, None, grads)
        msk.msk_surrogate_adam_step(s, 3e-3)
        msk.msk_surrogate_get_params(s, flat)
        torch.cuda.synchronize()
        g = unflatten(grads.cpu().numpy(), layout, dims)
        cur = sg.adam_step(cur, g, state, lr=3e-3, t=t)
        got = unflatten(flat.cpu().numpy(), layout, dims)
        for (a, b), (c, d) in zip(got, cur):
            np.testing.assert_allclose(a, c, rtol=1e-5, atol=1e-6)
            np.testing.assert_allclose(b, d, rtol=1e-5, atol=1e-6)
    msk.msk_surrogate_destroy(s)
    solver.close()


def test_loss_grads_rejects_bad_batches():
    w = LANGEVIN_TRIG_128.with_(d=32, n_fine=1024)
    solver, s = make(w, steps=16, rank=8, hidden=64, layers=1, train_batch=16, infer_batch=16)
    X = torch.zeros(32, 48, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(32, 8, device="cuda")
    with pytest.raises(msk.MskError):
        msk.msk_surrogate_loss_grads(s, X, C, 17)           # above train_batch
    with pytest.raises(msk.MskError):
        msk.msk_surrogate_decode(s, C, 4, torch.empty(4, 32, 32, device="cuda"))   # no POD yet
    with pytest.raises(msk.MskError):
        msk.msk_surrogate_create(solver.ctx, steps=7)       # 7 does not divide n_fine
    with pytest.raises(msk.MskError):
        msk.msk_surrogate_create(solver.ctx, steps=16, rank=65)
    msk.msk_surrogate_destroy(s)
    solver.close()


# ------------------------------------------------------------------ POD

def _spectrum_data(N, n, modes, ratio, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.normal(size=(N, modes)))
    V, _ = np.linalg.qr(rng.normal(size=(n, modes)))
    sv = ratio ** np.arange(modes)
    mean = rng.normal(size=n) * 0.1
    return ((U * sv) @ V.T + mean).astype(np.float32)


def _signed(Phi_cols):
    """Oracle modes (columns) with the library's sign convention (largest |entry| positive)."""
    P = Phi_cols.T.copy()
    for j in range(P.shape[0]):
        if P[j, np.argmax(np.abs(P[j]))] < 0:
            P[j] = -P[j]
    return P


def test_pod_matches_the_svd_and_round_trips():
    w = LANGEVIN_TRIG_128.with_(d=64, n_fine=1024)
    r = 16
    solver, s = make(w, steps=16, rank=r, hidden=64, layers=1, train_batch=64, infer_batch=64)
    N, n = 600, 64 * 64
    S = _spectrum_data(N, n, 40, 0.8, seed=31)
    Sd = torch.tensor(S, device="cuda")
    sv = msk.msk_surrogate_fit_pod(s, Sd, N)
    m, Phi, sv_o = sg.pod(S, r)
    mean, phi = torch.empty(n, device="cuda"), torch.empty(r, n, device="cuda")
    scale = msk.msk_surrogate_get_pod(s, mean, phi)
    np.testing.assert_allclose(mean.cpu().numpy(), m, atol=1e-6 * np.abs(S).max())
    np.testing.assert_allclose(sv[:r], sv_o[:r], rtol=1e-4)
    want = _signed(Phi)
    got = phi.cpu().numpy().astype(np.float64)
    for j in range(r):
        assert np.linalg.norm(got[j] - want[j]) <= 1e-3
    assert scale == pytest.approx(math.sqrt(np.sum(sv_o[:r] ** 2) / (N * r)), rel=1e-4)
    # coefficients and the decode round trip (rank-r reconstruction)
    C = torch.empty(N, r, device="cuda")
    msk.msk_surrogate_project(s, Sd, N, C)
    np.testing.assert_allclose(C.cpu().numpy(), (S - m) @ want.T / scale, atol=1e-4 * np.abs(C.cpu().numpy()).max())
    U = torch.empty(N, n, device="cuda")
    msk.msk_surrogate_decode(s, C, N, U)
    torch.cuda.synchronize()
    recon = m + (S - m) @ Phi @ Phi.T
    assert rel(U.cpu().numpy(), recon) <= 1e-5
    # set_pod / get_pod round trip
    s2 = msk.msk_surrogate_create(solver.ctx, steps=16, rank=r, hidden=64, layers=1, train_batch=64, infer_batch=64)
    msk.msk_surrogate_set_pod(s2, mean, phi, scale)
    U2 = torch.empty(N, n, device="cuda")
    msk.msk_surrogate_decode(s2, C, N, U2)
    torch.cuda.synchronize()
    assert rel(U2.cpu().numpy(), U.cpu().numpy()) <= 1e-6
    msk.msk_surrogate_destroy(s2)
    msk.msk_surrogate_destroy(s)
    solver.close()


def test_pod_of_rank_deficient_snapshots():
    """10 snapshots centred have rank 9 < r = 16: nine resolved modes, the rest zero."""
    w = LANGEVIN_TRIG_128.with_(d=32, n_fine=1024)
    solver, s = make(w, steps=16, rank=16, hidden=64, layers=1, train_batch=64, infer_batch=64)
    S = _spectrum_data(10, 1024, 10, 0.8, seed=32)
    sv = msk.msk_surrogate_fit_pod(s, torch.tensor(S, device="cuda"), 10)
    m, Phi, sv_o = sg.pod(S, 9)
    phi = torch.empty(16, 1024, device="cuda")
    msk.msk_surrogate_get_pod(s, None, phi)
    got = phi.cpu().numpy().astype(np.float64)
    want = _signed(Phi)
    for j in range(9):
        assert np.linalg.norm(got[j] - want[j]) <= 1e-3
    assert np.all(got[9:] == 0)
    np.testing.assert_allclose(sv[:9], sv_o[:9], rtol=1e-4)
    with pytest.raises(msk.MskError):
        msk.msk_surrogate_fit_pod(s, torch.ones(20, 1024, device="cuda"), 20)   # no variation
    msk.msk_surrogate_destroy(s)
    solver.close()


# ------------------------------------------------------------------ training and serving

SMALL = LANGEVIN_TRIG_128.with_(d=64, n_fine=1024)
N_TRAIN = 4096


@pytest.fixture(scope="module")
def trained():
    solver, s = make(SMALL, steps=16, rank=16, hidden=128, layers=2, train_batch=512, infer_batch=1000,
                     ref_order=2, ref_steps=4, init_seed=7)
    n = SMALL.d ** 2
    U = torch.empty(N_TRAIN, n, device="cuda")
    msk.msk_surrogate_reference(s, 0, N_TRAIN, U)
    msk.msk_surrogate_fit_pod(s, U, N_TRAIN)
    C = torch.empty(N_TRAIN, 16, device="cuda")
    msk.msk_surrogate_project(s, U, N_TRAIN, C)
    X = torch.empty(N_TRAIN, 48, dtype=torch.bfloat16, device="cuda")
    msk.msk_surrogate_features(s, 0, N_TRAIN, X)
    epochs, nb = 60, N_TRAIN // 512
    hist = torch.empty(epochs * nb, device="cuda")
    msk.msk_surrogate_train(s, X, C, N_TRAIN, epochs, 2e-3, hist)
    torch.cuda.synchronize()
    yield solver, s, U, hist.cpu().numpy().reshape(epochs, nb)
    msk.msk_surrogate_destroy(s)
    solver.close()


def test_reference_solutions_are_the_magnus_solver(trained):
    solver, s, U, _ = trained
    ref = solver.magnus(2, 4, paths=8, precision=msk.MSK_F32)
    assert torch.equal(U[:8].view(8, SMALL.d, SMALL.d), ref)


def test_training_reduces_the_loss(trained):
    _, _, _, hist = trained
    assert np.all(np.isfinite(hist))
    assert hist[-1].mean() <= 0.05 * hist[0].mean()


def test_infer_audit_and_fallback(trained):
    solver, s, _, _ = trained
    n, P, p0, every = SMALL.d ** 2, 2500, N_TRAIN, 7      # chunks of 1000: 1000, 1000, 500
    ref = torch.empty(P, n, device="cuda")
    msk.msk_surrogate_reference(s, p0, P, ref)
    # plain surrogate: features -> network -> decode
    X = torch.empty(P, 48, dtype=torch.bfloat16, device="cuda")
    msk.msk_surrogate_features(s, p0, P, X)
    C = torch.empty(P, 16, device="cuda")
    msk.msk_surrogate_forward(s, X, P, C)
    plain = torch.empty(P, n, device="cuda")
    msk.msk_surrogate_decode(s, C, P, plain)
    idx = np.concatenate([o + np.arange(0, min(1000, P - o), every) for o in range(0, P, 1000)])
    errs = (torch.linalg.norm(plain - ref, dim=1) / torch.linalg.norm(ref, dim=1)).cpu().numpy()

    U = torch.empty(P, n, device="cuda")
    flags = torch.full((P,), 77, dtype=torch.int32, device="cuda")
    rep = msk.msk_surrogate_infer(s, p0, P, U, flags, 0)
    torch.cuda.synchronize()
    assert rep == [0.0] * 5 and int(flags.abs().sum()) == 0 and torch.equal(U, plain)

    rep = msk.msk_surrogate_infer(s, p0, P, U, flags, every, tol=10.0, max_fail_frac=1.0)
    f = flags.cpu().numpy()
    assert rep[0] == len(idx) and rep[3] == 0 and rep[4] == 0
    assert rep[1] == pytest.approx(errs[idx].max(), rel=1e-5)
    assert rep[2] == pytest.approx(errs[idx].mean(), rel=1e-5)
    assert np.array_equal(np.nonzero(f)[0], idx) and np.all(f[idx] == 1)
    assert torch.equal(U, plain)

    rep = msk.msk_surrogate_infer(s, p0, P, U, flags, every, tol=0.0, max_fail_frac=1.0)
    f = flags.cpu().numpy()
    assert rep[3] == len(idx) and rep[4] == 0 and np.all(f[idx] == 3)
    assert torch.equal(U[idx], ref[idx])
    keep = np.setdiff1d(np.arange(P), idx)
    assert torch.equal(U[keep], plain[keep])

    rep = msk.msk_surrogate_infer(s, p0, P, U, flags, every, tol=0.0, max_fail_frac=0.5)
    f = flags.cpu().numpy()
    assert rep[4] == 1 and np.all(f & 4) and torch.equal(U, ref)


def test_trained_surrogate_is_accurate_and_faster_than_magnus(trained):
    """What the network gains: held-out accuracy against the Magnus solution it
    learned, and serving time against solving the same paths with Magnus."""
    solver, s, _, _ = trained
    n, P, p0 = SMALL.d ** 2, 4000, N_TRAIN + 10_000
    U = torch.empty(P, n, device="cuda")
    ref = torch.empty(P, n, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    msk.msk_surrogate_infer(s, p0, P, U)                   # warm
    msk.msk_surrogate_reference(s, p0, P, ref)
    ev[0].record()
    msk.msk_surrogate_infer(s, p0, P, U)
    ev[1].record()
    msk.msk_surrogate_reference(s, p0, P, ref)
    ev[2].record()
    torch.cuda.synchronize()
    t_sur, t_mag = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    err = (torch.linalg.norm(U - ref, dim=1) / torch.linalg.norm(ref, dim=1)).cpu().numpy()
    print(f"surrogate {t_sur:.3f} ms, Magnus {t_mag:.3f} ms, held-out rel L2 mean {err.mean():.3e} "
          f"p99 {np.quantile(err, 0.99):.3e} max {err.max():.3e}")
    assert t_sur < t_mag
    assert err.mean() < 5e-2

"""GPU parity: every step of the CUDA path against the CPU oracle on the same
seeded Philox paths (FP64 <= 1e-10 and FP32 <= 1e-4 relative L2, integer work
bit-exact)."""
import os

import numpy as np
import scipy.sparse as sp
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from oracle import brownian, errors, euler as oeuler, explicit, magnus as omagnus, philox  # noqa: E402
from oracle import discretization as disc  # noqa: E402
from workloads import COEF_TRIG, LANGEVIN_32, LANGEVIN_TRIG_128  # noqa: E402

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2207_09776_b300 import build
    build.build()
    msk.load_library()


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


def solver(w):
    return msk.Solver(w, device=0)


# ---------------------------------------------------------------- integer work (bit-exact)

@pytest.mark.parametrize("seed,path", [(0, 0), (20220719, 7), (2 ** 63 + 12345, (1 << 32) + 5)])
def test_philox_words_bit_exact(seed, path):
    n = 1000
    out = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    msk.msk_philox_words(seed, path, 0, 17, n, out)
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    ref = philox.brownian_words(seed, path, np.arange(17, 17 + n))
    for r in range(4):
        np.testing.assert_array_equal(got[:, r], np.asarray(ref[r], dtype=np.uint32))


# ---------------------------------------------------------------- Brownian functionals

@pytest.mark.parametrize("w,K", [(LANGEVIN_32.with_(paths=6), 1), (LANGEVIN_32.with_(paths=5), 8),
                                 (LANGEVIN_TRIG_128.with_(paths=4, n_fine=2048), 16),
                                 (LANGEVIN_32.with_(paths=3, path_offset=(1 << 32) - 1, n_fine=999), 3)])
def test_brownian_functionals(w, K):
    s = solver(w)
    F = s.functionals(K).cpu().numpy()
    keys = ("dW", "I1", "I2", "I3", "om", "Jom", "G1", "G2")
    for p in range(w.paths):
        ref = brownian.step_functionals(w, p, K)
        for q, k in enumerate(keys):
            np.testing.assert_allclose(F[p, :, q], ref[k], rtol=1e-11, atol=1e-13, err_msg=k)
    dW = s.increments(K).cpu().numpy()
    for p in range(w.paths):
        np.testing.assert_allclose(dW[p], brownian.coarse_increments(w, p, K), rtol=1e-11, atol=1e-13)
    s.close()


@pytest.mark.parametrize("w,K", [(LANGEVIN_TRIG_128.with_(paths=4, n_fine=2048), 16),
                                 (LANGEVIN_32.with_(paths=3, n_fine=999), 3)])
def test_brownian_functionals_float_normals(w, K):
    """The float solves' functionals: float Box-Muller, double accumulation -- within
    ~1e-6 of the double-normal functionals; the double variant is the plain call."""
    s = solver(w)
    F = torch.empty(w.paths * K * msk.MSK_NF, dtype=torch.float64, device="cuda")
    msk.msk_brownian_functionals(s.ctx, K, w.paths, F)
    F64 = s.functionals(K, normals=msk.MSK_F64)
    F32 = s.functionals(K, normals=msk.MSK_F32).cpu().numpy()
    assert torch.equal(F.view_as(F64), F64)
    F64 = F64.cpu().numpy()
    scale = np.abs(F64).max(axis=(0, 1))
    np.testing.assert_allclose(F32, F64, rtol=0, atol=1e-6 * scale.max())
    assert not np.array_equal(F32, F64)
    # a float solve is functionals (float normals) -> weights -> engine, bit for bit
    u = s.magnus(3, K, precision=msk.MSK_F32)
    Wt = s.weights(3, K, precision=msk.MSK_F32)
    u2 = s.state(w.paths, msk.MSK_F32)
    msk.msk_magnus_from_weights(s.ctx, K, w.paths, msk.MSK_F32, Wt, u2)
    torch.cuda.synchronize()
    assert torch.equal(u, u2)
    s.close()


# ---------------------------------------------------------------- widened-stencil operator

@pytest.mark.parametrize("w,order,K", [(LANGEVIN_32.with_(paths=3), 3, 1),
                                       (LANGEVIN_32.with_(paths=3, drift_sign=-1, d=64), 2, 4),
                                       (LANGEVIN_TRIG_128.with_(paths=2, d=32, n_fine=256), 3, 4)])
def test_omega_matvec_matches_the_oracle_matrix(w, order, K):
    s = solver(w)
    Wt = s.weights(order, K)
    rng = np.random.default_rng(5)
    u = rng.normal(size=(w.paths, w.d, w.d))
    ut = torch.tensor(u, device="cuda")
    for n in range(K):
        wts = Wt[:, n, :msk.MSK_NOPS].contiguous()
        out = torch.empty_like(ut)
        msk.msk_apply_omega(s.ctx, wts, w.paths, ut, out)
        got = out.cpu().numpy()
        for p in range(w.paths):
            Y = omagnus.omega_matrix(w, order, K, p, n)
            ref = (Y @ u[p].ravel()).reshape(w.d, w.d)
            scale = np.abs(ref).max()
            np.testing.assert_allclose(got[p], ref, rtol=0, atol=1e-12 * scale)
    s.close()


def _theta_rows():
    import re
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2207_09776_b300", "csrc",
                            "theta_tables.h")).read()
    rows = {}
    for prec, name in ((msk.MSK_F64, "msk_theta_f64"), (msk.MSK_F32, "msk_theta_f32")):
        body = re.search(name + r"\[[^\]]*\] = \{([^}]*)\}", src).group(1)
        rows[prec] = np.array([float(x) for x in body.split(",") if x.strip()])
    return rows


def _power_norms_exact(A, J=9):
    """||A^q||_inf, q = 1..J, by sparse matrix powers."""
    out, P = [], A.copy()
    for q in range(1, J + 1):
        if q > 1:
            P = (P @ A).tocsr()
        out.append(abs(P).sum(axis=1).max())
    return np.array(out)


@pytest.mark.parametrize("kind", ["trig", "const"])
def test_power_norms_of_the_deterministic_part_match_sparse_powers(kind):
    """msk_power_norms vs ||X^q||_inf of the oracle's Omega with every functional zero."""
    from oracle.coefficients import Coefficients
    from oracle.discretization import LangevinOperators
    base = LANGEVIN_TRIG_128 if kind == "trig" else LANGEVIN_32.with_(d=64, ax=-6.0, bx=6.0, av=-6.0, bv=6.0)
    w = base.with_(d=64, paths=2, n_fine=1024)
    K = 8 if kind == "trig" else 4      # steps long enough for the table (see power_norm_rows)
    s = solver(w)
    for order in (1, 3):
        got = msk.msk_power_norms(s.ctx, order, K).cpu().numpy().astype(np.float64)
        assert got.shape == ((K if kind == "trig" else 1), 9)
        # short steps need no table: one sub-step is admissible by the plain norm already
        assert msk.msk_power_norms(s.ctx, order, 256).shape == (0, 9)
        ops, coef, h = LangevinOperators(w), Coefficients.of(w), w.T / K
        f0 = {k: 0.0 for k in ("dW", "I1", "I2", "I3", "om", "Jom", "G1", "G2")}
        for n in range(got.shape[0]):
            if kind == "trig":
                X = omagnus.omega_timedep(ops, coef, n * h, h, f0, order)
            else:
                X = omagnus.omega_const(ops.B(w.a0), ops.A(w.s0), h, 0.0, 0.0, 0.0, 0.0, order)
            X = (X - (X.diagonal().sum() / X.shape[0]) * sp.identity(X.shape[0])).tocsr()
            np.testing.assert_allclose(got[n], _power_norms_exact(X), rtol=2e-5)
    s.close()


def test_taylor_parameters_are_admissible():
    """(s, m) of every record: the stored norm bounds the exact ||Omega - mu I||_inf of the
    oracle's matrix (within 0.1 %), the bound alpha that chose them is at least the exact
    min_p alpha_p (Al-Mohy & Higham's Theorem 4.2, p(p-1) <= m + 1) and at most the
    norm, alpha / s <= theta_m, s is the smallest admissible scaling count
    (alpha > (s - 1) theta_120) and m <= 120."""
    w = LANGEVIN_TRIG_128.with_(d=64, paths=4, n_fine=1024)
    K = 8
    s = solver(w)
    theta = _theta_rows()
    for prec in (msk.MSK_F64, msk.MSK_F32):
        Wt = s.weights(3, K, precision=prec).cpu().numpy()
        th = theta[prec]
        # the float solves draw float normals: their Omega differs from the oracle's by ~1e-7
        rt = 1e-12 if prec == msk.MSK_F64 else 1e-6
        gain = []
        for p in range(w.paths):
            for n in range(K):
                rec = Wt[p, n]
                sv, mv, nrm, al = rec[msk.MSK_WT_S], rec[msk.MSK_WT_M], rec[msk.MSK_WT_NORM], rec[msk.MSK_WT_ALPHA]
                Y = omagnus.omega_matrix(w, 3, K, p, n)
                A = (Y - (Y.diagonal().sum() / Y.shape[0]) * sp.identity(Y.shape[0])).tocsr()
                dq = _power_norms_exact(A) ** (1.0 / np.arange(1, 10))
                # an upper bound: the edge columns are bounded by their larger centre coefficient
                assert dq[0] * (1 - rt) <= nrm <= dq[0] * (1 + 1e-3)
                alpha_p = [max(dq[q - 1], dq[q]) for q in range(2, 9) if q * (q - 1) <= mv + 1]
                assert min([dq[0]] + alpha_p) <= al * (1 + rt) and al <= nrm * (1 + 1e-12)
                assert 1 <= mv <= 120 and sv >= 1 and sv == int(sv) and mv == int(mv)
                assert al / sv <= th[int(mv) - 1] * (1 + 1e-12)
                eps, theta_e = rec[msk.MSK_WT_EPS], (14.0 if prec == msk.MSK_F32 else 24.0)
                assert eps / sv <= theta_e * (1 + 1e-12)            # the Brownian part per sub-step
                assert sv == 1 or al > (sv - 1) * th[119] or eps > (sv - 1) * theta_e
                assert rec[msk.MSK_WT_WORK] > 0
                gain.append(al / nrm)
        assert np.mean(gain) < 0.97          # the power bounds are sharper than the norm
    s.close()


# ---------------------------------------------------------------- full solves

def _oracle_magnus(w, order, K, paths):
    return omagnus.solve(w, order, K, paths)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_magnus_fp64_small_config_all_paths(order):
    """d = 32, 100 paths, one step to T = 1 (orders 1, 2, 3)."""
    w = LANGEVIN_32
    s = solver(w)
    u, st = s.magnus(order, 1, precision=msk.MSK_F64, status=True)
    got = u.cpu().numpy()
    ref = _oracle_magnus(w, order, 1, list(range(w.paths)))
    err = rel_l2(got, ref)
    assert err.max() <= TOL64, err.max()
    s.close()


@pytest.mark.parametrize("w,order,K,paths", [
    (LANGEVIN_32.with_(paths=7), 2, 10, 7),
    (LANGEVIN_32.with_(paths=5, drift_sign=-1, a0=1.1, s0=10 ** -0.5), 3, 4, 5),
    (LANGEVIN_TRIG_128.with_(d=64, paths=3, n_fine=1024), 3, 8, 3),
    (LANGEVIN_TRIG_128.with_(paths=2, n_fine=1024), 2, 8, 2),
])
def test_magnus_fp64_parity(w, order, K, paths):
    s = solver(w)
    got = s.magnus(order, K, paths=paths, precision=msk.MSK_F64).cpu().numpy()
    ref = _oracle_magnus(w, order, K, list(range(paths)))
    err = rel_l2(got, ref)
    assert err.max() <= TOL64, err
    s.close()


@pytest.mark.parametrize("w,order,K,paths", [
    (LANGEVIN_32.with_(paths=20), 2, 1, 20),
    (LANGEVIN_TRIG_128.with_(d=64, paths=3, n_fine=1024), 3, 8, 3),
    (LANGEVIN_TRIG_128.with_(paths=2, n_fine=1024), 3, 8, 2),
])
def test_magnus_fp32_parity(w, order, K, paths):
    s = solver(w)
    u, st = s.magnus(order, K, paths=paths, precision=msk.MSK_F32, status=True)
    ref = _oracle_magnus(w, order, K, list(range(paths)))
    err = rel_l2(u.cpu().numpy(), ref)
    assert err.max() <= TOL32, err
    assert int(st.cpu().numpy()[:paths].max()) == 0
    s.close()


def test_fp64_and_fp32_agree_on_many_paths():
    """Ragged path count (not a multiple of the resident-CTA count), the FP32
    path against the (oracle-checked) FP64 path."""
    w = LANGEVIN_TRIG_128.with_(d=64, paths=301, n_fine=1024)
    s = solver(w)
    u64 = s.magnus(2, 8, precision=msk.MSK_F64)
    u32 = s.magnus(2, 8, precision=msk.MSK_F32)
    err = rel_l2(u32.cpu().numpy(), u64.cpu().numpy())
    assert err.max() <= TOL32
    # sampled paths against the oracle
    for p in (0, 150, 300):
        ref = omagnus.solve_path(w, 2, 8, p)
        assert rel_l2(u64[p:p + 1].cpu().numpy(), ref[None])[0] <= TOL64
    s.close()


@pytest.mark.parametrize("precision,tol", [(msk.MSK_F32, TOL32), (msk.MSK_F64, TOL64)])
def test_solve_with_host_buffers(precision, tol):
    """msk_solve_magnus_host: the kernels store every path straight into page-locked
    host memory; the results equal the device-buffer solve bit for bit (same kernels,
    ragged path count), an initial datum passed from the host replaces the context's,
    and pageable output memory is refused before any work is enqueued."""
    w = LANGEVIN_TRIG_128.with_(d=64, paths=301, n_fine=1024)
    s = solver(w)
    u_dev, st_dev = s.magnus(3, 8, precision=precision, status=True)
    u_host, st_host = s.magnus_host(3, 8, precision=precision, status=True)
    assert not u_host.is_cuda and u_host.is_pinned()
    np.testing.assert_array_equal(u_host.numpy(), u_dev.cpu().numpy())
    np.testing.assert_array_equal(st_host.numpy()[:w.paths], st_dev.cpu().numpy()[:w.paths])
    ref = omagnus.solve_path(w, 3, 8, 200)
    assert rel_l2(u_host[200:201].numpy(), ref[None])[0] <= tol
    # a host initial datum (a skewed Gaussian) replaces the context's
    g = disc.gaussian_initial(w.with_(u0_mean=(-1.0, 0.5), u0_cov=(0.8, 0.2, 0.6)))
    u0 = torch.from_numpy(np.ascontiguousarray(disc.vec(g)))
    got = s.magnus_host(3, 8, paths=3, precision=precision, u0=u0).numpy()
    ref = np.stack([omagnus.solve_path(w, 3, 8, p, u0=u0.numpy()) for p in range(3)])
    assert rel_l2(got, ref).max() <= tol
    # pageable host memory cannot be written by the kernels: refused
    bad = torch.empty(3 * w.d * w.d, dtype=torch.float32 if precision == msk.MSK_F32 else torch.float64)
    with pytest.raises(msk.MskError) as e:
        msk.msk_solve_magnus_host(s.ctx, 3, 8, 3, precision, None, bad)
    assert e.value.status == msk.MSK_ERR_ARG
    with pytest.raises(ValueError):
        msk.msk_solve_magnus_host(s.ctx, 3, 8, 3, precision, None, u_dev)   # a device tensor
    s.close()


@pytest.mark.parametrize("d,precision,paths", [(64, msk.MSK_F32, 700), (64, msk.MSK_F64, 700),
                                               (256, msk.MSK_F32, 320), (128, msk.MSK_F64, 320)])
def test_dynamic_path_queue_matches_static_assignment(d, precision, paths):
    """Above two paths per SM the engine hands out paths from an atomic queue in
    order of decreasing estimated cost (on clusters -- 256^2 float: 4 CTAs, 128^2
    double: 2 CTAs -- rank 0 takes the position and the others read it through
    distributed shared memory); every path's solution must be identical (bit for
    bit) to the static assignment used for small path counts."""
    w = LANGEVIN_TRIG_128.with_(d=d, paths=paths, n_fine=1024)
    s = solver(w)
    # the resident engine alone (at 256^2 in float the automatic choice splits a queued
    # solve with the streamed engine, which takes the last paths; tests/test_gpu_stream.py)
    msk.msk_set_engine(s.ctx, msk.MSK_ENGINE_RESIDENT)
    full = s.magnus(3, 8, precision=precision).cpu().numpy()        # queued
    parts = []
    cuts = [0, paths // 3, 2 * paths // 3, paths]
    for lo, hi in zip(cuts[:-1], cuts[1:]):                          # <= 2 per SM: static
        msk.msk_set_seed(s.ctx, w.seed, lo, w.n_fine, w.T)
        parts.append(s.magnus(3, 8, paths=hi - lo, precision=precision).cpu().numpy())
    np.testing.assert_array_equal(full, np.concatenate(parts))
    s.close()


@pytest.mark.parametrize("precision,tol", [(msk.MSK_F32, TOL32), (msk.MSK_F64, TOL64)])
def test_full_bench_configuration_on_sampled_paths(precision, tol):
    """The benchmark's own configuration at full size -- 4096 paths, d = 128, 2^14 fine
    cells, order 3, K = 8, time-dependent coefficients -- run exactly as the bench times
    it (functionals, weights, then the solve from the weights with the cost-ordered
    queue), checked against the oracle on sampled paths (first, last, middle and a few
    scattered ones) and for finiteness and clean status everywhere."""
    w = LANGEVIN_TRIG_128
    assert w.paths == 4096 and w.d == 128 and w.n_fine == 16384
    s = solver(w)
    K, P = 8, w.paths
    F = torch.empty(P * K * msk.MSK_NF, dtype=torch.float64, device="cuda")
    Wt = torch.empty(P * K * msk.MSK_NWT, dtype=torch.float64, device="cuda")
    out = s.state(P, precision)
    st = torch.full((P,), 7, dtype=torch.int32, device="cuda")
    msk.msk_brownian_functionals_ex(s.ctx, K, P, precision, F)
    msk.msk_omega_weights(s.ctx, 3, K, P, precision, F, Wt)
    msk.msk_magnus_from_weights(s.ctx, K, P, precision, Wt, out, st)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
    assert int(st.max()) == 0
    sample = [0, 1, 777, 2048, 3001, 4095]
    ref = np.stack([omagnus.solve_path(w, 3, K, p) for p in sample])
    err = rel_l2(out[sample].cpu().numpy(), ref)
    assert err.max() <= tol, err
    s.close()


def test_euler_parity():
    w = LANGEVIN_32.with_(paths=6)
    s = solver(w)
    got = s.euler(1000, precision=msk.MSK_F64).cpu().numpy()
    ref = oeuler.solve(w, 1000, list(range(w.paths)))
    assert rel_l2(got, ref).max() <= TOL64
    got32 = s.euler(1000, precision=msk.MSK_F32).cpu().numpy()
    assert rel_l2(got32, ref).max() <= TOL32
    s.close()


def test_euler_timedep_parity():
    w = LANGEVIN_TRIG_128.with_(d=32, paths=3, n_fine=2048, ax=-5.0, bx=5.0, av=-5.0, bv=5.0)
    s = solver(w)
    got = s.euler(2048, precision=msk.MSK_F64).cpu().numpy()
    ref = oeuler.solve(w, 2048, list(range(w.paths)))
    assert rel_l2(got, ref).max() <= TOL64
    s.close()


# ---------------------------------------------------------------- closed form, norms, moments

@pytest.mark.parametrize("w", [LANGEVIN_32.with_(paths=5),
                               LANGEVIN_TRIG_128.with_(paths=3, d=64, n_fine=2048),
                               LANGEVIN_32.with_(paths=2, drift_sign=-1, u0_mean=(0.3, -0.4),
                                                 u0_cov=(0.7, 0.2, 1.2), u0_scale=2 * np.pi)])
def test_explicit_solution_and_error_norms(w):
    s = solver(w)
    ex = s.explicit()
    ref = explicit.solutions(w)
    np.testing.assert_allclose(ex.cpu().numpy(), ref, rtol=1e-9, atol=1e-13 * np.abs(ref).max())
    u = s.magnus(2, 1 if w.n_fine % 2 else 2, precision=msk.MSK_F64)
    for kappa in (0, 1):
        e, m = s.error(u, msk.MSK_F64, kappa=kappa)
        oe = errors.rel_err_per_path(u.cpu().numpy(), ref, kappa)
        np.testing.assert_allclose(e.cpu().numpy(), oe, rtol=1e-8)
        assert float(m.cpu()[0]) == pytest.approx(errors.Err(u.cpu().numpy(), ref, kappa), rel=1e-8)
        e2, _ = s.error(u, msk.MSK_F64, ref=ex, kappa=kappa)
        np.testing.assert_allclose(e2.cpu().numpy(), oe, rtol=1e-8)
    mom = s.moments(u, msk.MSK_F64).cpu().numpy()
    xs, dx = disc.grid(w.d, w.ax, w.bx)
    vs, dv = disc.grid(w.d, w.av, w.bv)
    np.testing.assert_allclose(mom, errors.moments(u.cpu().numpy(), xs, vs, dx, dv), rtol=1e-10, atol=1e-12)
    s.close()


# ---------------------------------------------------------------- edge cases

def test_empty_and_invalid_calls():
    w = LANGEVIN_32.with_(paths=2)
    s = solver(w)
    out = s.state(1)
    msk.msk_solve_magnus(s.ctx, 2, 1, 0, msk.MSK_F64, out)          # zero paths: no-op
    msk.msk_solve_euler(s.ctx, 10, 0, msk.MSK_F64, out)
    with pytest.raises(msk.MskError) as e:
        msk.msk_solve_magnus(s.ctx, 4, 1, 1, msk.MSK_F64, out)       # order out of range
    assert e.value.status == msk.MSK_ERR_ARG
    with pytest.raises(msk.MskError):
        msk.msk_solve_magnus(s.ctx, 2, 3, 1, msk.MSK_F64, out)       # 3 does not divide 10000
    with pytest.raises(msk.MskError):
        msk.msk_set_seed(s.ctx, 1, 0, 0, 1.0)
    with pytest.raises(msk.MskError) as e:
        msk.msk_set_coefficients(s.ctx, 1, 0, float("inf"), 0, 0.5, 0)
    assert e.value.status == msk.MSK_ERR_NONFINITE
    # the binding refuses an output buffer smaller than paths x d x d before any launch
    with pytest.raises(ValueError):
        msk.msk_solve_magnus(s.ctx, 2, 1, 2, msk.MSK_F64, out)
    # a single path and the context still works after rejected calls
    u = s.magnus(2, 1, paths=1)
    ref = omagnus.solve(w, 2, 1, [0])
    assert rel_l2(u.cpu().numpy(), ref).max() <= TOL64
    s.close()


def test_deterministic_case_and_blowup_flag():
    # sigma = 0: order 1 with any step count is exp(T B) u0 (Remark determLangevin)
    w = LANGEVIN_32.with_(paths=2, s0=0.0)
    s = solver(w)
    u1 = s.magnus(1, 1).cpu().numpy()
    u8 = s.magnus(1, 8).cpu().numpy()
    assert rel_l2(u8, u1).max() <= 1e-11
    s.close()
    # sigma^2 > a: the Ito correction -A^2/2 outweighs the diffusion and the
    # order-2 solution grows without bound (flagged, not an error)
    w = LANGEVIN_32.with_(paths=8, s0=3.0)
    s = solver(w)
    _, st = s.magnus(2, 1, precision=msk.MSK_F64, status=True)
    assert (st.cpu().numpy() & msk.MSK_PATH_BLOWUP).any()
    s.close()


def test_paths_are_keyed_by_global_index():
    w = LANGEVIN_32.with_(paths=6)
    s = solver(w)
    full = s.magnus(2, 2).cpu().numpy()
    msk.msk_set_seed(s.ctx, w.seed, 3, w.n_fine, w.T)
    tail = s.magnus(2, 2, paths=3).cpu().numpy()
    np.testing.assert_array_equal(tail, full[3:])
    s.close()


# ---------------------------------------------------------------- cluster configurations

from workloads import BATCH_GRIDS, LARGE_512  # noqa: E402


@pytest.mark.parametrize("precision,tol", [(msk.MSK_F32, TOL32), (msk.MSK_F64, TOL64)])
def test_d256_cluster_slabs_match_the_oracle(precision, tol):
    """256 x 256: four (float) or eight (double) CTAs per path exchange halo rows
    through distributed shared memory."""
    w = BATCH_GRIDS[2].with_(paths=2, T=0.25, n_fine=256)
    s = solver(w)
    u, st = s.magnus(3, 2, precision=precision, status=True)
    ref = _oracle_magnus(w, 3, 2, [0, 1])
    assert rel_l2(u.cpu().numpy(), ref).max() <= tol
    assert int(st.cpu().numpy().max()) == 0
    s.close()


def test_d512_sixteen_cta_clusters_match_the_oracle():
    w = LARGE_512[1].with_(paths=1, T=0.05, n_fine=64)
    s = solver(w)
    msk.msk_set_engine(s.ctx, msk.MSK_ENGINE_RESIDENT)   # (what the automatic choice runs for one path)
    u = s.magnus(2, 1, precision=msk.MSK_F32)
    ref = _oracle_magnus(w, 2, 1, [0])
    assert rel_l2(u.cpu().numpy(), ref).max() <= TOL32
    # double at 512^2 does not fit a cluster's shared memory: the resident engine
    # refuses it (the automatic choice runs the streamed engine, tests/test_gpu_stream.py)
    with pytest.raises(msk.MskError) as e:
        s.magnus(2, 1, precision=msk.MSK_F64)
    assert e.value.status == msk.MSK_ERR_UNSUPPORTED
    s.close()


def test_d512_full_size_on_a_sampled_path():
    """The 512^2 configuration at full size as the bench runs it for sigma = 0.5 (1024 paths,
    order 2, K = 64 from the fixed-error protocol, 2^14 fine cells, 16-CTA clusters with
    the cost-ordered queue): every path finite and unflagged, the last path against the
    oracle (one oracle path takes most of a minute)."""
    w = LARGE_512[1]
    assert w.paths == 1024 and w.d == 512 and w.s0 == 0.5
    s = solver(w)
    msk.msk_set_engine(s.ctx, msk.MSK_ENGINE_RESIDENT)
    u, st = s.magnus(2, 64, precision=msk.MSK_F32, status=True)
    assert bool(torch.isfinite(u).all())
    assert int(st[: w.paths].max()) == 0
    ref = _oracle_magnus(w, 2, 64, [w.paths - 1])
    assert rel_l2(u[w.paths - 1:].cpu().numpy(), ref).max() <= TOL32
    s.close()


def test_d256_euler_clusters():
    w = BATCH_GRIDS[2].with_(paths=2, T=0.05, n_fine=64)
    s = solver(w)
    ref = oeuler.solve(w, 64, [0, 1])
    assert rel_l2(s.euler(64, precision=msk.MSK_F64).cpu().numpy(), ref).max() <= TOL64
    assert rel_l2(s.euler(64, precision=msk.MSK_F32).cpu().numpy(), ref).max() <= TOL32
    s.close()

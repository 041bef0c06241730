"""GPU parity of the variable-coefficient path (Section 3.2, Eq. coeffsLangevinVar):
the x-profile engine against the CPU oracle (FP64 <= 1e-10, FP32 <= 1e-4 relative
L2), against the constant-coefficient engine when psi = 1, and its operator norms
against the oracle's exact ones."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from oracle import discretization as disc, euler as oeuler, magnus as omagnus  # noqa: E402
from oracle.magnus import comm  # noqa: E402
from workloads import COEF_TRIG, PAPER_VAR, XPROF_NONE  # noqa: E402

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


def var_case(d, **kw):
    """The paper's variable-coefficient problem on a d x d grid."""
    base = dict(d=d, paths=3, n_fine=240)
    base.update(kw)
    return PAPER_VAR[0].with_(**base)


def record(w, w6, paths):
    """Weight records with s = m = 1, mu = 0 (one Taylor term: u + Omega u) for the
    six-operator logarithm, the other basis weights implied by B = Bx + a/2 Bvv."""
    al = 0.5 * w.a0
    rec = np.zeros((paths, 1, msk.MSK_NWT))
    for p in range(paths):
        wB, wA, wAA, wBA, wBAA, wBAB = w6[p]
        r = rec[p, 0]
        r[0], r[1], r[2], r[3] = wB, al * wB, wA, wAA             # Bx, Bvv, A0, A0^2
        r[4], r[5] = wBA, al * wBA                                 # [Bx,A0], [Bvv,A0]
        r[7], r[8] = wBAA, al * wBAA                               # [[Bx,A0],A0], [[Bvv,A0],A0]
        r[9], r[10], r[11], r[12] = wBAB, al * wBAB, al * wBAB, al * al * wBAB
        r[msk.MSK_WT_S], r[msk.MSK_WT_M] = 1.0, 1.0
    return rec


def oracle_omega(w, w6):
    ops = disc.LangevinOperators(w)
    B, A0 = ops.B(w.a0), ops.A0
    BA = comm(B, A0)
    wB, wA, wAA, wBA, wBAA, wBAB = w6
    return (wB * B + wA * A0 + wAA * (A0 @ A0) + wBA * BA + wBAA * comm(BA, A0) + wBAB * comm(BA, B)).tocsr()


def rounding_bound(w, w6, u, eps):
    """Elementwise rounding bound of evaluating u + Omega u as the sum of the operator
    words: eps x (|u| + sum over words |c| |M1| |M2| |M3| |u|), |M| entrywise, with a
    factor 16 for the few roundings per product and sum."""
    ops = disc.LangevinOperators(w)
    aB, aA = abs(ops.B(w.a0)), abs(ops.A0)
    au = np.abs(u)
    wB, wA, wAA, wBA, wBAA, wBAB = np.abs(w6)
    Au, Bu = aA @ au, aB @ au
    AAu, BAu, ABu, BBu = aA @ Au, aB @ Au, aA @ Bu, aB @ Bu
    s = (wB * Bu + wA * Au + wAA * AAu + wBA * (BAu + ABu)
         + wBAA * (aB @ AAu + 2 * (aA @ BAu) + aA @ ABu)
         + wBAB * (2 * (aB @ ABu) + aA @ BBu + aB @ BAu))
    return eps * (au + 16.0 * s)


@pytest.mark.parametrize("d,prec", [(24, msk.MSK_F64), (41, msk.MSK_F64), (100, msk.MSK_F64),
                                    (100, msk.MSK_F32), (200, msk.MSK_F32), (300, msk.MSK_F32),
                                    (151, msk.MSK_F64), (201, msk.MSK_F32)])
def test_one_omega_application_matches_the_oracle(d, prec):
    """u + Omega u with the six operators composed on the GPU (one CTA per path up to
    clusters of 9 for d = 24 .. 300; even d two columns per thread, odd d on clusters
    one column per thread with one cluster barrier per term) against the oracle's
    sparse commutators, within the rounding bound of the working precision."""
    w = var_case(d, paths=2, drift_sign=-1)
    rng = np.random.default_rng(d)
    w6 = rng.normal(size=(2, 6)) * np.array([2e-3, 0.05, 1e-3, 1e-3, 1e-4, 1e-5])
    s = msk.Solver(w)
    Wt = torch.tensor(record(w, w6, 2), device="cuda")
    out = s.state(2, prec)
    msk.msk_magnus_from_weights(s.ctx, 1, 2, prec, Wt, out)
    got = out.double().cpu().numpy().reshape(2, -1)
    u0 = disc.vec(disc.gaussian_initial(w))
    for p in range(2):
        ref = u0 + oracle_omega(w, w6[p]) @ u0
        if prec == msk.MSK_F64:
            assert np.abs(got[p] - ref).max() <= 1e-12 * np.abs(ref).max()
        else:   # the oracle's own double rounding is negligible against the float bound
            assert np.all(np.abs(got[p] - ref) <= rounding_bound(w, w6[p], u0, 2.0 ** -24))
            assert np.linalg.norm(got[p] - ref) <= TOL32 * np.linalg.norm(ref)
    s.close()


def test_operator_traces_and_norm_bounds():
    """mu = trace(Omega)/n exactly, and the norm bound dominates the exact infinity norm
    of Omega - mu I (and is not loose by more than the triangle inequality allows)."""
    w = var_case(20, paths=4, n_fine=64, s0=0.8)
    s = msk.Solver(w)
    Wt = s.weights(3, 4, precision=msk.MSK_F64).cpu().numpy()
    F = s.functionals(4).cpu().numpy()
    h = w.T / 4
    n = w.d * w.d
    for p in range(w.paths):
        for k in range(4):
            dW, I1, I2, I3 = (F[p, k, msk.MSK_F_DW], F[p, k, msk.MSK_F_I1], F[p, k, msk.MSK_F_I2],
                              F[p, k, msk.MSK_F_I3])
            Y = omagnus.omega_const(disc.LangevinOperators(w).B(w.a0), disc.LangevinOperators(w).A(w.s0),
                                    h, dW, I1, I2, I3, 3).toarray()
            mu = np.trace(Y) / n
            assert abs(Wt[p, k, msk.MSK_WT_MU] - mu) <= 1e-12 * max(1.0, abs(mu))
            exact = np.abs(Y - mu * np.eye(n)).sum(axis=1).max()
            bound = Wt[p, k, msk.MSK_WT_NORM]
            assert exact <= bound * (1 + 1e-12)
            assert bound <= 3.0 * exact
    s.close()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_variable_coefficient_magnus_fp64_matches_the_oracle(order):
    w = var_case(24, paths=3, n_fine=240)
    s = msk.Solver(w)
    got = s.magnus(order, 4, precision=msk.MSK_F64).cpu().numpy()
    ref = omagnus.solve(w, order, 4, list(range(w.paths)))
    assert rel_l2(got, ref).max() <= TOL64
    got32 = s.magnus(order, 4, precision=msk.MSK_F32).cpu().numpy()
    assert rel_l2(got32, ref).max() <= TOL32
    s.close()


def test_variable_coefficient_magnus_on_a_cluster_matches_the_oracle():
    """d = 90 in double needs a cluster of CTAs: halo exchange across the slabs."""
    w = var_case(90, paths=2, n_fine=120)
    s = msk.Solver(w)
    got = s.magnus(3, 3, precision=msk.MSK_F64).cpu().numpy()
    ref = omagnus.solve(w, 3, 3, [0, 1])
    assert rel_l2(got, ref).max() <= TOL64
    s.close()


def test_variable_coefficient_euler_matches_the_oracle():
    w = var_case(24, paths=3, n_fine=400)
    s = msk.Solver(w)
    ref = oeuler.solve(w, 400, [0, 1, 2])
    got = s.euler(400, precision=msk.MSK_F64).cpu().numpy()
    assert rel_l2(got, ref).max() <= TOL64
    got32 = s.euler(400, precision=msk.MSK_F32).cpu().numpy()
    assert rel_l2(got32, ref).max() <= TOL32
    # time-dependent coefficients are accepted by Euler
    wt = w.with_(kind=COEF_TRIG, a1=0.3, s1=0.2)
    st = msk.Solver(wt)
    assert rel_l2(st.euler(400, precision=msk.MSK_F64).cpu().numpy(), oeuler.solve(wt, 400, [0, 1, 2])).max() <= TOL64
    st.close()
    s.close()


@pytest.mark.parametrize("prec,tol", [(msk.MSK_F64, 1e-12), (msk.MSK_F32, TOL32)])
def test_unit_profile_reproduces_the_constant_coefficient_engine(prec, tol):
    """psi = 1 given as values: the composed operators equal the widened stencils."""
    w = PAPER_VAR[0].with_(d=64, paths=4, n_fine=1200, x_profile=XPROF_NONE)
    s = msk.Solver(w)
    ref = s.magnus(3, 12, precision=prec).double().cpu().numpy()
    ref_e = s.euler(1200, precision=prec).double().cpu().numpy()
    msk.msk_set_x_profile(s.ctx, msk.MSK_XPROF_VALUES, 0.0, [1.0] * w.d)
    got = s.magnus(3, 12, precision=prec).double().cpu().numpy()
    got_e = s.euler(1200, precision=prec).double().cpu().numpy()
    assert rel_l2(got, ref).max() <= tol
    assert rel_l2(got_e, ref_e).max() <= tol
    s.close()


@pytest.mark.parametrize("d,K", [(100, 20), (200, 40)])
def test_paper_grids_float_against_double(d, K):
    """Table errorsVar grids: the float engine against the double engine (same paths)."""
    w = PAPER_VAR[0].with_(d=d, paths=4)
    s = msk.Solver(w)
    u64, st64 = s.magnus(3, K, precision=msk.MSK_F64, status=True)
    u32, st32 = s.magnus(3, K, precision=msk.MSK_F32, status=True)
    assert int(st64.max()) == 0 and int(st32.max()) == 0
    assert rel_l2(u32.cpu().numpy(), u64.cpu().numpy()).max() <= TOL32
    s.close()


@pytest.mark.parametrize("d", [24, 200])
def test_dynamic_path_queue_matches_static_assignment(d):
    """More than two paths per SM: the float variable-coefficient engine takes paths
    from an atomic queue, costliest first (d = 200: rank 0 of each 3-CTA cluster
    takes them and the other CTAs read the path through distributed shared memory).
    Every path must equal, bit for bit, the static assignment of smaller batches."""
    w = PAPER_VAR[0].with_(d=d, paths=320, T=0.1, n_fine=64)
    s = msk.Solver(w)
    full = s.magnus(3, 4, precision=msk.MSK_F32).cpu().numpy()
    parts = []
    for lo, hi in ((0, 160), (160, 320)):
        msk.msk_set_seed(s.ctx, w.seed, lo, w.n_fine, w.T)
        parts.append(s.magnus(3, 4, paths=hi - lo, precision=msk.MSK_F32).cpu().numpy())
    np.testing.assert_array_equal(full, np.concatenate(parts))
    s.close()


@pytest.mark.parametrize("d,K,paths,sample", [(100, 20, 4096, [0, 2047, 4095]), (200, 40, 1024, [1023])])
def test_paper_grids_at_bench_size_on_sampled_paths(d, K, paths, sample):
    """Table errorsVar grids at the path counts the bench runs (order 3, the paper's steps,
    10^5 fine cells, float): every path finite and unflagged, sampled paths against the
    oracle."""
    w = PAPER_VAR[(100, 200, 300).index(d)].with_(paths=paths)
    s = msk.Solver(w)
    u, st = s.magnus(3, K, precision=msk.MSK_F32, status=True)
    assert bool(torch.isfinite(u).all())
    assert int(st[:paths].max()) == 0
    ref = omagnus.solve(w, 3, K, sample)
    assert rel_l2(u[sample].cpu().numpy(), ref).max() <= TOL32
    s.close()


def test_paper_grid_300_float_against_the_oracle():
    """d = 300 (a cluster of 7 CTAs per path in float) on a short horizon."""
    w = PAPER_VAR[2].with_(paths=1, T=0.02, n_fine=200)
    s = msk.Solver(w)
    got = s.magnus(3, 2, precision=msk.MSK_F32).cpu().numpy()
    ref = omagnus.solve(w, 3, 2, [0])
    assert rel_l2(got, ref).max() <= TOL32
    s.close()


def test_unsupported_combinations_are_reported():
    w = var_case(32, paths=1)
    s = msk.Solver(w)
    out = s.state(1, msk.MSK_F64)
    with pytest.raises(msk.MskError) as e:
        msk.msk_explicit_solution(s.ctx, 1, out)
    assert e.value.status == msk.MSK_ERR_UNSUPPORTED
    for kind, c, vals, status in ((7, 1.0, None, msk.MSK_ERR_ARG), (msk.MSK_XPROF_RATIONAL, -1.0, None, msk.MSK_ERR_ARG),
                                  (msk.MSK_XPROF_RATIONAL, float("nan"), None, msk.MSK_ERR_NONFINITE),
                                  (msk.MSK_XPROF_VALUES, 0.0, [1.0] * 31 + [0.0], msk.MSK_ERR_ARG)):
        with pytest.raises(msk.MskError) as e:
            msk.msk_set_x_profile(s.ctx, kind, c, vals)
        assert e.value.status == status
    s.close()


# ---------------------------------------------------------------- time-dependent coefficients
def trig_case(d, **kw):
    base = dict(kind=COEF_TRIG, a1=0.4, s1=0.3, n_fine=256)
    base.update(kw)
    return var_case(d, **base)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_time_dependent_coefficients_with_a_profile_match_the_oracle(order):
    """The thirteen-operator composition (X = Bx, V = Bvv, A = A0 with the profile)."""
    w = trig_case(24, paths=3)
    s = msk.Solver(w)
    ref = omagnus.solve(w, order, 4, list(range(w.paths)))
    assert rel_l2(s.magnus(order, 4, precision=msk.MSK_F64).cpu().numpy(), ref).max() <= TOL64
    assert rel_l2(s.magnus(order, 4, precision=msk.MSK_F32).cpu().numpy(), ref).max() <= TOL32
    s.close()


def test_time_dependent_coefficients_with_a_profile_on_a_cluster():
    w = trig_case(90, paths=2, n_fine=128)
    s = msk.Solver(w)
    got = s.magnus(3, 2, precision=msk.MSK_F64).cpu().numpy()
    assert rel_l2(got, omagnus.solve(w, 3, 2, [0, 1])).max() <= TOL64
    s.close()


@pytest.mark.parametrize("prec,tol", [(msk.MSK_F64, 1e-12), (msk.MSK_F32, TOL32)])
def test_unit_profile_with_time_dependent_coefficients_equals_the_main_engine(prec, tol):
    from workloads import LANGEVIN_TRIG_128
    w = LANGEVIN_TRIG_128.with_(d=64, paths=4, n_fine=1024)
    s = msk.Solver(w)
    ref = s.magnus(3, 8, precision=prec).double().cpu().numpy()
    msk.msk_set_x_profile(s.ctx, msk.MSK_XPROF_VALUES, 0.0, [1.0] * w.d)
    got = s.magnus(3, 8, precision=prec).double().cpu().numpy()
    assert rel_l2(got, ref).max() <= tol
    s.close()


def test_thirteen_operator_traces_and_norm_bounds():
    w = trig_case(16, paths=2, n_fine=64, s0=0.8)
    s = msk.Solver(w)
    Wt = s.weights(3, 4, precision=msk.MSK_F64).cpu().numpy()
    n = w.d * w.d
    for p in range(w.paths):
        for k in range(4):
            Y = omagnus.omega_matrix(w, 3, 4, p, k).toarray()
            mu = np.trace(Y) / n
            assert abs(Wt[p, k, msk.MSK_WT_MU] - mu) <= 1e-12 * max(1.0, abs(mu))
            exact = np.abs(Y - mu * np.eye(n)).sum(axis=1).max()
            assert exact <= Wt[p, k, msk.MSK_WT_NORM] * (1 + 1e-12) <= 3.0 * exact * (1 + 1e-12)
    s.close()

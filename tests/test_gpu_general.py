"""GPU parity of the general-coefficient path (Eq. generalSPDE): nine-point B and
five-point A with per-point coefficients, against the oracle's Kronecker assembly
(Section 2, "Computation of A and B") with its sparse commutators and expm action."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from oracle import brownian, discretization as disc, magnus as omagnus  # noqa: E402
from oracle.magnus import comm  # noqa: E402
from workloads import LANGEVIN_32, PAPER_VAR  # noqa: E402

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


# smooth coefficient functions with every term of Eq. generalSPDE present
COEFS = dict(
    h=lambda x, v: -0.1 * (1 + 0.2 * np.sin(x)),
    fx=lambda x, v: -v + 0.1 * np.cos(x),
    fv=lambda x, v: 0.2 * np.sin(x) - 0.1 * v,
    gxx=lambda x, v: 0.05 + 0.01 * np.cos(v),
    gxv=lambda x, v: 0.02 * np.exp(-0.1 * x * x),
    gvv=lambda x, v: 1.0 + 0.1 * np.cos(x * v / 4),
    s=lambda x, v: 0.1 + 0.0 * x,
    sx=lambda x, v: 0.05 * np.cos(v),
    sv=lambda x, v: 0.3 * (1 + 0.2 * np.sin(x)))
ORDER9 = ("h", "fx", "fv", "gxx", "gxv", "gvv", "s", "sx", "sv")


def grids(w, cf):
    """[9][v][x] coefficient values at the interior nodes."""
    xs, _ = disc.grid(w.d, w.ax, w.bx)
    vs, _ = disc.grid(w.d, w.av, w.bv)
    X, V = np.meshgrid(xs, vs, indexing="xy")   # [v][x]
    return np.stack([np.broadcast_to(cf[k](X, V), X.shape) for k in ORDER9])


def oracle_ops(w, cf):
    B, A = disc.assemble(w.d, w.ax, w.bx, w.d, w.av, w.bv, **cf)
    return B, A


def general_solver(w, cf=COEFS):
    s = msk.Solver(w)
    msk.msk_set_general_coefficients(s.ctx, grids(w, cf))
    return s


def case(d, **kw):
    base = dict(d=d, ax=-3.0, bx=3.0, av=-3.0, bv=3.0, n_fine=240, paths=3)
    base.update(kw)
    return LANGEVIN_32.with_(**base)


def oracle_magnus(w, B, A, order, K, p):
    U = disc.vec(disc.gaussian_initial(w))
    f = brownian.step_functionals(w, p, K)
    h = w.T / K
    for n in range(K):
        Y = omagnus.omega_const(B, A, h, f["dW"][n], f["I1"][n], f["I2"][n], f["I3"][n], order)
        U = omagnus.expm_action(Y, U)
    return U.reshape(w.d, w.d)


@pytest.mark.parametrize("d", [22, 21, 100])
def test_one_omega_application_matches_the_oracle(d):
    """u + Omega u on the GPU against the oracle's Kronecker assembly and sparse
    commutators: d = 22 two columns per thread on one CTA, d = 21 one column per thread,
    d = 100 two columns per thread on clusters (halos of the extended passes)."""
    w = case(d, paths=2)
    B, A = oracle_ops(w, COEFS)
    rng = np.random.default_rng(5)
    w6 = rng.normal(size=(2, 6)) * np.array([1e-2, 0.05, 1e-3, 1e-3, 1e-4, 1e-4])
    rec = np.zeros((2, 1, msk.MSK_NWT))
    for p in range(2):
        rec[p, 0, [0, 2, 3, 4, 7, 9]] = w6[p]
        rec[p, 0, msk.MSK_WT_S], rec[p, 0, msk.MSK_WT_M] = 1.0, 1.0
    s = general_solver(w)
    out = s.state(2, msk.MSK_F64)
    msk.msk_magnus_from_weights(s.ctx, 1, 2, msk.MSK_F64, torch.tensor(rec, device="cuda"), out)
    u0 = disc.vec(disc.gaussian_initial(w))
    BA = comm(B, A)
    for p in range(2):
        wB, wA, wAA, wBA, wBAA, wBAB = w6[p]
        Om = wB * B + wA * A + wAA * (A @ A) + wBA * BA + wBAA * comm(BA, A) + wBAB * comm(BA, B)
        ref = u0 + Om @ u0
        assert np.abs(out[p].cpu().numpy().ravel() - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_general_magnus_matches_the_oracle(order):
    w = case(20)
    B, A = oracle_ops(w, COEFS)
    s = general_solver(w)
    got = s.magnus(order, 4, precision=msk.MSK_F64).cpu().numpy()
    got32 = s.magnus(order, 4, precision=msk.MSK_F32).cpu().numpy()
    ref = np.stack([oracle_magnus(w, B, A, order, 4, p) for p in range(w.paths)])
    assert rel_l2(got, ref).max() <= TOL64
    assert rel_l2(got32, ref).max() <= TOL32
    s.close()


def test_general_euler_matches_the_oracle():
    w = case(20, n_fine=400)
    B, A = oracle_ops(w, COEFS)
    s = general_solver(w)
    got = s.euler(400, precision=msk.MSK_F64).cpu().numpy()
    got32 = s.euler(400, precision=msk.MSK_F32).cpu().numpy()
    dt = w.T / 400
    for p in range(w.paths):
        U = disc.vec(disc.gaussian_initial(w))
        for dW in brownian.coarse_increments(w, p, 400):
            U = U + dt * (B @ U) + dW * (A @ U)
        assert rel_l2(got[p:p + 1], U[None]).max() <= TOL64
        assert rel_l2(got32[p:p + 1], U[None]).max() <= TOL32
    s.close()


def test_operator_traces_and_norm_bounds():
    w = case(16, paths=2, n_fine=64)
    B, A = oracle_ops(w, COEFS)
    s = general_solver(w)
    Wt = s.weights(3, 4, precision=msk.MSK_F64).cpu().numpy()
    F = s.functionals(4).cpu().numpy()
    n = w.d * w.d
    for p in range(w.paths):
        for k in range(4):
            Y = omagnus.omega_const(B, A, w.T / 4, *(F[p, k, i] for i in (msk.MSK_F_DW, msk.MSK_F_I1,
                                                                           msk.MSK_F_I2, msk.MSK_F_I3)), 3).toarray()
            mu = np.trace(Y) / n
            assert abs(Wt[p, k, msk.MSK_WT_MU] - mu) <= 1e-12 * max(1.0, abs(mu))
            exact = np.abs(Y - mu * np.eye(n)).sum(axis=1).max()
            assert exact <= Wt[p, k, msk.MSK_WT_NORM] * (1 + 1e-12) <= 3.0 * exact * (1 + 1e-12)
    s.close()


def test_langevin_coefficients_reproduce_the_variable_coefficient_engine():
    """The paper's Section 3.2 operators written as general coefficients."""
    w = PAPER_VAR[0].with_(d=40, n_fine=400, paths=3)
    psi = lambda x: 1.0 + 1.0 / (1.0 + x * x)
    zero = lambda x, v: 0.0 * x
    cf = dict(h=zero, fx=lambda x, v: w.drift_sign * v + 0 * x, fv=zero, gxx=zero, gxv=zero,
              gvv=lambda x, v: w.a0 * psi(x) + 0 * v, s=zero, sx=zero, sv=lambda x, v: w.s0 * np.sqrt(psi(x)) + 0 * v)
    sv = msk.Solver(w)
    ref = sv.magnus(3, 8, precision=msk.MSK_F64).cpu().numpy()
    ref_e = sv.euler(400, precision=msk.MSK_F64).cpu().numpy()
    sv.close()
    s = general_solver(w, cf)
    assert rel_l2(s.magnus(3, 8, precision=msk.MSK_F64).cpu().numpy(), ref).max() <= 1e-12
    assert rel_l2(s.euler(400, precision=msk.MSK_F64).cpu().numpy(), ref_e).max() <= 1e-12
    s.close()


def test_general_on_a_cluster_float_against_double():
    w = case(100, ax=-4.0, bx=4.0, av=-4.0, bv=4.0, n_fine=1000, paths=4)
    s = general_solver(w)
    u64, st = s.magnus(3, 20, precision=msk.MSK_F64, status=True)
    u32 = s.magnus(3, 20, precision=msk.MSK_F32)
    assert int(st.max()) == 0
    assert rel_l2(u32.cpu().numpy(), u64.cpu().numpy()).max() <= TOL32
    s.close()


def test_unsupported_calls_and_bad_values():
    w = case(16, paths=1)
    s = general_solver(w)
    out = s.state(1, msk.MSK_F64)
    with pytest.raises(msk.MskError) as e:
        msk.msk_explicit_solution(s.ctx, 1, out)
    assert e.value.status == msk.MSK_ERR_UNSUPPORTED
    g = grids(w, COEFS)
    g[4, 3, 2] = np.nan
    with pytest.raises(msk.MskError) as e:
        msk.msk_set_general_coefficients(s.ctx, g)
    assert e.value.status == msk.MSK_ERR_NONFINITE
    msk.msk_set_general_coefficients(s.ctx, None)        # back to the Langevin operators
    msk.msk_explicit_solution(s.ctx, 1, out)
    s.close()

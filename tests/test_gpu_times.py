"""GPU parity of the solutions at several output times inside the Magnus sub-intervals
(Section 3, "Implementation"): against the oracle's exp(Y(t_n, t)) u(t_n) for constant,
time-dependent and x-dependent coefficients, and against the plain solve at t = T."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from oracle import magnus as omagnus  # noqa: E402
from workloads import COEF_TRIG, LANGEVIN_32, LANGEVIN_TRIG_128, PAPER_VAR  # noqa: E402

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


def check(w, order, K, cells, paths):
    s = msk.Solver(w)
    got = s.magnus_times(order, K, cells, paths=paths, precision=msk.MSK_F64).cpu().numpy()
    got32, st = s.magnus_times(order, K, cells, paths=paths, precision=msk.MSK_F32, status=True)
    for p in range(paths):
        ref = omagnus.solve_times(w, order, K, p, cells)
        assert rel_l2(got[p], ref).max() <= TOL64
        assert rel_l2(got32[p].cpu().numpy(), ref).max() <= TOL32
    assert st.numel() == paths * len(cells) and int(st.max()) == 0
    s.close()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_output_times_constant_coefficients(order):
    """d = 32, K = 4 steps of 60 cells: times inside steps, two in one step, step ends, T."""
    w = LANGEVIN_32.with_(n_fine=240, paths=3)
    check(w, order, 4, [13, 60, 61, 100, 101, 180, 239, 240], 3)


def test_output_times_time_dependent_coefficients():
    w = LANGEVIN_TRIG_128.with_(d=32, n_fine=256, paths=2)
    check(w, 3, 8, [5, 32, 47, 128, 200, 256], 2)


def test_output_times_on_a_cluster():
    """d = 128 in double runs on clusters of two CTAs (halo rows read from the output slot)."""
    w = LANGEVIN_TRIG_128.with_(paths=2, n_fine=512)
    s = msk.Solver(w)
    cells = [40, 64, 300, 512]
    got = s.magnus_times(3, 8, cells, paths=2, precision=msk.MSK_F64).cpu().numpy()
    for p in range(2):
        assert rel_l2(got[p], omagnus.solve_times(w, 3, 8, p, cells)).max() <= TOL64
    s.close()


def test_output_times_variable_coefficients():
    w = PAPER_VAR[0].with_(d=24, n_fine=240, paths=2)
    check(w, 3, 4, [30, 60, 90, 200, 240], 2)


@pytest.mark.parametrize("prec,tol", [(msk.MSK_F64, 1e-13), (msk.MSK_F32, 1e-6)])
def test_output_at_T_equals_the_plain_solve(prec, tol):
    w = LANGEVIN_TRIG_128.with_(d=64, n_fine=1024, paths=16)
    s = msk.Solver(w)
    u = s.magnus_times(3, 8, [512, 1024], precision=prec)
    ref = s.magnus(3, 8, precision=prec)
    assert rel_l2(u[:, 1].double().cpu().numpy(), ref.double().cpu().numpy()).max() <= tol
    ref_half = msk.Solver(w.with_(T=0.5, n_fine=512)).magnus(3, 4, precision=prec)
    assert rel_l2(u[:, 0].double().cpu().numpy(), ref_half.double().cpu().numpy()).max() <= tol
    s.close()


def test_bad_output_times_are_rejected():
    w = LANGEVIN_32.with_(n_fine=240, paths=1)
    s = msk.Solver(w)
    out = torch.empty(4 * 32 * 32, dtype=torch.float64, device="cuda")
    for cells in ([0, 10], [10, 10], [20, 10], [241]):
        with pytest.raises(msk.MskError) as e:
            msk.msk_solve_magnus_times(s.ctx, 2, 4, 1, msk.MSK_F64, cells, out)
        assert e.value.status == msk.MSK_ERR_ARG
    s.close()

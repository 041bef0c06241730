"""Sampled paths of the step-size experiments (Section 3.1 Fig. StepTest, Section 3.2
Fig. StepTestVar) against the CPU oracle: d = 200, the paper's coefficients, the same
fine Brownian grids as the bench sweep, float Taylor arithmetic (<= 1e-4)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from oracle import magnus as omagnus  # noqa: E402
from workloads import PAPER_CONST, PAPER_VAR  # noqa: E402

TOL32 = 1e-4
NFINE_CONST = 1_201_200      # the constant-coefficient sweep's fine grid (divisible by every step count)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2207_09776_b300 import build
    build.build()
    msk.load_library()


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("order,K", [(2, 16), (3, 12)])
def test_constant_sweep_sampled_path(order, K):
    """Constant coefficients on the variable-coefficient engine with psi = 1 (d = 200 is
    not a multiple of 32), path 7 of 8 at step 1/K."""
    w = PAPER_CONST.with_(d=200, n_fine=NFINE_CONST, paths=8)
    s = msk.Solver(w)
    msk.msk_set_x_profile(s.ctx, msk.MSK_XPROF_VALUES, psi=[1.0] * w.d)
    u, st = s.magnus(order, K, precision=msk.MSK_F32, status=True)
    assert int(st[7]) == 0           # other paths may explode at these steps (the scheme, not the code)
    ref = omagnus.solve(w, order, K, [7])
    assert rel_l2(u[7:].cpu().numpy(), ref).max() <= TOL32
    s.close()


def test_x_profile_sweep_sampled_path():
    """The x profile psi = 1 + 1/(1 + x^2) (Eq. coeffsLangevinVar), order 3, step 0.04."""
    w = PAPER_VAR[1].with_(paths=4)
    s = msk.Solver(w)
    u, st = s.magnus(3, 25, precision=msk.MSK_F32, status=True)
    assert int(st[3]) == 0
    ref = omagnus.solve(w, 3, 25, [3])
    assert rel_l2(u[3:].cpu().numpy(), ref).max() <= TOL32
    s.close()


def test_float_explodes_only_where_double_does():
    """Order 3 at step 0.2 (beyond the stable range): the float solves flag exactly the
    paths the double solves flag -- the Brownian part of each Taylor sub-step is small
    enough for float rounding (without that bound float flags most paths here)."""
    w = PAPER_CONST.with_(d=200, n_fine=NFINE_CONST, paths=100)
    s = msk.Solver(w)
    msk.msk_set_x_profile(s.ctx, msk.MSK_XPROF_VALUES, psi=[1.0] * w.d)
    _, st32 = s.magnus(3, 5, precision=msk.MSK_F32, status=True)
    _, st64 = s.magnus(3, 5, precision=msk.MSK_F64, status=True)
    assert torch.equal(st32[: w.paths] != 0, st64[: w.paths] != 0)
    assert int((st64[: w.paths] != 0).sum()) <= 10
    s.close()

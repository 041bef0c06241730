"""Step-size control by the order-2 / order-3 distance (Remark stepSizeControl)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from oracle import magnus as omagnus  # noqa: E402
from workloads import LANGEVIN_TRIG_128  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2207_09776_b300 import build
    build.build()
    msk.load_library()


def _oracle_distance(w, K, paths):
    u2 = omagnus.solve(w, 2, K, paths).reshape(len(paths), -1)
    u3 = omagnus.solve(w, 3, K, paths).reshape(len(paths), -1)
    return float(np.max(np.linalg.norm(u3 - u2, axis=1) / np.linalg.norm(u3, axis=1)))


def test_distances_match_the_oracle_and_the_first_accepted_step_count_is_returned():
    w = LANGEVIN_TRIG_128.with_(d=64, paths=3, n_fine=1024)
    s = msk.Solver(w)
    K, d = msk.msk_select_steps(s.ctx, 1e-30, 2, 8, 3, msk.MSK_F64)   # nothing accepted: all of 2, 4, 8
    assert K == 8 and len(d) == 3
    for k, dk in zip((2, 4, 8), d):
        assert dk == pytest.approx(_oracle_distance(w, k, [0, 1, 2]), rel=1e-6)
    assert d[0] > d[1] > d[2] > 0                                      # orders 2 and 3 converge together
    tol = 0.5 * (d[0] + d[1])
    K, dd = msk.msk_select_steps(s.ctx, tol, 2, 8, 3, msk.MSK_F64)
    assert K == 4 and len(dd) == 2 and dd == pytest.approx(d[:2], rel=1e-12)
    K, dd = msk.msk_select_steps(s.ctx, 1.0, 2, 8, 3, msk.MSK_F64)
    assert K == 2 and len(dd) == 1
    # the float solves (float normals, float Taylor action) give the same distances to ~1e-4
    K, d32 = msk.msk_select_steps(s.ctx, 1e-30, 2, 8, 3, msk.MSK_F32)
    assert K == 8 and d32 == pytest.approx(d, rel=1e-2, abs=1e-5)
    s.close()


def test_step_selection_arguments():
    w = LANGEVIN_TRIG_128.with_(d=32, paths=2, n_fine=1000)
    s = msk.Solver(w)
    with pytest.raises(msk.MskError):
        msk.msk_select_steps(s.ctx, 1e-3, 3, 3, 2, msk.MSK_F64)     # 3 does not divide 1000
    with pytest.raises(msk.MskError):
        msk.msk_select_steps(s.ctx, 0.0, 2, 8, 2, msk.MSK_F64)      # tol must be positive
    with pytest.raises(msk.MskError):
        msk.msk_select_steps(s.ctx, 1e-3, 8, 2, 2, msk.MSK_F64)     # k_min > k_max
    K, d = msk.msk_select_steps(s.ctx, 1e-30, 4, 100, 2, msk.MSK_F64)   # 4, 8 divide 1000; 16 does not
    assert K == 8 and len(d) == 2
    s.close()

"""msk_solve_magnus_noalloc: the solve for callers that cannot allocate device
memory (their memory belongs to another allocator, or cudaMalloc/cudaFree would
synchronise a latency-bound loop).  Its scratch is a static device array, so
its output must equal msk_solve_magnus's on the same inputs, call after call,
and oversized requests must be refused before any device work.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from workloads import LANGEVIN_32, LANGEVIN_TRIG_128  # noqa: E402

TOL = {msk.MSK_F64: 1e-10, msk.MSK_F32: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2207_09776_b300 import build
    build.build()
    msk.load_library()


def rel_l2(a, b):
    a = a.double().reshape(a.shape[0], -1)
    b = b.double().reshape(b.shape[0], -1)
    return ((a - b).norm(dim=1) / b.norm(dim=1)).max().item()


@pytest.mark.parametrize("w,order,K,precision", [
    (LANGEVIN_TRIG_128.with_(d=64, paths=37, n_fine=1024), 3, 8, msk.MSK_F32),
    (LANGEVIN_TRIG_128.with_(d=64, paths=5, n_fine=1024), 2, 4, msk.MSK_F64),
    (LANGEVIN_32.with_(paths=11), 2, 1, msk.MSK_F64),
])
def test_noalloc_matches_the_allocating_solve_twice(w, order, K, precision):
    s = msk.Solver(w)
    ref = s.magnus(order, K, precision=precision)
    for _ in range(2):                         # the static scratch keeps the previous call's contents
        out = s.state(w.paths, precision)
        st = torch.full((w.paths,), 7, dtype=torch.int32, device="cuda")
        msk.msk_solve_magnus_noalloc(s.ctx, order, K, w.paths, precision, out, st)
        torch.cuda.synchronize()
        assert rel_l2(out, ref) <= TOL[precision]
        assert int(st.max()) == 0
    s.close()


def test_noalloc_refuses_requests_beyond_the_static_scratch():
    w = LANGEVIN_32.with_(paths=100000, n_fine=10000)
    s = msk.Solver(w)
    # the library refuses before touching the output (called directly: the binding would
    # refuse the one-element buffer itself)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    lib = msk.load_library()
    st = lib.msk_solve_magnus_noalloc(s.ctx, 2, 1, 100000, msk.MSK_F64, out.data_ptr(), None,
                                      torch.cuda.current_stream().cuda_stream)   # 2.8e6 doubles > 2^21
    assert st == msk.MSK_ERR_ARG
    assert "static scratch" in msk.msk_last_error(s.ctx)
    # the context is still usable after the refusal
    u = s.state(3)
    msk.msk_solve_magnus_noalloc(s.ctx, 2, 1, 3, msk.MSK_F64, u)
    assert rel_l2(u, s.magnus(2, 1, paths=3)) <= TOL[msk.MSK_F64]
    s.close()

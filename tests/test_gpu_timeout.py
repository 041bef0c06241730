"""The bounded waits of the tensor-core GEMM, made to run out on a healthy pipeline.

With the test hook on, every GEMM's epilogue warps first wait on an mbarrier that no
thread ever arrives at; the wait gives up after a bounded number of polls, the warps
skip their tiles while still releasing each accumulator, the producer waits for its
issued TMA loads and the MMA issuer for its issued MMAs, and the call reports
MSK_ERR_TIMEOUT through msk_surrogate_sync_status.  No fault, trap or hang is
involved.  Afterwards the same GPU context still computes correct results: a fresh
surrogate's forward pass matches the oracle and a Magnus solve matches the solve
made before the timeout."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from oracle import surrogate as sg  # noqa: E402
from workloads import LANGEVIN_TRIG_128  # noqa: E402

DIMS = [48, 64, 64, 8]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2207_09776_b300 import build
    build.build()
    msk.load_library()


def _surrogate(solver, seed):
    s = msk.msk_surrogate_create(solver.ctx, steps=16, rank=8, hidden=64, layers=2, train_batch=96,
                                 infer_batch=256)
    rng = np.random.default_rng(seed)
    flat = np.zeros(msk.msk_surrogate_num_params(s), np.float32)
    params = []
    for l, (ow, ob) in enumerate(msk.msk_surrogate_param_layout(s, 2)):
        W = (rng.normal(size=(DIMS[l + 1], DIMS[l])) * math.sqrt(2.0 / DIMS[l])).astype(np.float32)
        b = (rng.normal(size=DIMS[l + 1]) * 0.1).astype(np.float32)
        flat[ow:ow + W.size] = W.ravel()
        flat[ob:ob + b.size] = b
        params.append((W.astype(np.float64), b.astype(np.float64)))
    msk.msk_surrogate_set_params(s, torch.tensor(flat, device="cuda"))
    return s, params


def test_a_tensor_core_wait_that_runs_out_is_reported_and_the_context_survives():
    w = LANGEVIN_TRIG_128.with_(d=32, n_fine=1024, paths=8)
    solver = msk.Solver(w)
    before = solver.magnus(3, 8, precision=msk.MSK_F32)
    B = 200
    rng = np.random.default_rng(5)
    X = sg.to_bf16(rng.normal(size=(B, 48)))
    Xd = torch.tensor(np.asarray(X, np.float32), device="cuda").to(torch.bfloat16)
    out = torch.zeros(B, DIMS[-1], device="cuda")

    s, _ = _surrogate(solver, 1)
    msk.msk_surrogate_set_wait_test(s, 1)
    msk.msk_surrogate_forward(s, Xd, B, out)          # three GEMMs, each wait runs out
    with pytest.raises(msk.MskError) as e:
        msk.msk_surrogate_sync_status(s)
    assert e.value.status == msk.MSK_ERR_TIMEOUT
    msk.msk_surrogate_destroy(s)

    # the context is healthy: a fresh surrogate computes the oracle's forward pass ...
    s2, params = _surrogate(solver, 1)
    msk.msk_surrogate_forward(s2, Xd, B, out)
    msk.msk_surrogate_sync_status(s2)
    want, _ = sg.forward(params, X, bf16=True)
    got = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-3
    msk.msk_surrogate_destroy(s2)
    # ... and the solver reproduces its earlier result bit for bit
    after = solver.magnus(3, 8, precision=msk.MSK_F32)
    torch.cuda.synchronize()
    assert torch.equal(after, before)
    solver.close()

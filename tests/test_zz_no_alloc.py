"""msk_solve_magnus_noalloc: the solve for callers that cannot allocate device
memory (their memory belongs to another allocator, or cudaMalloc/cudaFree would
synchronise a latency-bound loop).  Its scratch is a static device array; the
kernels it launches are the ones msk_solve_magnus launches, on the same inputs,
so its output must equal msk_solve_magnus's bit for bit, call after call, for the
constant, time-dependent, x-profile and general-coefficient engines alike.
Oversized requests must be refused before any device work.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2207_09776_b300 as msk  # noqa: E402
from workloads import LANGEVIN_32, LANGEVIN_TRIG_128, PAPER_VAR  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2207_09776_b300 import build
    build.build()
    msk.load_library()


def _general_grids(w):
    """[9][v][x] values of smooth coefficient functions with every term of Eq. generalSPDE."""
    from oracle import discretization as disc
    xs, _ = disc.grid(w.d, w.ax, w.bx)
    vs, _ = disc.grid(w.d, w.av, w.bv)
    X, V = np.meshgrid(xs, vs, indexing="xy")
    f = [-0.1 * (1 + 0.2 * np.sin(X)), -V + 0.1 * np.cos(X), 0.2 * np.sin(X) - 0.1 * V,
         0.05 + 0.01 * np.cos(V), 0.02 * np.exp(-0.1 * X * X), 1.0 + 0.1 * np.cos(X * V / 4),
         0.1 + 0.0 * X, 0.05 * np.cos(V), 0.3 * (1 + 0.2 * np.sin(X))]
    return np.stack([np.broadcast_to(g, X.shape) for g in f])


def _solver(w, general=False):
    s = msk.Solver(w)
    if general:
        msk.msk_set_general_coefficients(s.ctx, _general_grids(w))
    return s


CASES = [
    ("trig_d64_f32", LANGEVIN_TRIG_128.with_(d=64, paths=37, n_fine=1024), False, 3, 8, msk.MSK_F32),
    ("trig_d64_f64", LANGEVIN_TRIG_128.with_(d=64, paths=5, n_fine=1024), False, 2, 4, msk.MSK_F64),
    ("const_d32_f64", LANGEVIN_32.with_(paths=11), False, 2, 1, msk.MSK_F64),
    ("xprofile_d100_f32", PAPER_VAR[0].with_(paths=6, n_fine=400), False, 3, 20, msk.MSK_F32),
    ("xprofile_trig_d40_f64", PAPER_VAR[0].with_(d=40, paths=3, n_fine=240, kind=LANGEVIN_TRIG_128.kind,
                                                  a1=0.3, s1=0.3), False, 3, 6, msk.MSK_F64),
    ("general_d48_f32", LANGEVIN_32.with_(d=48, ax=-3.0, bx=3.0, av=-3.0, bv=3.0, n_fine=240, paths=4),
     True, 3, 4, msk.MSK_F32),
]


@pytest.mark.parametrize("name,w,general,order,K,precision", CASES, ids=[c[0] for c in CASES])
def test_noalloc_equals_the_allocating_solve_bit_for_bit(name, w, general, order, K, precision):
    s = _solver(w, general)
    ref = s.magnus(order, K, precision=precision)
    ref_st = torch.full((w.paths,), 7, dtype=torch.int32, device="cuda")
    msk.msk_solve_magnus(s.ctx, order, K, w.paths, precision, s.state(w.paths, precision), ref_st)
    for _ in range(2):                         # the static scratch keeps the previous call's contents
        out = s.state(w.paths, precision)
        st = torch.full((w.paths,), 7, dtype=torch.int32, device="cuda")
        msk.msk_solve_magnus_noalloc(s.ctx, order, K, w.paths, precision, out, st)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), f"{name}: max |diff| {(out.double() - ref.double()).abs().max().item()}"
        assert torch.equal(st, ref_st)
    s.close()


@pytest.mark.parametrize("general", [False, True], ids=["xprofile", "general"])
def test_noalloc_first_solve_of_a_fresh_context_takes_no_device_memory(general):
    """The operator table of the x-profile and general-coefficient engines is allocated
    when the profile or coefficients are set, not by the first solve: the first
    no-alloc solve of a fresh context leaves the device's free memory unchanged.  A
    first context runs the same call beforehand, so every kernel it launches is loaded."""
    w = (LANGEVIN_32.with_(d=48, ax=-3.0, bx=3.0, av=-3.0, bv=3.0, n_fine=240, paths=4) if general
         else PAPER_VAR[0].with_(d=40, paths=4, n_fine=240))
    warm = _solver(w, general)
    out = warm.state(w.paths, msk.MSK_F32)
    msk.msk_solve_magnus_noalloc(warm.ctx, 3, 4, w.paths, msk.MSK_F32, out)
    torch.cuda.synchronize()
    fresh = _solver(w, general)
    out2 = fresh.state(w.paths, msk.MSK_F32)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    msk.msk_solve_magnus_noalloc(fresh.ctx, 3, 4, w.paths, msk.MSK_F32, out2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out2, out)
    warm.close()
    fresh.close()


def test_noalloc_refuses_requests_beyond_the_static_scratch():
    w = LANGEVIN_32.with_(paths=100000, n_fine=10000)
    s = msk.Solver(w)
    # the library refuses before touching the output (called directly: the binding would
    # refuse the one-element buffer itself)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    lib = msk.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    for paths, steps in ((100000, 1),            # 2.8e6 doubles > 2^21
                         (2 ** 62 + 1000, 1),     # paths * 28 wraps around 2^64 without the division check
                         (2 ** 40, 10000)):
        st = lib.msk_solve_magnus_noalloc(s.ctx, 2, steps, paths, msk.MSK_F64, out.data_ptr(), None, stream)
        assert st == msk.MSK_ERR_ARG
        assert "static scratch" in msk.msk_last_error(s.ctx)
    # the streamed engine needs library scratch: refused, before any device work
    msk.msk_set_engine(s.ctx, msk.MSK_ENGINE_STREAMED)
    st = lib.msk_solve_magnus_noalloc(s.ctx, 2, 1, 3, msk.MSK_F64, out.data_ptr(), None, stream)
    assert st == msk.MSK_ERR_UNSUPPORTED
    msk.msk_set_engine(s.ctx, msk.MSK_ENGINE_AUTO)
    # the context is still usable after the refusals
    u = s.state(3)
    msk.msk_solve_magnus_noalloc(s.ctx, 2, 1, 3, msk.MSK_F64, u)
    assert torch.equal(u, s.magnus(2, 1, paths=3))
    s.close()

"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, the binding declares the same names, and argument validation
rejects bad calls before any device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2207_09776_b300 as msk
from paper_2207_09776_b300 import build as _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msk.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(msk_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return msk.load_library()


def test_header_declares_the_boundary():
    names = header_functions()
    for n in ("msk_create", "msk_destroy", "msk_set_coefficients", "msk_set_seed", "msk_solve_magnus",
              "msk_solve_euler", "msk_error", "msk_moments", "msk_brownian_functionals",
              "msk_omega_weights", "msk_explicit_solution"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert set(header_functions()) == set(msk.SIGNATURES)
    for name in header_functions():
        assert callable(getattr(msk, name))


def test_argument_validation_needs_no_device(lib):
    h = ctypes.c_void_p()
    bad = [msk.msk_grid(7, 7, -1, 1, -1, 1), msk.msk_grid(513, 513, -1, 1, -1, 1),
           msk.msk_grid(32, 64, -1, 1, -1, 1), msk.msk_grid(32, 32, 1, -1, -1, 1)]
    for g in bad:
        assert lib.msk_create(ctypes.byref(h), ctypes.byref(g), 0) == msk.MSK_ERR_ARG
        assert h.value is None
    g = msk.msk_grid(32, 32, float("nan"), 1, -1, 1)
    assert lib.msk_create(ctypes.byref(h), ctypes.byref(g), 0) == msk.MSK_ERR_NONFINITE
    assert lib.msk_create(None, ctypes.byref(g), 0) == msk.MSK_ERR_ARG
    # calls on a NULL context fail with MSK_ERR_ARG, destroy(NULL) is a no-op
    assert lib.msk_solve_magnus(None, 2, 1, 1, 0, None, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_solve_magnus_host(None, 2, 1, 1, 0, None, None, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_magnus_from_weights(None, 1, 1, 0, None, None, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_set_x_profile(None, msk.MSK_XPROF_RATIONAL, 1.0, None) == msk.MSK_ERR_ARG
    assert lib.msk_solve_euler(None, 1, 1, 0, None, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_set_seed(None, 1, 0, 100, 1.0) == msk.MSK_ERR_ARG
    assert lib.msk_philox_words(1, 1, 0, -1, 1, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_philox_words(1, 1, 0, 0, 0, None, None) == msk.MSK_OK
    lib.msk_destroy(None)
    assert lib.msk_last_error(None) == b"null context"
    assert lib.msk_brownian_functionals_ex(None, 1, 1, 0, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_select_steps(None, 1e-3, 1, 8, 1, 0, None, None, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_set_general_coefficients(None, None) == msk.MSK_ERR_ARG
    cells = (ctypes.c_int64 * 2)(10, 20)
    assert lib.msk_solve_magnus_times(None, 3, 4, 1, 0, cells, 2, None, None, None) == msk.MSK_ERR_ARG
    # surrogate: NULL handles and missing arguments are rejected before any device work
    cfg = msk.msk_surrogate_config(16, 64, 512, 4, 4096, 65536, 3, 8, 0)
    assert lib.msk_surrogate_create(ctypes.byref(h), None, ctypes.byref(cfg)) == msk.MSK_ERR_ARG
    assert h.value is None
    assert lib.msk_surrogate_create(None, None, ctypes.byref(cfg)) == msk.MSK_ERR_ARG
    assert lib.msk_surrogate_num_params(None) == -1
    assert lib.msk_surrogate_infer(None, 0, 1, None, None, 0, 0.01, 0.05, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_surrogate_train(None, None, None, 1, 1, 1e-3, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_surrogate_fit_pod(None, None, 1, None, None) == msk.MSK_ERR_ARG
    assert lib.msk_surrogate_sync_status(None, None) == msk.MSK_ERR_ARG
    assert lib.msk_surrogate_param_layout(None, None) == msk.MSK_ERR_ARG
    lib.msk_surrogate_destroy(None)
    assert lib.msk_surrogate_last_error(None) == b"null surrogate"


def test_create_without_a_device_reports_a_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    g = msk.msk_grid(32, 32, -5, 5, -5, 5)
    assert lib.msk_create(ctypes.byref(h), ctypes.byref(g), 0) in (msk.MSK_ERR_CUDA, msk.MSK_ERR_OOM)
    assert h.value is None


def test_header_constants_match_the_binding():
    """Every numeric constant of include/msk.h (the #defines and the enum members, with
    C's implicit numbering) that the binding exports has the header's value, and every
    #define is exported: the binding passes these integers straight through the ABI."""
    text = re.sub(r"/\*.*?\*/", " ", open(HEADER).read(), flags=re.S)
    values = {}
    for name, val in re.findall(r"#define\s+(MSK_\w+)\s+(-?\d+)u?\b", text):
        values[name] = int(val)
    defines = set(values)
    for body in re.findall(r"enum\s*\w*\s*\{([^}]*)\}", text):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            if "=" in item:
                name, val = (s.strip() for s in item.split("="))
                nxt = int(val)
            else:
                name = item
            values[name] = nxt
            nxt += 1
    assert values["MSK_ENGINE_SPLIT"] == 3 and values["MSK_OP_BX"] == 0 and values["MSK_ERR_UNSUPPORTED"] == 6
    for name, val in values.items():
        if name in defines:
            assert hasattr(msk, name), name
        if hasattr(msk, name):
            assert getattr(msk, name) == val, (name, getattr(msk, name), val)

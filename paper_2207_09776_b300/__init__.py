"""Python binding of libmsk, the B300 stochastic Magnus solver (C ABI in include/msk.h).

Argument marshalling only: every numerical step runs in the CUDA kernels of
libmsk.so.  Device buffers are torch tensors on the context's CUDA device;
work is enqueued on the current torch stream unless a stream is given.
Loading fails loudly if the library has not been built (there is no CPU
fallback).

The functions carry the C names (msk_create, msk_solve_magnus, ...); the
`Solver` class bundles a context with tensor allocation for convenience.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsk.so")

MSK_OK, MSK_ERR_ARG, MSK_ERR_CUDA, MSK_ERR_OOM, MSK_ERR_TIMEOUT, MSK_ERR_NONFINITE, MSK_ERR_UNSUPPORTED = range(7)
MSK_COEF_CONST, MSK_COEF_TRIG = 0, 1
MSK_XPROF_NONE, MSK_XPROF_RATIONAL, MSK_XPROF_VALUES = 0, 1, 2
MSK_F64, MSK_F32 = 0, 1
MSK_REF_EXPLICIT, MSK_REF_BUFFER = 0, 1
MSK_PATH_NONFINITE, MSK_PATH_SCALE_CAP, MSK_PATH_BLOWUP = 1, 2, 4
MSK_NF, MSK_NOPS, MSK_NWT = 8, 13, 20
MSK_F_DW, MSK_F_I1, MSK_F_I2, MSK_F_I3, MSK_F_OM, MSK_F_JOM, MSK_F_G1, MSK_F_G2 = range(8)
MSK_WT_ALPHA, MSK_WT_WORK, MSK_WT_EPS = 13, 14, 15
MSK_WT_MU, MSK_WT_NORM, MSK_WT_S, MSK_WT_M = 16, 17, 18, 19
OP_NAMES = ("Bx", "Bvv", "A0", "A0A0", "[Bx,A0]", "[Bvv,A0]", "[Bx,Bvv]", "[[Bx,A0],A0]",
            "[[Bvv,A0],A0]", "[[Bx,A0],Bx]", "[[Bx,A0],Bvv]", "[[Bvv,A0],Bx]", "[[Bvv,A0],Bvv]")
STATUS_NAMES = {0: "MSK_OK", 1: "MSK_ERR_ARG", 2: "MSK_ERR_CUDA", 3: "MSK_ERR_OOM",
                4: "MSK_ERR_TIMEOUT", 5: "MSK_ERR_NONFINITE", 6: "MSK_ERR_UNSUPPORTED"}


class msk_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nv", ctypes.c_int32), ("ax", ctypes.c_double),
                ("bx", ctypes.c_double), ("av", ctypes.c_double), ("bv", ctypes.c_double)]


class msk_coeffs(ctypes.Structure):
    _fields_ = [("drift_sign", ctypes.c_int32), ("kind", ctypes.c_int32), ("a0", ctypes.c_double),
                ("a1", ctypes.c_double), ("s0", ctypes.c_double), ("s1", ctypes.c_double)]


class msk_gaussian(ctypes.Structure):
    _fields_ = [("mean_x", ctypes.c_double), ("mean_v", ctypes.c_double), ("cov_xx", ctypes.c_double),
                ("cov_xv", ctypes.c_double), ("cov_vv", ctypes.c_double), ("scale", ctypes.c_double)]


class msk_surrogate_config(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("rank", ctypes.c_int32), ("hidden", ctypes.c_int32),
                ("layers", ctypes.c_int32), ("train_batch", ctypes.c_int32), ("infer_batch", ctypes.c_int32),
                ("ref_order", ctypes.c_int32), ("ref_steps", ctypes.c_int32), ("init_seed", ctypes.c_uint64)]


class msk_batch_item(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("order", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("paths", ctypes.c_int64), ("u_out_dev", ctypes.c_void_p), ("status_dev", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_INT = ctypes.c_int
_DBL = ctypes.c_double

# name -> (restype, argtypes); mirrors include/msk.h
SIGNATURES = {
    "msk_create": (_INT, [ctypes.POINTER(_P), ctypes.POINTER(msk_grid), _INT]),
    "msk_destroy": (None, [_P]),
    "msk_last_error": (ctypes.c_char_p, [_P]),
    "msk_set_coefficients": (_INT, [_P, ctypes.POINTER(msk_coeffs)]),
    "msk_set_initial_gaussian": (_INT, [_P, ctypes.POINTER(msk_gaussian)]),
    "msk_set_x_profile": (_INT, [_P, _INT, _DBL, _P]),
    "msk_set_general_coefficients": (_INT, [_P, _P]),
    "msk_set_initial": (_INT, [_P, _P, _P]),
    "msk_set_seed": (_INT, [_P, _U64, _U64, _I64, _DBL]),
    "msk_philox_words": (_INT, [_U64, _U64, ctypes.c_uint32, _I64, _I64, _P, _P]),
    "msk_brownian_functionals": (_INT, [_P, _INT, _I64, _P, _P]),
    "msk_brownian_functionals_ex": (_INT, [_P, _INT, _I64, _INT, _P, _P]),
    "msk_brownian_increments": (_INT, [_P, _INT, _I64, _P, _P]),
    "msk_omega_weights": (_INT, [_P, _INT, _INT, _I64, _INT, _P, _P, _P]),
    "msk_power_norms": (_INT, [_P, _INT, _INT, _P, ctypes.POINTER(_INT), _P]),
    "msk_fma_throughput": (_INT, [_INT, _INT, ctypes.POINTER(_DBL), _P]),
    "msk_set_engine": (_INT, [_P, _INT]),
    "msk_apply_omega": (_INT, [_P, _P, _I64, _P, _P, _P]),
    "msk_solve_magnus": (_INT, [_P, _INT, _INT, _I64, _INT, _P, _P, _P]),
    "msk_solve_magnus_host": (_INT, [_P, _INT, _INT, _I64, _INT, _P, _P, _P, _P]),
    "msk_solve_euler": (_INT, [_P, _INT, _I64, _INT, _P, _P, _P]),
    "msk_magnus_from_weights": (_INT, [_P, _INT, _I64, _INT, _P, _P, _P, _P]),
    "msk_solve_magnus_noalloc": (_INT, [_P, _INT, _INT, _I64, _INT, _P, _P, _P]),
    "msk_solve_magnus_times": (_INT, [_P, _INT, _INT, _I64, _INT, ctypes.POINTER(_I64), _INT, _P, _P, _P]),
    "msk_work_counter": (_INT, [_P, ctypes.POINTER(ctypes.c_uint64), _INT, _P]),
    "msk_batch_create": (_INT, [ctypes.POINTER(_P), ctypes.POINTER(msk_batch_item), _INT, ctypes.c_char_p]),
    "msk_batch_run": (_INT, [_P, _P]),
    "msk_batch_tune": (_INT, [_P, _P, ctypes.c_char_p, ctypes.POINTER(_INT), ctypes.POINTER(ctypes.c_float)]),
    "msk_batch_variant": (_INT, [_P]),
    "msk_batch_set_variant": (_INT, [_P, _INT]),
    "msk_batch_last_error": (ctypes.c_char_p, [_P]),
    "msk_batch_destroy": (None, [_P]),
    "msk_surrogate_create": (_INT, [ctypes.POINTER(_P), _P, ctypes.POINTER(msk_surrogate_config)]),
    "msk_surrogate_destroy": (None, [_P]),
    "msk_surrogate_last_error": (ctypes.c_char_p, [_P]),
    "msk_surrogate_num_params": (_I64, [_P]),
    "msk_surrogate_param_layout": (_INT, [_P, ctypes.POINTER(_I64)]),
    "msk_surrogate_get_params": (_INT, [_P, _P, _P]),
    "msk_surrogate_set_params": (_INT, [_P, _P, _P]),
    "msk_surrogate_features": (_INT, [_P, _I64, _I64, _P, _P]),
    "msk_surrogate_reference": (_INT, [_P, _I64, _I64, _P, _P]),
    "msk_surrogate_fit_pod": (_INT, [_P, _P, _I64, ctypes.POINTER(_DBL), _P]),
    "msk_surrogate_get_pod": (_INT, [_P, _P, _P, ctypes.POINTER(_DBL), _P]),
    "msk_surrogate_set_pod": (_INT, [_P, _P, _P, _DBL, _P]),
    "msk_surrogate_project": (_INT, [_P, _P, _I64, _P, _P]),
    "msk_surrogate_decode": (_INT, [_P, _P, _I64, _P, _P]),
    "msk_surrogate_forward": (_INT, [_P, _P, _I64, _P, _P]),
    "msk_surrogate_loss_grads": (_INT, [_P, _P, _P, _I64, _P, _P, _P]),
    "msk_surrogate_adam_step": (_INT, [_P, ctypes.c_float, _P]),
    "msk_surrogate_train": (_INT, [_P, _P, _P, _I64, _INT, ctypes.c_float, _P, _P]),
    "msk_surrogate_infer": (_INT, [_P, _I64, _I64, _P, _P, _I64, _DBL, _DBL, ctypes.POINTER(_DBL), _P]),
    "msk_surrogate_sync_status": (_INT, [_P, _P]),
    "msk_surrogate_set_wait_test": (_INT, [_P, _INT]),
    "msk_select_steps": (_INT, [_P, _DBL, _INT, _INT, _I64, _INT, ctypes.POINTER(_INT), ctypes.POINTER(_DBL),
                                ctypes.POINTER(_INT), _P]),
    "msk_explicit_solution": (_INT, [_P, _I64, _P, _P]),
    "msk_error": (_INT, [_P, _P, _INT, _I64, _INT, _P, _INT, _INT, _P, _P, _P]),
    "msk_moments": (_INT, [_P, _P, _INT, _I64, _P, _P]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmsk.so and declare its C signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmsk.so not built at {path}; run paper_2207_09776_b300/build.py")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MskError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st: int, ctx=None):
    if st != MSK_OK:
        msg = load_library().msk_last_error(ctx).decode() if ctx else ""
        raise MskError(st, msg)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    return t.data_ptr()


def _host_ptr(t) -> Optional[int]:
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("host buffers must be contiguous CPU tensors")
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dtype(precision):
    import torch
    return torch.float64 if precision == MSK_F64 else torch.float32


def _need(t, n, dtype, name):
    if t.dtype != dtype or t.numel() < n:
        raise ValueError(f"{name}: need {n} elements of {dtype}, got {t.numel()} of {t.dtype}")


# grid size d of every context created through this binding (nx = nv = d), so that
# output buffers can be checked against paths x d x d before the kernels write them
_CTX_D = {}


def _key(ctx):
    return ctx.value if hasattr(ctx, "value") else int(ctx)


def _dd(ctx) -> int:
    """d * d of the context (1 for a handle this binding did not create)."""
    d = _CTX_D.get(_key(ctx)) if ctx is not None else None
    return d * d if d else 1


def _need_status(st, n):
    if st is not None and (st.numel() < n or st.element_size() != 4):
        raise ValueError(f"status: need {n} 32-bit elements, got {st.numel()} of {st.dtype}")


# ---- thin wrappers with the C names --------------------------------------------------

def msk_create(nx: int, nv: int, ax: float, bx: float, av: float, bv: float, device: int = 0):
    h = _P()
    g = msk_grid(nx, nv, ax, bx, av, bv)
    st = load_library().msk_create(ctypes.byref(h), ctypes.byref(g), device)
    if st != MSK_OK:
        raise MskError(st, load_library().msk_last_error(None).decode())
    _CTX_D[h.value] = nx
    return h


def msk_destroy(ctx):
    if ctx is not None:
        _CTX_D.pop(_key(ctx), None)
    load_library().msk_destroy(ctx)


def msk_last_error(ctx) -> str:
    return load_library().msk_last_error(ctx).decode()


def msk_set_coefficients(ctx, drift_sign, kind, a0, a1, s0, s1):
    _check(load_library().msk_set_coefficients(ctx, ctypes.byref(msk_coeffs(drift_sign, kind, a0, a1, s0, s1))), ctx)


def msk_set_x_profile(ctx, kind, c=1.0, psi=None):
    """psi: None, or a sequence of d host values for MSK_XPROF_VALUES."""
    buf = None
    if psi is not None:
        vals = [float(x) for x in psi]
        buf = (ctypes.c_double * len(vals))(*vals)
    _check(load_library().msk_set_x_profile(ctx, kind, c, ctypes.cast(buf, _P) if buf is not None else None), ctx)


def msk_set_general_coefficients(ctx, coef=None):
    """coef: None, or 9 x d x d host values (numpy array or nested sequence) of h, f^x, f^v,
    g^xx, g^xv, g^vv, sigma, sigma^x, sigma^v on the [v][x] grid."""
    if coef is None:
        _check(load_library().msk_set_general_coefficients(ctx, None), ctx)
        return
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1))
    _check(load_library().msk_set_general_coefficients(ctx, arr.ctypes.data_as(_P)), ctx)


def msk_set_initial_gaussian(ctx, mean, cov, scale=1.0):
    g = msk_gaussian(mean[0], mean[1], cov[0], cov[1], cov[2], scale)
    _check(load_library().msk_set_initial_gaussian(ctx, ctypes.byref(g)), ctx)


def msk_set_initial(ctx, u0, stream=None):
    import torch
    _need(u0, _dd(ctx), torch.float64, "u0")
    _check(load_library().msk_set_initial(ctx, _ptr(u0), _stream(stream)), ctx)


def msk_set_seed(ctx, seed, path_offset, n_fine, T):
    _check(load_library().msk_set_seed(ctx, seed, path_offset, n_fine, T), ctx)


def msk_philox_words(seed, path, tag, first_pair, npairs, out, stream=None):
    import torch
    _need(out, 4 * npairs, torch.int32, "out")
    _check(load_library().msk_philox_words(seed, path, tag, first_pair, npairs, _ptr(out), _stream(stream)))


def msk_brownian_functionals(ctx, steps, paths, F, stream=None):
    import torch
    _need(F, paths * steps * MSK_NF, torch.float64, "F")
    _check(load_library().msk_brownian_functionals(ctx, steps, paths, _ptr(F), _stream(stream)), ctx)


def msk_brownian_functionals_ex(ctx, steps, paths, normals, F, stream=None):
    import torch
    _need(F, paths * steps * MSK_NF, torch.float64, "F")
    _check(load_library().msk_brownian_functionals_ex(ctx, steps, paths, normals, _ptr(F), _stream(stream)), ctx)


def msk_brownian_increments(ctx, steps, paths, dW, stream=None):
    import torch
    _need(dW, paths * steps, torch.float64, "dW")
    _check(load_library().msk_brownian_increments(ctx, steps, paths, _ptr(dW), _stream(stream)), ctx)


def msk_omega_weights(ctx, order, steps, paths, precision, F, Wt, stream=None):
    import torch
    _need(F, paths * steps * MSK_NF, torch.float64, "F")
    _need(Wt, paths * steps * MSK_NWT, torch.float64, "Wt")
    _check(load_library().msk_omega_weights(ctx, order, steps, paths, precision, _ptr(F), _ptr(Wt),
                                            _stream(stream)), ctx)


def msk_power_norms(ctx, order, steps, stream=None):
    """||X_n^q||_inf (q = 1..9) of the deterministic part of each step's Omega: a float
    tensor of shape (rows, 9), rows = 1 (constant coefficients), steps (time-dependent)
    or 0 (x profile / general coefficients)."""
    import torch
    lib = load_library()
    rows = ctypes.c_int(0)
    _check(lib.msk_power_norms(ctx, order, steps, None, ctypes.byref(rows), _stream(stream)), ctx)
    out = torch.empty(max(rows.value, 1) * 9, dtype=torch.float32, device="cuda")
    if rows.value:
        _check(lib.msk_power_norms(ctx, order, steps, _ptr(out), ctypes.byref(rows), _stream(stream)), ctx)
    return out[: rows.value * 9].view(rows.value, 9)


MSK_ENGINE_AUTO, MSK_ENGINE_RESIDENT, MSK_ENGINE_STREAMED, MSK_ENGINE_SPLIT = 0, 1, 2, 3


def msk_set_engine(ctx, mode):
    """Engine of the Magnus solves: MSK_ENGINE_AUTO / _RESIDENT / _STREAMED / _SPLIT."""
    _check(load_library().msk_set_engine(ctx, mode), ctx)


def msk_fma_throughput(device=0, precision=MSK_F32, stream=None):
    """Measured multiply-add throughput (TFLOP/s) of the CUDA cores."""
    v = ctypes.c_double(0.0)
    st = load_library().msk_fma_throughput(device, precision, ctypes.byref(v), _stream(stream))
    if st != MSK_OK:
        raise MskError(st, "msk_fma_throughput failed")
    return v.value


def msk_apply_omega(ctx, weights, paths, u, out, stream=None):
    _check(load_library().msk_apply_omega(ctx, _ptr(weights), paths, _ptr(u), _ptr(out), _stream(stream)), ctx)


def msk_solve_magnus(ctx, order, steps, paths, precision, u_out, status=None, stream=None):
    _need(u_out, paths * _dd(ctx), _dtype(precision), "u_out")
    _need_status(status, paths)
    _check(load_library().msk_solve_magnus(ctx, order, steps, paths, precision, _ptr(u_out), _ptr(status),
                                           _stream(stream)), ctx)


def msk_solve_magnus_host(ctx, order, steps, paths, precision, u0, u_out, status=None, stream=None):
    """msk_solve_magnus with host buffers: u0 optional float64 CPU tensor of d*d values (the initial
    datum, copied on the stream), u_out and status page-locked CPU tensors (tensor.pin_memory()),
    into which the kernels store each finished path.  Synchronise the stream before reading."""
    import torch
    _need(u_out, paths * _dd(ctx), _dtype(precision), "u_out")
    _need_status(status, paths)
    if u0 is not None:
        _need(u0, _dd(ctx), torch.float64, "u0")
    _check(load_library().msk_solve_magnus_host(ctx, order, steps, paths, precision, _host_ptr(u0),
                                                _host_ptr(u_out), _host_ptr(status), _stream(stream)), ctx)


def msk_solve_magnus_noalloc(ctx, order, steps, paths, precision, u_out, status=None, stream=None):
    """msk_solve_magnus without device allocation: scratch comes from the library's
    16 MiB static device array (see include/msk.h for the limits and sharing rules)."""
    _need(u_out, paths * _dd(ctx), _dtype(precision), "u_out")
    _need_status(status, paths)
    _check(load_library().msk_solve_magnus_noalloc(ctx, order, steps, paths, precision, _ptr(u_out), _ptr(status),
                                                   _stream(stream)), ctx)


def msk_solve_magnus_times(ctx, order, steps, paths, precision, times_cells, u_out, status=None, stream=None):
    """times_cells: output times in fine cells (strictly increasing, 1 .. n_fine);
    u_out: [paths][len(times_cells)][d][d] tensor; status: optional int32[paths * n_times]."""
    import torch
    cells = [int(c) for c in times_cells]
    arr = (_I64 * max(len(cells), 1))(*cells)
    _need(u_out, paths * len(cells) * _dd(ctx), _dtype(precision), "u_out")
    _need_status(status, paths * len(cells))
    _check(load_library().msk_solve_magnus_times(ctx, order, steps, paths, precision, arr, len(cells), _ptr(u_out),
                                                 _ptr(status), _stream(stream)), ctx)


def msk_magnus_from_weights(ctx, steps, paths, precision, Wt, u_out, status=None, stream=None):
    import torch
    _need(Wt, paths * steps * MSK_NWT, torch.float64, "Wt")
    _need(u_out, paths * _dd(ctx), _dtype(precision), "u_out")
    _need_status(status, paths)
    _check(load_library().msk_magnus_from_weights(ctx, steps, paths, precision, _ptr(Wt), _ptr(u_out),
                                                  _ptr(status), _stream(stream)), ctx)


def msk_work_counter(ctx, reset=False, stream=None) -> int:
    v = ctypes.c_uint64(0)
    _check(load_library().msk_work_counter(ctx, ctypes.byref(v), int(bool(reset)), _stream(stream)), ctx)
    return int(v.value)


def msk_select_steps(ctx, tol, k_min, k_max, paths, precision, stream=None):
    """Step-size control by the order-2 / order-3 distance; returns (K, [distance of each K tried])."""
    K = _INT(0)
    n = _INT(0)
    d = (_DBL * 16)()
    _check(load_library().msk_select_steps(ctx, tol, k_min, k_max, paths, precision, ctypes.byref(K), d,
                                           ctypes.byref(n), _stream(stream)), ctx)
    return K.value, list(d)[: n.value]


def msk_solve_euler(ctx, steps, paths, precision, u_out, status=None, stream=None):
    _need(u_out, paths * _dd(ctx), _dtype(precision), "u_out")
    _need_status(status, paths)
    _check(load_library().msk_solve_euler(ctx, steps, paths, precision, _ptr(u_out), _ptr(status),
                                          _stream(stream)), ctx)


def msk_explicit_solution(ctx, paths, u_out, stream=None):
    import torch
    _need(u_out, paths * _dd(ctx), torch.float64, "u_out")
    _check(load_library().msk_explicit_solution(ctx, paths, _ptr(u_out), _stream(stream)), ctx)


def msk_error(ctx, u, u_precision, paths, ref_kind, ref, ref_precision, kappa, err_per_path, err_mean=None,
              stream=None):
    _check(load_library().msk_error(ctx, _ptr(u), u_precision, paths, ref_kind, _ptr(ref), ref_precision, kappa,
                                    _ptr(err_per_path), _ptr(err_mean), _stream(stream)), ctx)


def msk_moments(ctx, u, precision, paths, mom, stream=None):
    _check(load_library().msk_moments(ctx, _ptr(u), precision, paths, _ptr(mom), _stream(stream)), ctx)


def msk_batch_create(items, tune_cache=None):
    """items: sequence of (ctx, order, steps, paths, u_out float tensor, status int32 tensor or None)."""
    arr = (msk_batch_item * len(items))()
    for k, (ctx, order, steps, paths, out, st) in enumerate(items):
        arr[k] = msk_batch_item(ctx.value if hasattr(ctx, "value") else ctx, order, steps, paths,
                                _ptr(out), _ptr(st))
    h = _P()
    rc = load_library().msk_batch_create(ctypes.byref(h), arr, len(items),
                                         tune_cache.encode() if tune_cache else None)
    if rc != MSK_OK:
        raise MskError(rc, "batch creation failed")
    return h


def msk_batch_run(b, stream=None):
    rc = load_library().msk_batch_run(b, _stream(stream))
    if rc != MSK_OK:
        raise MskError(rc, load_library().msk_batch_last_error(b).decode())


def msk_batch_tune(b, tune_cache=None, stream=None):
    v = _INT(0)
    ms = (ctypes.c_float * 5)()
    rc = load_library().msk_batch_tune(b, _stream(stream), tune_cache.encode() if tune_cache else None,
                                       ctypes.byref(v), ms)
    if rc != MSK_OK:
        raise MskError(rc, load_library().msk_batch_last_error(b).decode())
    return v.value, list(ms)


def msk_batch_variant(b) -> int:
    return load_library().msk_batch_variant(b)


def msk_batch_set_variant(b, variant):
    rc = load_library().msk_batch_set_variant(b, variant)
    if rc != MSK_OK:
        raise MskError(rc, load_library().msk_batch_last_error(b).decode())


def msk_batch_last_error(b) -> str:
    return load_library().msk_batch_last_error(b).decode()


def msk_batch_destroy(b):
    load_library().msk_batch_destroy(b)


def _scheck(st: int, s):
    if st != MSK_OK:
        raise MskError(st, load_library().msk_surrogate_last_error(s).decode())


def msk_surrogate_create(ctx, steps=16, rank=64, hidden=512, layers=4, train_batch=4096, infer_batch=65536,
                         ref_order=3, ref_steps=8, init_seed=0):
    h = _P()
    cfg = msk_surrogate_config(steps, rank, hidden, layers, train_batch, infer_batch, ref_order, ref_steps, init_seed)
    _check(load_library().msk_surrogate_create(ctypes.byref(h), ctx, ctypes.byref(cfg)), ctx)
    return h


def msk_surrogate_destroy(s):
    load_library().msk_surrogate_destroy(s)


def msk_surrogate_last_error(s) -> str:
    return load_library().msk_surrogate_last_error(s).decode()


def msk_surrogate_num_params(s) -> int:
    return int(load_library().msk_surrogate_num_params(s))


def msk_surrogate_param_layout(s, layers):
    """[(offset of W_l, offset of b_l)] for l = 0..layers (weight layers = hidden layers + 1)."""
    arr = (_I64 * (2 * (layers + 1)))()
    _scheck(load_library().msk_surrogate_param_layout(s, arr), s)
    return [(arr[2 * l], arr[2 * l + 1]) for l in range(layers + 1)]


def msk_surrogate_get_params(s, params, stream=None):
    import torch
    _need(params, msk_surrogate_num_params(s), torch.float32, "params")
    _scheck(load_library().msk_surrogate_get_params(s, _ptr(params), _stream(stream)), s)


def msk_surrogate_set_params(s, params, stream=None):
    import torch
    _need(params, msk_surrogate_num_params(s), torch.float32, "params")
    _scheck(load_library().msk_surrogate_set_params(s, _ptr(params), _stream(stream)), s)


def _bf16_ptr(X):
    import torch
    if X.dtype not in (torch.bfloat16, torch.int16):
        raise ValueError("features must be a bfloat16 (or int16 bit-pattern) tensor")
    return _ptr(X)


def msk_surrogate_features(s, path0, paths, X, stream=None):
    _scheck(load_library().msk_surrogate_features(s, path0, paths, _bf16_ptr(X) if paths else None,
                                                  _stream(stream)), s)


def msk_surrogate_reference(s, path0, paths, U, stream=None):
    import torch
    _need(U, 1, torch.float32, "U")
    _scheck(load_library().msk_surrogate_reference(s, path0, paths, _ptr(U), _stream(stream)), s)


def msk_surrogate_fit_pod(s, S, N, stream=None):
    import torch
    _need(S, 1, torch.float32, "S")
    sv = (_DBL * 80)()
    _scheck(load_library().msk_surrogate_fit_pod(s, _ptr(S), N, sv, _stream(stream)), s)
    return list(sv)


def msk_surrogate_get_pod(s, mean=None, phi=None, stream=None):
    sc = _DBL(0)
    _scheck(load_library().msk_surrogate_get_pod(s, _ptr(mean), _ptr(phi), ctypes.byref(sc), _stream(stream)), s)
    return sc.value


def msk_surrogate_set_pod(s, mean, phi, coef_scale, stream=None):
    _scheck(load_library().msk_surrogate_set_pod(s, _ptr(mean), _ptr(phi), coef_scale, _stream(stream)), s)


def msk_surrogate_project(s, S, N, C, stream=None):
    _scheck(load_library().msk_surrogate_project(s, _ptr(S), N, _ptr(C), _stream(stream)), s)


def msk_surrogate_decode(s, C, N, U, stream=None):
    _scheck(load_library().msk_surrogate_decode(s, _ptr(C), N, _ptr(U), _stream(stream)), s)


def msk_surrogate_forward(s, X, B, C, stream=None):
    _scheck(load_library().msk_surrogate_forward(s, _bf16_ptr(X), B, _ptr(C), _stream(stream)), s)


def msk_surrogate_loss_grads(s, X, C, B, loss=None, grads=None, stream=None):
    _scheck(load_library().msk_surrogate_loss_grads(s, _bf16_ptr(X), _ptr(C), B, _ptr(loss), _ptr(grads),
                                                    _stream(stream)), s)


def msk_surrogate_adam_step(s, lr, stream=None):
    _scheck(load_library().msk_surrogate_adam_step(s, lr, _stream(stream)), s)


def msk_surrogate_train(s, X, C, N, epochs, lr, loss_hist=None, stream=None):
    _scheck(load_library().msk_surrogate_train(s, _bf16_ptr(X), _ptr(C), N, epochs, lr, _ptr(loss_hist),
                                               _stream(stream)), s)


def msk_surrogate_infer(s, path0, paths, U, flags=None, audit_every=0, tol=1e-2, max_fail_frac=0.05,
                        stream=None):
    """Returns the audit report (audited, max error, mean error, failed, whole-batch fallback)."""
    rep = (_DBL * 5)()
    _scheck(load_library().msk_surrogate_infer(s, path0, paths, _ptr(U), _ptr(flags), audit_every, tol,
                                               max_fail_frac, rep, _stream(stream)), s)
    return list(rep)


def msk_surrogate_set_wait_test(s, on):
    """Test hook: the GEMM epilogues wait on a barrier nothing arrives at (bounded), so the
    next msk_surrogate_sync_status raises MSK_ERR_TIMEOUT."""
    _scheck(load_library().msk_surrogate_set_wait_test(s, int(bool(on))), s)


def msk_surrogate_sync_status(s, stream=None):
    """Synchronise the stream; raises MskError (MSK_ERR_TIMEOUT) if a tensor-core pipeline wait ran out."""
    _scheck(load_library().msk_surrogate_sync_status(s, _stream(stream)), s)


# ---- convenience ---------------------------------------------------------------------

class Solver:
    """A context configured from a workload description (see workloads.Workload)."""

    def __init__(self, w, device: int = 0):
        import torch
        self.w = w
        self.device = torch.device("cuda", device)
        self.ctx = msk_create(w.d, w.d, w.ax, w.bx, w.av, w.bv, device)
        msk_set_coefficients(self.ctx, w.drift_sign, w.kind, w.a0, w.a1, w.s0, w.s1)
        msk_set_initial_gaussian(self.ctx, w.u0_mean, w.u0_cov, w.u0_scale)
        msk_set_seed(self.ctx, w.seed, w.path_offset, w.n_fine, w.T)
        if getattr(w, "x_profile", MSK_XPROF_NONE) != MSK_XPROF_NONE:
            msk_set_x_profile(self.ctx, w.x_profile, getattr(w, "x_profile_c", 1.0))

    def close(self):
        if self.ctx:
            msk_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, n, dtype):
        import torch
        return torch.empty(n, dtype=dtype, device=self.device)

    def state(self, paths, precision=MSK_F64):
        return self._empty(paths * self.w.d * self.w.d, _dtype(precision)).view(paths, self.w.d, self.w.d)

    def magnus(self, order, steps, paths=None, precision=MSK_F64, status=False, out=None):
        import torch
        paths = self.w.paths if paths is None else paths
        u = self.state(paths, precision) if out is None else out
        st = torch.zeros(max(paths, 1), dtype=torch.int32, device=self.device) if status else None
        msk_solve_magnus(self.ctx, order, steps, paths, precision, u, st)
        return (u, st) if status else u

    def magnus_host(self, order, steps, paths=None, precision=MSK_F64, status=False, u0=None):
        """The solve with page-locked host results (shape (paths, d, d)); waits for the stream."""
        import torch
        paths = self.w.paths if paths is None else paths
        n = max(paths, 1) * self.w.d * self.w.d
        u = torch.empty(n, dtype=_dtype(precision), pin_memory=True)[: paths * self.w.d ** 2]
        st = torch.zeros(max(paths, 1), dtype=torch.int32, pin_memory=True) if status else None
        msk_solve_magnus_host(self.ctx, order, steps, paths, precision, u0, u, st)
        torch.cuda.current_stream().synchronize()
        u = u.view(paths, self.w.d, self.w.d)
        return (u, st) if status else u

    def magnus_times(self, order, steps, times_cells, paths=None, precision=MSK_F64, status=False):
        """Solutions at the output times (fine-cell units); shape (paths, n_times, d, d)."""
        import torch
        paths = self.w.paths if paths is None else paths
        q = len(times_cells)
        u = self._empty(max(paths, 1) * q * self.w.d * self.w.d, _dtype(precision))[: paths * q * self.w.d ** 2]
        u = u.view(paths, q, self.w.d, self.w.d)
        st = torch.zeros(max(paths * q, 1), dtype=torch.int32, device=self.device) if status else None
        msk_solve_magnus_times(self.ctx, order, steps, paths, precision, times_cells, u, st)
        return (u, st) if status else u

    def euler(self, steps, paths=None, precision=MSK_F64, status=False):
        import torch
        paths = self.w.paths if paths is None else paths
        u = self.state(paths, precision)
        st = torch.zeros(max(paths, 1), dtype=torch.int32, device=self.device) if status else None
        msk_solve_euler(self.ctx, steps, paths, precision, u, st)
        return (u, st) if status else u

    def explicit(self, paths=None):
        paths = self.w.paths if paths is None else paths
        u = self.state(paths, MSK_F64)
        msk_explicit_solution(self.ctx, paths, u)
        return u

    def functionals(self, steps, paths=None, normals=MSK_F64):
        import torch
        paths = self.w.paths if paths is None else paths
        F = self._empty(paths * steps * MSK_NF, torch.float64)
        msk_brownian_functionals_ex(self.ctx, steps, paths, normals, F)
        return F.view(paths, steps, MSK_NF)

    def increments(self, steps, paths=None):
        import torch
        paths = self.w.paths if paths is None else paths
        dW = self._empty(paths * steps, torch.float64)
        msk_brownian_increments(self.ctx, steps, paths, dW)
        return dW.view(paths, steps)

    def weights(self, order, steps, paths=None, precision=MSK_F64):
        """Weights of the functionals the solve of this precision uses (float solves: float normals)."""
        import torch
        paths = self.w.paths if paths is None else paths
        F = self.functionals(steps, paths, normals=precision)
        Wt = self._empty(paths * steps * MSK_NWT, torch.float64)
        msk_omega_weights(self.ctx, order, steps, paths, precision, F, Wt)
        return Wt.view(paths, steps, MSK_NWT)

    def error(self, u, precision, ref=None, ref_precision=MSK_F64, kappa=0):
        import torch
        paths = u.shape[0]
        e = self._empty(max(paths, 1), torch.float64)
        m = self._empty(1, torch.float64)
        kind = MSK_REF_EXPLICIT if ref is None else MSK_REF_BUFFER
        msk_error(self.ctx, u, precision, paths, kind, ref, ref_precision, kappa, e, m)
        return e[:paths], m

    def moments(self, u, precision):
        import torch
        paths = u.shape[0]
        mom = self._empty(max(paths, 1) * 6, torch.float64)
        msk_moments(self.ctx, u, precision, paths, mom)
        return mom[: paths * 6].view(paths, 6)

#!/usr/bin/env python
"""Benchmark: paths/s of the iterated stochastic Magnus solver at a fixed L2 error.

Workload: the time-dependent Langevin SPDE on a 128 x 128 grid over [-6, 6]^2,
a(t) = 1 + 0.5 sin 2 pi t, sigma(t) = 0.5 (1 + 0.3 cos 2 pi t), Gaussian
u0 = N((0.5, 0), diag(0.5, 1)), 4096 Philox paths per GPU, 2^14 fine Brownian
increments on [0, 1], Magnus order 3 with float stencil/Taylor arithmetic and
double-precision functionals, weights, norm bound and (s, m).

Fixed-error protocol: before timing, the number of Magnus steps K is the
cheapest of 8/16/32/64 whose mean relative L2 error (Err, whole grid) against
the double-precision order-3 solution with 1024 steps stays <= 1e-3 on a
subset of paths (that reference path is itself checked against the CPU
oracle by the test suite).

One timed step = one full solve of the batch (Brownian functionals, Magnus
weights and Taylor parameters, iterated Taylor action), inputs resident on the
device.  Prints one JSON line.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import LANGEVIN_TRIG_128  # noqa: E402

ORDER = 3
K_CANDIDATES = (8, 16, 32, 64)
ERR_TARGET = 1e-3
REF_K = 1024
REF_PATHS = 128
COMPARATOR_PATHS = 512
# algorithmic work of one stencil application per grid point: 13 multiply-adds of the
# folded 15-point stencil (the x differences share their coefficient) + the Taylor
# accumulate, 28 flop; the plain 15-nonzero count (15 multiply-adds + accumulate) is 32
FLOPS_PER_POINT = 28
FLOPS_PER_POINT_15 = 32
METRIC = "paths/s to T at fixed L2 err (Magnus FP32/FP64/surrogate vs EM); HBM GB/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=("ours", "reference"))
    p.add_argument("--paths", type=int, default=LANGEVIN_TRIG_128.paths)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-comparators", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=0, help="paths in the CPU-oracle sample (0 = auto)")
    p.add_argument("--workload", default="trig128", choices=("trig128", "batch", "surrogate", "large512",
                                                              "paper_var", "small32", "step_sweep"),
                   help="trig128: the time-dependent 128^2 workload (default); batch: grids 64/128/256 "
                        "in ratio 4:2:1 of 16384 paths in one persistent launch; surrogate: the learned "
                        "surrogate of the 128^2 workload served 65536 paths per step with a 1%% Magnus audit; "
                        "large512: the 512^2 constant-coefficient grids, sigma = 0.25 / 0.5 / 1, 1024 paths, m2")
    p.add_argument("--no-surrogate", action="store_true", help="skip the surrogate summary of the default line")
    p.add_argument("--no-fp64", action="store_true", help="skip the timed double-precision sub-line")
    p.add_argument("--no-other-workloads", action="store_true",
                   help="skip the compact timings of the batch, 512^2 and variable-coefficient configurations")
    p.add_argument("--clock-csv-dir", default=None,
                   help="directory for the clock samples taken during the timed region (default: a temporary one)")
    p.add_argument("--surrogate-profile-case", type=int, default=0, metavar="PATHS",
                   help="serve PATHS paths twice with an untrained surrogate of the 128^2 workload (random "
                        "weights, random orthonormal POD basis; features, network, decode; no audit) -- a "
                        "small case for ncu captures of the surrogate kernels -- and exit")
    p.add_argument("--profile-grid", type=int, default=128, choices=(128, 512, 100, 200, 300),
                   help="grid of --profile-case: 128 (the bench workload, m3, K = 8) or 512 "
                        "(sigma = 0.5, m2, K = 64)")
    p.add_argument("--profile-engine", default="auto", choices=("auto", "resident", "streamed"),
                   help="engine of the --profile-case solves")
    p.add_argument("--profile-precision", default="f32", choices=("f32", "f64"),
                   help="precision of the --profile-case solves")
    p.add_argument("--profile-general", action="store_true",
                   help="with --profile-grid 100 / 200 / 300: the same problem written as general "
                        "coefficients (nine-point B, five-point A stencil fields)")
    p.add_argument("--profile-case", type=int, default=0, metavar="PATHS",
                   help="run two plain solves of the benchmark workload with PATHS paths at K = 8 "
                        "(a small case for ncu captures) and exit")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# ------------------------------------------------------------------ CPU oracle timing

def _oracle_paths(args):
    w, order, K, paths = args
    from oracle import magnus
    from oracle.discretization import LangevinOperators
    ops = LangevinOperators(w)
    for p in paths:
        magnus.solve_path(w, order, K, p, ops)
    return len(paths)


def time_oracle(w, order, K, npaths, cores):
    """Wall-clock paths/s of the oracle on `npaths` paths spread over `cores` processes."""
    chunks = [list(range(c, npaths, cores)) for c in range(cores)]
    chunks = [c for c in chunks if c]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(chunks)) as pool:
        pool.map(_oracle_paths, [(w, order, K, [0])] * len(chunks))      # imports, warm caches
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_paths, [(w, order, K, c) for c in chunks]))
        dt = time.perf_counter() - t0
    return done / dt, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """SM clock, power and clock-event reasons of one GPU, read (never set) every 10 ms
    through NVML in a background thread while the timed region runs; nvidia-smi at
    200 ms where the NVML library cannot be loaded.  The samples are also kept in a
    CSV file among the run's outputs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    csv_dir = None            # --clock-csv-dir; None: a temporary directory

    def __init__(self, index):
        import tempfile
        self.index = index
        self.proc = None
        self.thread = None
        self.rows = []
        out_dir = ClockSampler.csv_dir or tempfile.mkdtemp(prefix="msk_clocks_")
        self.path = os.path.join(out_dir, f"clocks_gpu{index}.csv")

    def _nvml_index(self):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if ids and all(v.isdigit() for v in ids) and self.index < len(ids):
            return int(ids[self.index])
        return self.index

    class _Nvml:
        """The few read-only NVML queries the sampler needs, through ctypes on the
        driver's libnvidia-ml (no Python NVML package required)."""
        SM = 1   # NVML_CLOCK_SM
        # clock-event reason bits: hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
        BITS = [0x8, 0x40, 0x20, 0x4]

        def __init__(self, index):
            import ctypes
            self.c = ctypes
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")
            self.h = ctypes.c_void_p()
            if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
                raise RuntimeError("no NVML handle")
            self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

        def _u(self, fn, *args):
            v = self.c.c_uint()
            if fn(self.h, *args, self.c.byref(v)) != 0:
                raise RuntimeError("NVML query failed")
            return v.value

        def sm_clock(self):
            return self._u(self.lib.nvmlDeviceGetClockInfo, self.c.c_int(self.SM))

        def sm_max_clock(self):
            return self._u(self.lib.nvmlDeviceGetMaxClockInfo, self.c.c_int(self.SM))

        def power_w(self):
            return self._u(self.lib.nvmlDeviceGetPowerUsage) / 1000.0

        def reasons(self):
            v = self.c.c_ulonglong()
            if self.reasons_fn(self.h, self.c.byref(v)) != 0:
                raise RuntimeError("NVML query failed")
            return v.value

    def _nvml_loop(self, nv, stop):
        smax = nv.sm_max_clock()
        while not stop.is_set():
            try:
                sm, rs, pw = nv.sm_clock(), nv.reasons(), nv.power_w()
                self.rows.append((float(sm), float(smax), ["Active" if rs & b else "Not Active" for b in nv.BITS], pw))
            except Exception:
                pass
            stop.wait(0.01)

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        self.rows = []
        try:
            import threading
            nv = self._Nvml(self._nvml_index())
            self.stop_ev = threading.Event()
            self.thread = threading.Thread(target=self._nvml_loop, args=(nv, self.stop_ev), daemon=True)
            self.thread.start()
            return
        except Exception:
            self.thread = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        rows = []
        source = "nvml"
        if self.thread is not None:
            self.stop_ev.set()
            self.thread.join(timeout=5)
            rows = [(r[0], r[1], r[2]) for r in self.rows]
            with open(self.path, "w") as f:
                f.write("sm_mhz,sm_max_mhz,hw_slowdown,hw_thermal_slowdown,sw_thermal_slowdown,sw_power_cap,power_w\n")
                for r in self.rows:
                    f.write(",".join([str(r[0]), str(r[1])] + r[2] + [f"{r[3]:.1f}"]) + "\n")
        elif self.proc is not None:
            source = "nvidia-smi"
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
            for line in open(self.path):
                t = [x.strip() for x in line.split(",")]
                if len(t) < 9:
                    continue
                try:
                    rows.append((float(t[1]), float(t[2]), t[5:9]))
                except ValueError:
                    continue
        if not rows:
            return None
        reasons = sorted({self.NAMES[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "source": source}


# ------------------------------------------------------------------ helpers

def queued(paths):
    """1 if a Magnus solve of `paths` paths launches the path-order kernel (the library
    orders the paths by estimated cost once every SM gets more than two)."""
    import torch
    return 1 if paths > 2 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count else 0


def engine_source_hash():
    h = hashlib.sha256()
    for f in ("engine.cu", "engine_core.cuh", "stencil.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2207_09776_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


_FMA_PEAK = {}


def fma_peak(msk, device, stream, precision):
    """CUDA-core multiply-add throughput measured on this GPU (cached per precision)."""
    if precision not in _FMA_PEAK:
        _FMA_PEAK[precision] = msk.msk_fma_throughput(device, precision, stream)
    return _FMA_PEAK[precision]


def engine_roofline(msk, device, stream, point_apps, ms, kernel, precision=None):
    """ALU roofline of a resident stencil engine: algorithmic flops (point_apps stencil
    applications per launch x 28 flop) over its CUDA-event time, against the measured
    FMA throughput; the unit-count figure and the 15-nonzero count beside it."""
    precision = msk.MSK_F32 if precision is None else precision
    peaks, peak_src = measured_peaks()
    sm_mhz_peak = float(peaks.get("sm_max_mhz", 2032.0))
    lanes = 128 if precision == msk.MSK_F32 else 2
    derived = 148 * lanes * 2 * sm_mhz_peak * 1e6 / 1e12
    measured = fma_peak(msk, device, stream, precision)
    achieved = point_apps * FLOPS_PER_POINT / (ms / 1e3) / 1e12
    traffic, _ = engine_profile() if precision == msk.MSK_F32 and "128" in kernel else (None, None)
    return {"bound": "alu", "achieved": achieved, "peak": measured, "unit": "TFLOP/s",
            "frac": achieved / measured, "traffic": traffic, "kernel": kernel, "engine_ms": ms,
            "flops_per_point": FLOPS_PER_POINT,
            "frac_15_point_count": point_apps * FLOPS_PER_POINT_15 / (ms / 1e3) / 1e12 / measured,
            "peak_derived": derived,
            "peak_note": (f"measured FMA-chain throughput of the CUDA cores (msk_fma_throughput); "
                          f"unit count 148 SMs x {lanes} lanes x 2 x {sm_mhz_peak:.0f} MHz ({peak_src} clock) "
                          f"= {derived:.1f}"),
            "hbm_equivalent": hbm_equivalent(point_apps, ms / 1e3)}


def engine_profile():
    """ncu DRAM traffic of the engine kernel from the committed profile summary,
    valid only if the engine sources are unchanged since it was taken."""
    h = engine_source_hash()
    prof = os.path.join(ROOT, "profiles", "magnus_engine_d128_f32.txt")
    if not os.path.exists(prof):
        return None, h
    vals = {}
    for line in open(prof):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("engine_source_sha256_16") != h:
        return None, h
    try:
        return float(vals["dram_bytes_per_launch_full_workload"]), h
    except (KeyError, ValueError):
        return None, h


def surrogate_source_hash():
    h = hashlib.sha256()
    for f in ("surrogate_kernels.cuh", "umma.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2207_09776_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def surrogate_profile():
    """DRAM bytes per served path of the decode kernel from the committed ncu summary
    (valid while the kernel sources hash to the recorded value)."""
    prof = os.path.join(ROOT, "profiles", "surrogate_kernels_serve16384.txt")
    if not os.path.exists(prof):
        return None
    vals = {}
    for line in open(prof):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("surrogate_source_sha256_16") != surrogate_source_hash():
        return None
    try:
        return float(vals["decode_dram_bytes_per_path"])
    except (KeyError, ValueError):
        return None


def hbm_equivalent(matvec_points, seconds, bytes_per_point=8):
    """The HBM rate a streaming implementation would need to match the resident engine:
    each stencil application reads and writes every grid point once (8 bytes in float),
    against the measured copy bandwidth."""
    peaks, src = measured_peaks()
    gbs = matvec_points * bytes_per_point / seconds / 1e9
    return {"gbs": gbs, "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6400.0)),
            "frac_of_hbm": gbs / float(peaks.get("hbm_gbs", 6400.0)), "peak_source": src,
            "note": "algorithmic bytes (read + write of the state per stencil application); the state "
                    "stays on chip, so these bytes never reach HBM"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# ------------------------------------------------------------------ learned surrogate

SURR_CFG = dict(steps=16, rank=64, hidden=512, layers=4, train_batch=4096, infer_batch=65536)
SURR_TRAIN = 393216          # Magnus solutions the surrogate is trained on
SURR_EPOCHS = 800
SURR_LR = 6e-4               # cosine decay to zero over the epochs
SURR_SERVE = 65536           # paths per serve step
SURR_AUDIT_EVERY = 100       # 1% Magnus audit
SURR_TOL = 1e-2              # per-path relative L2 fallback threshold
SURR_MAX_FAIL = 0.05         # whole-batch fallback above this audited failure rate
SURR_HELDOUT = 8192
MLP_FLOPS_PER_PATH = 2 * (48 * 512 + 3 * 512 * 512 + 512 * 64)


def _events(torch, stream):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# configuration 5: POD basis and training targets from double-precision order-3 Magnus with 16
# steps on about 200k paths (the --workload surrogate run); the default line's quick summary trains
# on float order-3 K = 8 solutions of twice as many paths (the audit's solver)
SURR_TRAIN_FP64 = 196608
SURR_EPOCHS_FP64 = 1600           # the same 76800 Adam steps as the float-target recipe
SURR_TARGET_K_FP64 = 16


def fp64_targets(msk, torch, solver, first, P, K, stream, chunk=16384):
    """Double-precision order-3 Magnus solutions (K steps) of paths first .. first + P - 1 of the
    solver's path range, rounded to float: the training targets of configuration 5."""
    w = solver.w
    n = w.d * w.d
    U = torch.empty(P, n, device="cuda")
    buf = torch.empty(min(chunk, P) * n, dtype=torch.float64, device="cuda")
    try:
        for c0 in range(0, P, chunk):
            m = min(chunk, P - c0)
            msk.msk_set_seed(solver.ctx, w.seed, w.path_offset + first + c0, w.n_fine, w.T)
            msk.msk_solve_magnus(solver.ctx, ORDER, K, m, msk.MSK_F64, buf[: m * n], None, stream)
            U[c0:c0 + m].copy_(buf[: m * n].view(m, n))
    finally:
        msk.msk_set_seed(solver.ctx, w.seed, w.path_offset, w.n_fine, w.T)
    return U


def train_surrogate(msk, torch, solver, K, stream, fp64=False):
    """Untimed setup: reference solutions, POD, features, Adam training; returns (s, info).
    fp64: targets from double-precision order-3 Magnus with 16 steps (configuration 5);
    else float solutions of the audit's solver (order 3, K steps)."""
    w = solver.w
    n = w.d * w.d
    s = msk.msk_surrogate_create(solver.ctx, ref_order=ORDER, ref_steps=K, init_seed=w.seed, **SURR_CFG)
    P = SURR_TRAIN_FP64 if fp64 else SURR_TRAIN
    epochs = SURR_EPOCHS_FP64 if fp64 else SURR_EPOCHS

    def timed(fn):
        a, b = _events(torch, stream)
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), r

    if fp64:
        t_ref, U = timed(lambda: fp64_targets(msk, torch, solver, 0, P, SURR_TARGET_K_FP64, stream))
    else:
        U = torch.empty(P, n, device="cuda")
        t_ref, _ = timed(lambda: msk.msk_surrogate_reference(s, 0, P, U, stream))
    t0 = time.perf_counter()
    sv = msk.msk_surrogate_fit_pod(s, U, P, stream)
    t_pod = time.perf_counter() - t0
    C = torch.empty(P, SURR_CFG["rank"], device="cuda")
    msk.msk_surrogate_project(s, U, P, C, stream)
    X = torch.empty(P, 3 * SURR_CFG["steps"], dtype=torch.bfloat16, device="cuda")
    msk.msk_surrogate_features(s, 0, P, X, stream)
    del U
    torch.cuda.empty_cache()
    nb = P // SURR_CFG["train_batch"]
    hist = torch.empty(epochs * nb, device="cuda")

    def train():
        for e in range(epochs):
            lr = SURR_LR * 0.5 * (1 + math.cos(math.pi * e / epochs)) + 1e-6
            msk.msk_surrogate_train(s, X, C, P, 1, lr, hist[e * nb:], stream)
    t_train, _ = timed(train)
    msk.msk_surrogate_sync_status(s, stream)
    h = hist.view(epochs, nb).mean(1).cpu().numpy()
    steps = epochs * nb
    info = {"train_paths": P, "epochs": epochs, "adam_steps": steps, "batch": SURR_CFG["train_batch"],
            "lr": f"{SURR_LR} cosine",
            "ref": (f"Magnus FP64 order {ORDER}, K={SURR_TARGET_K_FP64}" if fp64 else
                    f"Magnus FP32 order {ORDER}, K={K}"),
            "ref_solve_paths_per_s": P / (t_ref / 1e3), "pod_fit_s": t_pod,
            "pod_rank_resolved": int(sum(1 for v in sv[:SURR_CFG["rank"]] if v > 0)),
            "train_ms_per_step": t_train / steps,
            "train_tflops": 3 * MLP_FLOPS_PER_PATH * SURR_CFG["train_batch"] / (t_train / steps / 1e3) / 1e12,
            "loss_first_epoch": float(h[0]), "loss_last_epoch": float(h[-1])}
    del X, C
    return s, info


def surrogate_accuracy(msk, torch, solver, s, K, stream, fp64=False):
    """Held-out accuracy against the Magnus solution it learned (double K = 16 with fp64,
    else the audit's float solver) and against the double-precision reference of the
    fixed-error protocol; frac_above_tol is the fraction of all (unaudited) paths whose
    error exceeds the audit tolerance."""
    w = solver.w
    n = w.d * w.d
    p0 = SURR_TRAIN_FP64 if fp64 else SURR_TRAIN
    U = torch.empty(SURR_HELDOUT, n, device="cuda")
    msk.msk_surrogate_infer(s, p0, SURR_HELDOUT, U, None, 0, SURR_TOL, SURR_MAX_FAIL, stream)
    if fp64:
        ref = fp64_targets(msk, torch, solver, p0, SURR_HELDOUT, SURR_TARGET_K_FP64, stream)
    else:
        ref = torch.empty(SURR_HELDOUT, n, device="cuda")
        msk.msk_surrogate_reference(s, p0, SURR_HELDOUT, ref, stream)
    e = (torch.linalg.norm(U - ref, dim=1) / torch.linalg.norm(ref, dim=1)).double()
    tag = "magnus_fp64_K16" if fp64 else "magnus_fp32"
    out = {"heldout_paths": SURR_HELDOUT, f"vs_{tag}_mean": float(e.mean()),
           f"vs_{tag}_p95": float(e.quantile(0.95)), f"vs_{tag}_max": float(e.max()),
           "frac_above_tol": float((e > SURR_TOL).double().mean())}
    # Err against FP64 order-3 Magnus with REF_K steps on REF_PATHS held-out paths
    import paper_2207_09776_b300 as _m
    s64 = _m.Solver(w.with_(path_offset=w.path_offset + p0))
    r64 = s64.magnus(ORDER, REF_K, paths=REF_PATHS, precision=_m.MSK_F64)
    _, e_sur = s64.error(U[:REF_PATHS].view(REF_PATHS, w.d, w.d).contiguous(), _m.MSK_F32, ref=r64,
                         ref_precision=_m.MSK_F64)
    u32 = s64.magnus(ORDER, K, paths=REF_PATHS, precision=_m.MSK_F32)
    _, e_mag = s64.error(u32, _m.MSK_F32, ref=r64, ref_precision=_m.MSK_F64)
    out["err_vs_fp64_ref"] = {"surrogate": float(e_sur.cpu()[0]), f"magnus_fp32_K{K}": float(e_mag.cpu()[0]),
                              "paths": REF_PATHS}
    s64.close()
    return out


def surrogate_serve(msk, torch, solver, s, steps, warmup, stream):
    """Timed serve steps (features, network, decode, 1% audit with fallback) and a component breakdown."""
    w = solver.w
    n = w.d * w.d
    P = SURR_SERVE
    U = torch.empty(P, n, device="cuda")
    flags = torch.zeros(P, dtype=torch.int32, device="cuda")
    base = SURR_TRAIN + SURR_HELDOUT
    for i in range(max(warmup, 0)):
        msk.msk_surrogate_infer(s, base, P, U, flags, SURR_AUDIT_EVERY, SURR_TOL, SURR_MAX_FAIL, stream)
    torch.cuda.synchronize()
    reps = []
    a, b = _events(torch, stream)
    a.record(stream)
    for i in range(steps):
        reps.append(msk.msk_surrogate_infer(s, base + i * P, P, U, flags, SURR_AUDIT_EVERY, SURR_TOL,
                                            SURR_MAX_FAIL, stream))
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    # without the audit
    a2, b2 = _events(torch, stream)
    a2.record(stream)
    for i in range(steps):
        msk.msk_surrogate_infer(s, base + i * P, P, U, None, 0, SURR_TOL, SURR_MAX_FAIL, stream)
    b2.record(stream)
    torch.cuda.synchronize()
    ms_noaudit = a2.elapsed_time(b2) / steps
    # component breakdown (same work as one step)
    X = torch.empty(P, 3 * SURR_CFG["steps"], dtype=torch.bfloat16, device="cuda")
    C = torch.empty(P, SURR_CFG["rank"], device="cuda")
    na = (P + SURR_AUDIT_EVERY - 1) // SURR_AUDIT_EVERY
    Ua = torch.empty(na, n, device="cuda")

    def timed(fn, reps=3):
        fn()
        a, b = _events(torch, stream)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    t_feat = timed(lambda: msk.msk_surrogate_features(s, base, P, X, stream))
    t_mlp = timed(lambda: msk.msk_surrogate_forward(s, X, P, C, stream))
    t_dec = timed(lambda: msk.msk_surrogate_decode(s, C, P, U, stream))
    torch.cuda.synchronize()
    msk.msk_work_counter(solver.ctx, reset=True, stream=stream)
    t_aud = timed(lambda: msk.msk_surrogate_reference(s, base, na, Ua, stream))
    aud_matvecs = msk.msk_work_counter(solver.ctx, reset=True, stream=stream) / 4   # warm call + 3 timed
    msk.msk_surrogate_sync_status(s, stream)
    fails = sum(r[3] for r in reps)
    audited = sum(r[0] for r in reps)
    return {"ms": ms, "ms_no_audit": ms_noaudit, "paths_per_s": P / (ms / 1e3),
            "paths_per_s_no_audit": P / (ms_noaudit / 1e3),
            "audit": {"every": SURR_AUDIT_EVERY, "tol": SURR_TOL, "audited": audited, "failed": fails,
                      "whole_batch_fallbacks": sum(r[4] for r in reps),
                      "max_err": max(r[1] for r in reps), "mean_err": sum(r[2] for r in reps) / len(reps)},
            "breakdown_ms": {"features": t_feat, "mlp": t_mlp, "decode": t_dec,
                             "audit_magnus_contiguous": t_aud},
            "decode_gbs": P * n * 4 / (t_dec / 1e3) / 1e9,
            "mlp_tflops": P * MLP_FLOPS_PER_PATH / (t_mlp / 1e3) / 1e12,
            "audit_paths": na, "audit_matvecs": aud_matvecs,
            "audit_tflops": aud_matvecs * n * FLOPS_PER_POINT / (t_aud / 1e3) / 1e12}, U


# ------------------------------------------------------------------ double precision and Euler comparators

def time_fp64(a, msk, torch, solver, ref, P, stream, dev):
    """The plain double-precision Magnus form of the same step (double normals, functionals,
    weights and Taylor action), K by the same fixed-error protocol, timed over the same
    warm-up and step counts as the headline; its roofline is the measured double FMA rate."""
    ctx, w = solver.ctx, solver.w
    K64, sweep64 = None, {}
    for Kc in K_CANDIDATES:
        u = solver.magnus(ORDER, Kc, paths=REF_PATHS, precision=msk.MSK_F64)
        _, em = solver.error(u, msk.MSK_F64, ref=ref, ref_precision=msk.MSK_F64)
        sweep64[f"K{Kc}"] = float(em.cpu()[0])
        if K64 is None and sweep64[f"K{Kc}"] <= ERR_TARGET:
            K64 = Kc
    K64 = K64 or K_CANDIDATES[-1]
    F = torch.empty(P * K64 * msk.MSK_NF, dtype=torch.float64, device=dev)
    Wt = torch.empty(P * K64 * msk.MSK_NWT, dtype=torch.float64, device=dev)
    out = torch.empty(P * w.d * w.d, dtype=torch.float64, device=dev)
    st = torch.zeros(P, dtype=torch.int32, device=dev)
    ev = [_events(torch, stream) for _ in range(a.steps)]

    def step(i=None):
        msk.msk_brownian_functionals_ex(ctx, K64, P, msk.MSK_F64, F, stream)
        msk.msk_omega_weights(ctx, ORDER, K64, P, msk.MSK_F64, F, Wt, stream)
        if i is not None:
            ev[i][0].record(stream)
        msk.msk_magnus_from_weights(ctx, K64, P, msk.MSK_F64, Wt, out, st, stream)
        if i is not None:
            ev[i][1].record(stream)

    for _ in range(max(a.warmup, 0)):
        step()
    torch.cuda.synchronize()
    msk.msk_work_counter(ctx, reset=True, stream=stream)
    t0, t1 = _events(torch, stream)
    t0.record(stream)
    for i in range(a.steps):
        step(i)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / a.steps
    engine_ms = sum(x.elapsed_time(y) for x, y in ev) / a.steps
    pts = msk.msk_work_counter(ctx, reset=True, stream=stream) / a.steps * w.d * w.d
    roof = engine_roofline(msk, torch.cuda.current_device(), stream, pts, engine_ms,
                           "engine_kernel<double,128,2,256> (2-CTA clusters)", precision=msk.MSK_F64)
    return {"value": P / (ms / 1e3), "unit": "paths/s", "ms_per_step": ms, "steps": a.steps,
            "warmup": a.warmup, "K": K64, "err": sweep64[f"K{K64}"], "err_sweep": sweep64,
            "dtype": "f64", "engine_ms": engine_ms, "roofline": roof,
            "path_status_max": int(st.max().item())}


EQ_NFINE = 65536          # fine Brownian cells of the equal-error comparison (Euler needs up to 65536 steps)
EQ_MAGNUS_K = (4, 8, 16)
EQ_EULER_N = (4096, 16384, 32768, 65536)


def equal_error_vs_euler(msk, torch, solver, Pc, stream):
    """Magnus (float, order 3) against Euler-Maruyama (float) at the same fixed error: both on
    the same Philox paths refined to 2^16 fine cells, so that Euler can take up to 65536
    steps; error against the double-precision order-3 Magnus solution with 1024 steps on
    128 paths; each method at the cheapest setting with Err <= 1e-3, timed on the same
    path count.  The context's Brownian grid is restored afterwards."""
    ctx, w = solver.ctx, solver.w
    msk.msk_set_seed(ctx, w.seed, w.path_offset, EQ_NFINE, w.T)
    try:
        ref = solver.magnus(ORDER, REF_K, paths=REF_PATHS, precision=msk.MSK_F64)
        n = ref.shape[0]

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            s0, s1 = _events(torch, stream)
            s0.record(stream)
            r = fn()
            s1.record(stream)
            torch.cuda.synchronize()
            return r, s0.elapsed_time(s1)
        res = {"n_fine": EQ_NFINE, "paths_timed": Pc, "err_paths": n, "target": ERR_TARGET,
               "magnus_fp32": {}, "euler_fp32": {}}
        for Kc in EQ_MAGNUS_K:
            u, ms = timed(lambda: solver.magnus(ORDER, Kc, paths=Pc, precision=msk.MSK_F32))
            _, e = solver.error(u[:n].contiguous(), msk.MSK_F32, ref=ref, ref_precision=msk.MSK_F64)
            res["magnus_fp32"][f"K{Kc}"] = {"paths_per_s": Pc / (ms / 1e3), "err": float(e.cpu()[0])}
        for ne in EQ_EULER_N:
            u, ms = timed(lambda: solver.euler(ne, paths=Pc, precision=msk.MSK_F32))
            _, e = solver.error(u[:n].contiguous(), msk.MSK_F32, ref=ref, ref_precision=msk.MSK_F64)
            res["euler_fp32"][f"N{ne}"] = {"paths_per_s": Pc / (ms / 1e3), "err": float(e.cpu()[0])}

        def cheapest(tab):
            ok = [(v["paths_per_s"], k) for k, v in tab.items() if v["err"] <= ERR_TARGET]
            return max(ok)[1] if ok else None
        km, ke = cheapest(res["magnus_fp32"]), cheapest(res["euler_fp32"])
        res["magnus_choice"], res["euler_choice"] = km, ke
        res["speedup_magnus_over_euler"] = (res["magnus_fp32"][km]["paths_per_s"] /
                                            res["euler_fp32"][ke]["paths_per_s"]) if km and ke else None
        return res
    finally:
        msk.msk_set_seed(ctx, w.seed, w.path_offset, w.n_fine, w.T)


# ------------------------------------------------------------------ our implementation

def run_ours(a):
    import numpy as np
    import torch

    import paper_2207_09776_b300 as msk
    from paper_2207_09776_b300 import build as mbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mbuild.build()
    msk.load_library()

    P = a.paths
    w = LANGEVIN_TRIG_128.with_(paths=P, path_offset=rank * P)
    solver = msk.Solver(w, device=local)
    ctx = solver.ctx
    stream = torch.cuda.current_stream()

    # ---- fixed-error protocol (untimed) -------------------------------------------
    wref = w.with_(paths=REF_PATHS)
    msk.msk_set_seed(ctx, w.seed, w.path_offset, w.n_fine, w.T)
    ref = solver.magnus(ORDER, REF_K, paths=REF_PATHS, precision=msk.MSK_F64)
    sweep = {}
    chosen = None
    for K in K_CANDIDATES:
        u = solver.magnus(ORDER, K, paths=REF_PATHS, precision=msk.MSK_F32)
        _, em = solver.error(u, msk.MSK_F32, ref=ref, ref_precision=msk.MSK_F64)
        sweep[K] = float(em.cpu()[0])
        if chosen is None and sweep[K] <= ERR_TARGET:
            chosen = K
    if chosen is None:
        chosen = K_CANDIDATES[-1]
    K = chosen
    del wref
    # reference-free alternative: the order-2 / order-3 distance (Remark stepSizeControl)
    # on the same paths, same target; reported beside the protocol's choice
    K_sc, d_sc = msk.msk_select_steps(ctx, ERR_TARGET, 4, 64, REF_PATHS, msk.MSK_F32)
    step_control = {"tol": ERR_TARGET, "paths": REF_PATHS, "K_selected": K_sc,
                    "m2_m3_distance": {f"K{4 * 2 ** i}": v for i, v in enumerate(d_sc)},
                    "K_fixed_error_protocol": K}

    # ---- buffers of one step ------------------------------------------------------------
    F = torch.empty(P * K * msk.MSK_NF, dtype=torch.float64, device=dev)
    Wt = torch.empty(P * K * msk.MSK_NWT, dtype=torch.float64, device=dev)
    out = torch.empty(P * w.d * w.d, dtype=torch.float32, device=dev)
    st = torch.zeros(P, dtype=torch.int32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]

    def step(i=None):
        msk.msk_brownian_functionals_ex(ctx, K, P, msk.MSK_F32, F, stream)   # as msk_solve_magnus(F32)
        msk.msk_omega_weights(ctx, ORDER, K, P, msk.MSK_F32, F, Wt, stream)
        if i is not None:
            ev[i][0].record(stream)
        msk.msk_magnus_from_weights(ctx, K, P, msk.MSK_F32, Wt, out, st, stream)
        if i is not None:
            ev[i][1].record(stream)

    for _ in range(max(a.warmup, 0)):
        step()
    torch.cuda.synchronize()
    msk.msk_work_counter(ctx, reset=True, stream=stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(a.steps):
        step(i)
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    engine_ms = sum(s.elapsed_time(e) for s, e in ev) / a.steps
    matvecs = msk.msk_work_counter(ctx, reset=True, stream=stream)
    status_bits = int(st.cpu().numpy().max())

    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())

    ms_per_step = elapsed_ms / a.steps
    value = world * P * a.steps / (elapsed_ms / 1e3)

    # ---- end to end through the public call with host buffers -------------------------
    u0_host = torch.empty(w.d * w.d, dtype=torch.float64).pin_memory()
    import numpy as _np
    xs = w.ax + (w.bx - w.ax) / (w.d + 1) * _np.arange(1, w.d + 1)
    X, V = _np.meshgrid(xs, xs, indexing="xy")
    mx, mv = w.u0_mean
    cxx, cxv, cvv = w.u0_cov
    det = cxx * cvv - cxv * cxv
    q = (cvv * (X - mx) ** 2 - 2 * cxv * (X - mx) * (V - mv) + cxx * (V - mv) ** 2) / det
    u0_host.copy_(torch.from_numpy((_np.exp(-0.5 * q) / (2 * math.pi * math.sqrt(det))).ravel()))
    out_host = torch.empty(P * w.d * w.d, dtype=torch.float32).pin_memory()

    def e2e_step():
        # u0 copied in on the stream; the engine stores every finished path straight into
        # the page-locked out_host, overlapping the 268 MB readback with the solve
        msk.msk_solve_magnus_host(ctx, ORDER, K, P, msk.MSK_F32, u0_host, out_host, None, stream)

    for _ in range(2):
        e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_e2e = max(3, a.steps // 2)
    for _ in range(n_e2e):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / n_e2e
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())

    # ---- the plain double-precision form, timed like the headline -----------------------
    fp64 = None
    if not a.no_fp64:
        fp64 = time_fp64(a, msk, torch, solver, ref, P, stream, dev)

    # ---- comparators (untimed by the main loop; events) --------------------------------
    comparators = {}
    if not a.no_comparators:
        Pc = min(COMPARATOR_PATHS, P)
        refc = ref[: min(Pc, REF_PATHS)]
        def timed(fn):
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            fn()
            torch.cuda.synchronize()
            s0.record(stream)
            r = fn()
            s1.record(stream)
            torch.cuda.synchronize()
            return r, s0.elapsed_time(s1)
        n = refc.shape[0]
        for Kc in K_CANDIDATES:
            u64, ms64 = timed(lambda: solver.magnus(ORDER, Kc, paths=Pc, precision=msk.MSK_F64))
            _, e64 = solver.error(u64[:n].contiguous(), msk.MSK_F64, ref=refc, ref_precision=msk.MSK_F64)
            comparators.setdefault("magnus_fp64", {})[f"K{Kc}"] = {
                "paths_per_s": Pc / (ms64 / 1e3), "err": float(e64.cpu()[0])}
        for ne in (2048, 16384):
            uem, msem = timed(lambda: solver.euler(ne, paths=Pc, precision=msk.MSK_F32))
            _, eem = solver.error(uem[:n].contiguous(), msk.MSK_F32, ref=refc, ref_precision=msk.MSK_F64)
            comparators.setdefault("euler_fp32", {})[f"N{ne}"] = {
                "paths_per_s": Pc / (msem / 1e3), "err": float(eem.cpu()[0])}
        comparators["magnus_fp32_sweep_err"] = {f"K{k}": v for k, v in sweep.items()}
        comparators["equal_error_vs_euler"] = equal_error_vs_euler(msk, torch, solver, Pc, stream)
        comparators["step_control"] = step_control
        for Kc in K_CANDIDATES:   # order 2 on the same paths and reference
            u2, ms2 = timed(lambda: solver.magnus(2, Kc, paths=Pc, precision=msk.MSK_F32))
            _, e2 = solver.error(u2[:n].contiguous(), msk.MSK_F32, ref=refc, ref_precision=msk.MSK_F64)
            comparators.setdefault("magnus_fp32_m2", {})[f"K{Kc}"] = {
                "paths_per_s": Pc / (ms2 / 1e3), "err": float(e2.cpu()[0])}
        # solutions at the midpoint and the end of every sub-interval (2K output times,
        # the parallel-in-time evaluation of Section 3 "Implementation") against the plain solve
        L = w.n_fine // K
        cells = sorted([(2 * i + 1) * L // 2 for i in range(K)] + [(i + 1) * L for i in range(K)])
        ut = torch.empty(Pc * len(cells) * w.d * w.d, dtype=torch.float32, device=dev)
        _, ms_t = timed(lambda: msk.msk_solve_magnus_times(ctx, ORDER, K, Pc, msk.MSK_F32, cells, ut, None,
                                                           stream))
        _, ms_p = timed(lambda: solver.magnus(ORDER, K, paths=Pc, precision=msk.MSK_F32))
        # the same time-dependent workload with the paper's x profile psi = 1 + 1/(1 + x^2)
        # (Eq. coeffsLangevinVar): the thirteen-operator composition engine
        uvar = torch.empty(Pc * w.d * w.d, dtype=torch.float32, device=dev)
        msk.msk_set_x_profile(ctx, msk.MSK_XPROF_RATIONAL, 1.0)
        _, ms_v = timed(lambda: msk.msk_solve_magnus(ctx, ORDER, K, Pc, msk.MSK_F32, uvar, None, stream))
        msk.msk_set_x_profile(ctx, msk.MSK_XPROF_NONE)
        comparators["x_profile_time_dependent"] = {"paths": Pc, "K": K, "paths_per_s": Pc / (ms_v / 1e3),
                                                   "engine": "thirteen-operator composition"}
        comparators["output_times"] = {
            "paths": Pc, "n_times": len(cells), "paths_per_s": Pc / (ms_t / 1e3),
            "solutions_per_s": Pc * len(cells) / (ms_t / 1e3), "ms": ms_t, "plain_solve_ms": ms_p,
            "time_vs_plain_solve": ms_t / ms_p}

    # ---- learned surrogate of the same workload (setup untimed; own timed serve steps) ----------
    if not a.no_surrogate and world == 1:
        try:
            s_sur, tinfo = train_surrogate(msk, torch, solver, K, stream)
            acc = surrogate_accuracy(msk, torch, solver, s_sur, K, stream)
            serve, _ = surrogate_serve(msk, torch, solver, s_sur, max(3, a.steps // 2), 2, stream)
            comparators["surrogate"] = {"serve_paths": SURR_SERVE, **{k: serve[k] for k in (
                "paths_per_s", "paths_per_s_no_audit", "ms", "audit", "breakdown_ms")},
                "accuracy": acc, "training": tinfo}
            msk.msk_surrogate_destroy(s_sur)
        except Exception as exc:   # the Magnus line stands on its own
            comparators["surrogate"] = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- the other configurations, compactly (after every timed region of the headline) -----
    others = None
    if not a.no_other_workloads and world == 1:
        others = other_workloads(msk, torch, local, stream)

    # ---- roofline of the engine kernel ------------------------------------------------------
    roof = engine_roofline(msk, local, stream, matvecs / a.steps * w.d * w.d, engine_ms,
                           "engine_kernel<float,128,1,512>")
    roof["matvecs_per_launch"] = matvecs / a.steps

    # ---- CPU oracle baseline -------------------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cores = host_cores()
        npaths = a.cpu_sample or 32 * cores     # about 15 s of oracle work on 16 cores
        v, secs = time_oracle(w.with_(paths=npaths), ORDER, K, npaths, cores)
        cpu = {"value": v, "unit": "paths/s", "cores": cores, "kind": "oracle",
               "sample": f"{npaths} paths of the same workload (FP64 oracle, order {ORDER}, K={K}), {secs:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "d": w.d, "paths_per_gpu": P, "order": ORDER, "magnus_steps": K,
                   "n_fine": w.n_fine, "err_target": ERR_TARGET, "err_measured": sweep[K],
                   "reference": f"FP64 order-3 Magnus with {REF_K} steps on {REF_PATHS} paths",
                   "precision": "float stencil/Taylor, double functionals/weights/norm/(s,m)",
                   "l2": "output 268 MB/step > 126 MB L2; Brownian paths regenerated in-kernel each step",
                   "parallelism": f"replicas x{world} (path ranges)"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": world * P / (e2e_ms / 1e3), "unit": "paths/s",
                "h2d_bytes_per_step": u0_host.numel() * 8, "d2h_bytes_per_step": out_host.numel() * 4},
        "clocks": clk,
        "gpu_launches": (3 + queued(P)) * a.steps,   # functionals, weights, [path order,] engine
        "path_status_max": status_bits,
        "fp64": fp64,
        "comparators": comparators,
        "other_workloads": others,
    }
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ the other configurations, compactly

def other_workloads(msk, torch, local, stream):
    """The other configurations timed once each after the headline, with the L2 flushed
    before every timed call (event-timed on the launching stream): the uneven batch
    (autotuned layout, three runs), the 512^2 grid at sigma = 0.5 (float order 2, K = 64,
    1024 paths) and the paper's variable-coefficient grids (float order 3 at the paper's
    steps).  The full protocols -- error gates, double precision, Euler references -- are
    --workload batch / large512 / paper_var."""
    from workloads import BATCH_GRIDS, LARGE_512, PAPER_VAR
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}

    def ev_ms(fn, reps=1):
        flush.fill_(1)
        e0, e1 = _events(torch, stream)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # uneven batch: 9362 x 64^2, 4681 x 128^2, 2341 x 256^2, order 3, K = 16
    solvers = [msk.Solver(w, device=local) for w in BATCH_GRIDS]
    outs = [s.state(w.paths, msk.MSK_F32) for s, w in zip(solvers, BATCH_GRIDS)]
    sts = [torch.zeros(w.paths, dtype=torch.int32, device="cuda") for w in BATCH_GRIDS]
    b = msk.msk_batch_create([(s.ctx, 3, 16, w.paths, o, st)
                              for s, w, o, st in zip(solvers, BATCH_GRIDS, outs, sts)])
    variant, tune_ms = msk.msk_batch_tune(b, stream=stream)
    ms = ev_ms(lambda: msk.msk_batch_run(b, stream), reps=3)
    total = sum(w.paths for w in BATCH_GRIDS)
    out["batch_64_128_256"] = {"paths": total, "order": 3, "magnus_steps": 16, "ms": ms,
                               "paths_per_s": total / (ms / 1e3), "variant": variant, "tune_ms": tune_ms,
                               "flagged_paths": int(sum(int((st != 0).sum()) for st in sts))}
    msk.msk_batch_destroy(b)
    for s in solvers:
        s.close()
    # 512^2, sigma = 0.5: float order 2 with K = 64 (the step the error gate picks there)
    w = LARGE_512[1]
    s = msk.Solver(w, device=local)
    u = s.state(w.paths, msk.MSK_F32)
    msk.msk_solve_magnus(s.ctx, 2, 64, w.paths, msk.MSK_F32, u, None, stream)   # warm-up (scratch of both engines)
    ms = ev_ms(lambda: msk.msk_solve_magnus(s.ctx, 2, 64, w.paths, msk.MSK_F32, u, None, stream))
    out["large512_sigma0.5"] = {"paths": w.paths, "order": 2, "magnus_steps": 64, "ms": ms,
                                "paths_per_s": w.paths / (ms / 1e3),
                                "engine": "automatic (split: resident 16-CTA clusters + streamed CTAs on the free SMs)"}
    s.close()
    # the paper's variable-coefficient grids (Section 3.2), float order 3 at the paper's steps
    for w0 in PAPER_VAR:
        d = w0.d
        P, K = VAR_PATHS[d], VAR_STEPS[d]
        s = msk.Solver(w0.with_(paths=P), device=local)
        u = s.state(P, msk.MSK_F32)
        msk.msk_solve_magnus(s.ctx, ORDER, K, 16, msk.MSK_F32, u, None, stream)   # warm-up (16 paths)
        ms = ev_ms(lambda: msk.msk_solve_magnus(s.ctx, ORDER, K, P, msk.MSK_F32, u, None, stream))
        out[f"paper_var_d{d}"] = {"paths": P, "order": ORDER, "magnus_steps": K, "ms": ms,
                                  "paths_per_s": P / (ms / 1e3)}
        s.close()
    return out


# ------------------------------------------------------------------ reference arm (CPU oracle)

def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    K = K_CANDIDATES[0]
    cores = host_cores()
    npaths = a.cpu_sample or 2 * cores
    w = LANGEVIN_TRIG_128.with_(paths=npaths)
    for _ in range(max(a.warmup, 0)):
        time_oracle(w, ORDER, K, min(npaths, cores), cores)
    times = []
    for _ in range(a.steps):
        v, secs = time_oracle(w, ORDER, K, npaths, cores)
        times.append(secs)
    total = sum(times)
    value = npaths * a.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "d": w.d, "order": ORDER, "magnus_steps": K, "n_fine": w.n_fine,
                       "sample_paths_per_step": npaths},
            "cpu_baseline": {"value": value, "unit": "paths/s", "cores": cores, "kind": "oracle",
                             "sample": f"{npaths} paths per step of the same workload"},
            "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(a):
    """Uneven batch: one persistent launch (CUDA graph) over 64^2, 128^2 and 256^2 paths."""
    import torch

    import paper_2207_09776_b300 as msk
    from paper_2207_09776_b300 import build as mbuild
    from workloads import BATCH_GRIDS

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    mbuild.build()
    msk.load_library()
    K, order = 16, 3
    ws = [g.with_(path_offset=rank * g.paths) for g in BATCH_GRIDS]
    solvers = [msk.Solver(w, device=local) for w in ws]
    outs = [s.state(w.paths, msk.MSK_F32) for s, w in zip(solvers, ws)]
    sts = [torch.zeros(w.paths, dtype=torch.int32, device="cuda") for w in ws]
    items = [(s.ctx, order, K, w.paths, o, st) for s, w, o, st in zip(solvers, ws, outs, sts)]
    b = msk.msk_batch_create(items)
    variant, tune_ms = msk.msk_batch_tune(b)
    stream = torch.cuda.current_stream()
    for _ in range(max(a.warmup, 0)):
        msk.msk_batch_run(b, stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for s in solvers:
        msk.msk_work_counter(s.ctx, reset=True, stream=stream)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        msk.msk_batch_run(b, stream)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    matvec_pts = sum(msk.msk_work_counter(s.ctx, stream=stream) * w.d * w.d for s, w in zip(solvers, ws)) / a.steps
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    total = sum(w.paths for w in ws)
    # kernels per batch run: functionals, [power norms,] weights per grid; then each grid's
    # [path order and] engine (per-grid variant) or each grid's path order, the megakernel
    # and, when the smaller grids run as tasks (variants 0 and 2), the task kernel
    pn = sum(1 for s in solvers if msk.msk_power_norms(s.ctx, order, K, stream=stream).shape[0] > 0)
    if variant == 4:
        batch_launches = 2 * len(ws) + pn + sum(1 + queued(w.paths) for w in ws)
    else:
        small = any(w.d < 256 for w in ws)
        batch_launches = 3 * len(ws) + pn + (1 if (any(w.d == 256 for w in ws) or variant & 1) else 0) + \
            (1 if small and not variant & 1 else 0)
    # per-grid launches one after another, for comparison
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for s, w, o in zip(solvers, ws, outs):
        msk.msk_solve_magnus(s.ctx, order, K, w.paths, msk.MSK_F32, o, None, stream)
    t0.record(stream)
    for s, w, o in zip(solvers, ws, outs):
        msk.msk_solve_magnus(s.ctx, order, K, w.paths, msk.MSK_F32, o, None, stream)
    t1.record(stream)
    torch.cuda.synchronize()
    seq_ms = t0.elapsed_time(t1)
    msk.msk_batch_run(b, stream)
    torch.cuda.synchronize()
    errs, flagged = {}, {}
    for s, w, o, st in zip(solvers, ws, outs, sts):
        e, m = s.error(o[:64].contiguous(), msk.MSK_F32)
        errs[f"d{w.d}"] = float(m.cpu()[0])
        flagged[f"d{w.d}"] = int((st[: w.paths] != 0).sum())
    peaks, peak_src = measured_peaks()
    fp32_peak = fma_peak(msk, local, stream, msk.MSK_F32)   # measured
    achieved = matvec_pts * FLOPS_PER_POINT / (ms / 1e3) / 1e12
    line = {"metric": METRIC, "value": world * total / (ms / 1e3), "unit": "paths/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_64_128_256", "grids": [w.d for w in ws],
                       "paths_per_gpu": [w.paths for w in ws], "order": order, "magnus_steps": K,
                       "n_fine": ws[0].n_fine, "variant": variant, "tune_ms": tune_ms,
                       "err_vs_closed_form_64_paths": errs,
                       # order 3 with step 1/16 explodes on a few 256^2 trajectories (flag BLOWUP)
                       "flagged_paths": flagged,
                       "parallelism": f"replicas x{world} (path ranges)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": None, "kernel": "batch_kernel (whole step)"},
            "clocks": clk,
            "gpu_launches": a.steps * batch_launches,
            "comparators": {"per_grid_launches_ms": seq_ms,
                            "per_grid_paths_per_s": total / (seq_ms / 1e3)}}
    msk.msk_batch_destroy(b)
    for s in solvers:
        s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_surrogate(a):
    """The learned surrogate of the 128^2 workload: one step serves SURR_SERVE new paths
    (features, BF16 network, tensor-core decode, 1% Magnus audit with fallback)."""
    import numpy as np
    import torch

    import paper_2207_09776_b300 as msk
    from paper_2207_09776_b300 import build as mbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    mbuild.build()
    msk.load_library()
    w = LANGEVIN_TRIG_128.with_(path_offset=rank * 10 ** 9)
    solver = msk.Solver(w, device=local)
    stream = torch.cuda.current_stream()
    K = K_CANDIDATES[0]
    s, tinfo = train_surrogate(msk, torch, solver, K, stream, fp64=True)
    acc = surrogate_accuracy(msk, torch, solver, s, K, stream, fp64=True)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    serve, U = surrogate_serve(msk, torch, solver, s, a.steps, a.warmup, stream)
    barrier()
    clk = clocks.stop()
    ms = serve["ms"]
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # end to end: the public call, solutions copied to pinned host memory every step
    n = w.d * w.d
    host = torch.empty(SURR_SERVE * n, dtype=torch.float32).pin_memory()
    base = SURR_TRAIN + SURR_HELDOUT
    msk.msk_surrogate_infer(s, base, SURR_SERVE, U, None, SURR_AUDIT_EVERY, SURR_TOL, SURR_MAX_FAIL, stream)
    host.copy_(U.view(-1), non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = _events(torch, stream)
    n_e2e = max(2, a.steps // 3)
    e0.record(stream)
    for i in range(n_e2e):
        msk.msk_surrogate_infer(s, base + i * SURR_SERVE, SURR_SERVE, U, None, SURR_AUDIT_EVERY, SURR_TOL,
                                SURR_MAX_FAIL, stream)
        host.copy_(U.view(-1), non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / n_e2e
    # rooflines of the serve components
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    bf16 = float(peaks.get("bf16_tflops", 1800.0))
    bd = serve["breakdown_ms"]
    fp32_peak = fma_peak(msk, local, stream, msk.MSK_F32)
    dec_bytes = surrogate_profile()
    roofs = {
        "audit_magnus": {"bound": "alu", "achieved": serve["audit_tflops"], "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": serve["audit_tflops"] / fp32_peak, "traffic": None,
                         "kernel": "engine_kernel<float,128,1,512> (audit paths solved alone; time includes "
                                   "their functionals and weights)"},
        "decode": {"bound": "hbm", "achieved": serve["decode_gbs"], "peak": hbm, "unit": "GB/s",
                   "frac": serve["decode_gbs"] / hbm,
                   "traffic": None if dec_bytes is None else dec_bytes * SURR_SERVE,
                   "kernel": "gemm_tc_kernel<256, EPI_ADD_MEAN, 3>",
                   "algorithmic_bytes": SURR_SERVE * n * 4},
        "mlp": {"bound": "tensor", "achieved": serve["mlp_tflops"], "peak": bf16, "unit": "TFLOP/s",
                "frac": serve["mlp_tflops"] / bf16, "traffic": None, "kernel": "gemm_tc_kernel (5 layers)"},
    }
    dominant = "audit_magnus"   # the largest share of a serve step (see breakdown_ms)
    # CPU oracle of the same serve (features, bf16 network, decode) on a bounded sample
    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        cpu = time_surrogate_oracle(msk, torch, solver, s, base, a.cpu_sample or 4096)   # about 10 s
    line = {"metric": METRIC, "value": world * SURR_SERVE / (ms / 1e3), "unit": "paths/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "surrogate_" + w.name, "d": w.d, "serve_paths_per_gpu": SURR_SERVE,
                       "network": "48 -> 4 x 512 GELU -> 64 (bf16 operands, fp32 accumulation)",
                       "features": "dW, int W ds, int s dW per substep, K=16", "pod_rank": SURR_CFG["rank"],
                       "audit": f"1 in {SURR_AUDIT_EVERY} paths re-solved by Magnus FP32 order {ORDER} K={K}; "
                                f"replaced above {SURR_TOL} relative L2; whole batch above {SURR_MAX_FAIL:.0%} failures",
                       "l2": "output 4.3 GB/step > 126 MB L2",
                       "parallelism": f"replicas x{world} (path ranges)"},
            "roofline": roofs[dominant], "roofline_components": roofs, "cpu_baseline": cpu,
            "e2e": {"value": world * SURR_SERVE / (e2e_ms / 1e3), "unit": "paths/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": SURR_SERVE * n * 4},
            "clocks": clk,
            # per step: features, layers + 1 GEMMs, decode GEMM, audit (functionals, weights,
            # [path order,] engine, audit)
            "gpu_launches": a.steps * (1 + (SURR_CFG["layers"] + 1) + 1 + 4
                                       + queued(SURR_SERVE // SURR_AUDIT_EVERY)),
            "serve": serve, "accuracy": acc, "training": tinfo,
            # the audit sees 1 % of the paths: beside its failure rate, the held-out estimate of the
            # fraction of all served (unaudited) paths above the tolerance
            "paths_above_tol": {"audited_failed_frac": serve["audit"]["failed"] / max(1, serve["audit"]["audited"]),
                                "all_paths_heldout_frac": acc["frac_above_tol"], "tol": SURR_TOL}}
    msk.msk_surrogate_destroy(s)
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _oracle_features(args):
    w, K, paths = args
    from oracle import surrogate as osg
    return osg.features(w, K, paths)


def time_surrogate_oracle(msk, torch, solver, s, base, npaths):
    """Paths/s of the CPU oracle serving the trained network: features from the
    oracle's Brownian functionals (spread over the host cores), the bf16-rounded
    MLP and the POD decode in float64."""
    import numpy as np
    from oracle import surrogate as osg
    w = solver.w
    n = w.d * w.d
    layers = SURR_CFG["layers"]
    flat = torch.empty(msk.msk_surrogate_num_params(s), device="cuda")
    msk.msk_surrogate_get_params(s, flat)
    mean = torch.empty(n, device="cuda")
    phi = torch.empty(SURR_CFG["rank"], n, device="cuda")
    scale = msk.msk_surrogate_get_pod(s, mean, phi)
    flat = flat.cpu().numpy()
    dims = [48] + [SURR_CFG["hidden"]] * layers + [SURR_CFG["rank"]]
    params = []
    for l, (ow, ob) in enumerate(msk.msk_surrogate_param_layout(s, layers)):
        params.append((flat[ow:ow + dims[l] * dims[l + 1]].reshape(dims[l + 1], dims[l]).astype(np.float64),
                       flat[ob:ob + dims[l + 1]].astype(np.float64)))
    m = mean.cpu().numpy().astype(np.float64)
    P = phi.cpu().numpy().astype(np.float64)
    wl = w.with_(path_offset=w.path_offset + base)
    cores = host_cores()
    chunks = [list(range(c, npaths, cores)) for c in range(cores)]
    order = np.argsort(np.concatenate(chunks))
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_features, [(wl, 16, [0])] * cores)        # imports, warm caches
        t0 = time.perf_counter()
        X = np.concatenate(pool.map(_oracle_features, [(wl, 16, c) for c in chunks]))[order]
        X = osg.to_bf16(X)
        c, _ = osg.forward(params, X, bf16=True)
        u = m + scale * c @ P
        dt = time.perf_counter() - t0
    assert u.shape == (npaths, n)
    return {"value": npaths / dt, "unit": "paths/s", "cores": cores, "kind": "oracle",
            "sample": f"{npaths} paths of the same serve (oracle features on {cores} processes, bf16 MLP, "
                      f"POD decode), {dt:.1f} s"}


def run_large512(a):
    """512^2 grids (262144 unknowns) on [-8, 8]^2, a = 1, sigma in {0.25, 0.5, 1}: order-2
    float Magnus on 1024 paths each at the cheapest K in {8, 16, 32, 64} whose Err against the
    closed-form solution is <= 1e-3 with no path flagged (non-finite / blow-up) on a 128-path
    subset; sigma = 1 (a = sigma^2, degenerate) is reported at K = 64 without a gate.  Each
    solve is timed on both engines (resident 16-CTA clusters, streamed one CTA per path) and
    on the split of the two (the automatic choice: clusters plus streamed CTAs on the SMs
    they leave free); the step runs the fastest.  The double-precision solution of all 1024 paths (streamed engine)
    gives the float form's relative L2 error per path and its own speed."""
    import torch

    import paper_2207_09776_b300 as msk
    from paper_2207_09776_b300 import build as mbuild
    from workloads import LARGE_512

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    mbuild.build()
    msk.load_library()
    stream = torch.cuda.current_stream()
    order, sub = 2, 128
    peaks, _ = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    fp32_peak = fma_peak(msk, local, stream, msk.MSK_F32)
    fp64_peak = fma_peak(msk, local, stream, msk.MSK_F64)
    per_sigma = {}
    tot = {"ms": 0.0, "paths": 0, "pts": 0.0}
    eng_tot = {m: {"ms": 0.0, "pts": 0.0} for m in ("resident", "streamed", "split")}
    clocks = ClockSampler(local)
    started = False
    reps = max(1, a.steps // 3)
    modes = {"resident": msk.MSK_ENGINE_RESIDENT, "streamed": msk.MSK_ENGINE_STREAMED,
             "split": msk.MSK_ENGINE_SPLIT}

    def timed(s, K, P, prec, out, st):
        msk.msk_work_counter(s.ctx, reset=True, stream=stream)
        e0, e1 = _events(torch, stream)
        e0.record(stream)
        for _ in range(reps):
            msk.msk_solve_magnus(s.ctx, order, K, P, prec, out, st, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, msk.msk_work_counter(s.ctx, reset=True, stream=stream) / reps

    for w0 in LARGE_512:
        w = w0.with_(path_offset=rank * w0.paths)
        s = msk.Solver(w, device=local)
        sweep, chosen = {}, None
        for Kc in K_CANDIDATES:
            u, stv = s.magnus(order, Kc, paths=sub, precision=msk.MSK_F32, status=True)
            e = float(s.error(u, msk.MSK_F32)[1].cpu()[0])
            flagged = int((stv != 0).sum())
            sweep[f"K{Kc}"] = {"err": e, "flagged_paths": flagged}
            if chosen is None and flagged == 0 and e <= 1e-3 and w.s0 < 1.0:
                chosen = Kc
        K = chosen if chosen is not None else K_CANDIDATES[-1]
        P = w.paths
        out = s.state(P, msk.MSK_F32)
        st = torch.zeros(P, dtype=torch.int32, device="cuda")
        while True:   # the whole batch must be free of flagged paths, else the next K
            for _ in range(max(a.warmup, 1)):
                msk.msk_solve_magnus(s.ctx, order, K, P, msk.MSK_F32, out, st, stream)
            torch.cuda.synchronize()
            if not bool((st != 0).any()) or K >= K_CANDIDATES[-1] or w.s0 >= 1.0:
                break
            K = K_CANDIDATES[K_CANDIDATES.index(K) + 1]
        if not started:
            clocks.start()
            started = True
        eng = {}
        for name, mode in modes.items():
            msk.msk_set_engine(s.ctx, mode)
            msk.msk_solve_magnus(s.ctx, order, K, P, msk.MSK_F32, out, st, stream)   # warm (scratch)
            ms, mv = timed(s, K, P, msk.MSK_F32, out, st)
            eng[name] = {"ms": ms, "paths_per_s": P / (ms / 1e3), "matvecs_per_path": mv / P,
                         "tflops": mv * w.d * w.d * FLOPS_PER_POINT / (ms / 1e3) / 1e12,
                         "hbm_equivalent_gbs": mv * w.d * w.d * 8 / (ms / 1e3) / 1e9}
            eng_tot[name]["ms"] += ms
            eng_tot[name]["pts"] += mv * w.d * w.d
        best = min(eng, key=lambda k: eng[k]["ms"])
        msk.msk_set_engine(s.ctx, modes[best])
        msk.msk_solve_magnus(s.ctx, order, K, P, msk.MSK_F32, out, st, stream)
        torch.cuda.synchronize()
        errs, _ = s.error(out, msk.MSK_F32)
        errs = errs.cpu()
        ok = torch.isfinite(errs)
        # double precision (streamed engine) for every path: its speed, and the float error per path
        msk.msk_set_engine(s.ctx, msk.MSK_ENGINE_AUTO)
        out64 = s.state(P, msk.MSK_F64)
        st64 = torch.zeros(P, dtype=torch.int32, device="cuda")
        msk.msk_work_counter(s.ctx, reset=True, stream=stream)
        e0, e1 = _events(torch, stream)
        e0.record(stream)
        msk.msk_solve_magnus(s.ctx, order, K, P, msk.MSK_F64, out64, st64, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        mv64 = msk.msk_work_counter(s.ctx, reset=True, stream=stream)
        okb = ((st == 0) & (st64 == 0)).cpu()
        d32 = (out.double() - out64).reshape(P, -1).norm(dim=1) / out64.reshape(P, -1).norm(dim=1)
        d32 = d32.cpu()[okb]
        per_sigma[f"sigma{w.s0}"] = {
            "K": K, "gated": w.s0 < 1.0 and chosen is not None, "engine": best,
            "paths_per_s": P / (eng[best]["ms"] / 1e3), "ms": eng[best]["ms"],
            "err_vs_closed_form_mean_finite": float(errs[ok].mean()) if bool(ok.any()) else None,
            "flagged_paths": int((st != 0).sum()), "engines": eng,
            "double": {"paths_per_s": P / (ms64 / 1e3), "ms": ms64, "matvecs_per_path": mv64 / P,
                       "tflops": mv64 * w.d * w.d * FLOPS_PER_POINT / (ms64 / 1e3) / 1e12,
                       "frac_of_fp64_fma_peak": mv64 * w.d * w.d * FLOPS_PER_POINT / (ms64 / 1e3) / 1e12 / fp64_peak,
                       "flagged_paths": int((st64 != 0).sum())},
            "float_vs_double_rel_l2": {"paths": int(okb.sum()), "mean": float(d32.mean()) if len(d32) else None,
                                       "max": float(d32.max()) if len(d32) else None},
            f"sweep_{sub}_paths": sweep}
        tot["ms"] += eng[best]["ms"]
        tot["paths"] += P
        tot["pts"] += eng[best]["matvecs_per_path"] * P * w.d * w.d
        s.close()
    clk = clocks.stop()
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([tot["ms"]], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot["ms"] = float(t.item())
    streamed = eng_tot["streamed"]
    st_gbs = streamed["pts"] * 8 / (streamed["ms"] / 1e3) / 1e9
    achieved = tot["pts"] * FLOPS_PER_POINT / (tot["ms"] / 1e3) / 1e12
    line = {"metric": METRIC, "value": world * tot["paths"] / (tot["ms"] / 1e3), "unit": "paths/s", "n_gpus": world,
            "steps": reps, "warmup": max(a.warmup, 1), "ms_per_step": tot["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "langevin_const_d512_sigma_0.25_0.5_1", "d": 512, "paths_per_gpu": tot["paths"],
                       "order": order, "n_fine": LARGE_512[0].n_fine,
                       "step": "one float solve of 1024 paths for each of the three sigma, at each one's K, "
                               "on the fastest engine (resident, streamed or split)",
                       "err_target": "1e-3 vs the closed form, no flagged path (sigma = 1 not gated)",
                       "parallelism": f"replicas x{world} (path ranges)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": None,
                         "kernel": "the fastest engine per sigma (per_sigma.engine)",
                         "peak_note": "measured FMA-chain throughput (msk_fma_throughput)"},
            "streamed_engine": {"bound": "hbm", "achieved": st_gbs, "peak": hbm_peak, "unit": "GB/s",
                                "frac": st_gbs / hbm_peak,
                                "note": "algorithmic bytes: 8 per grid point per stencil application (read + "
                                        "write of the float state); the engine moves 16 bytes per point per "
                                        "sweep of 4 applications, so its DRAM traffic is about half of these",
                                "tflops": streamed["pts"] * FLOPS_PER_POINT / (streamed["ms"] / 1e3) / 1e12,
                                "frac_of_fp32_fma_peak": streamed["pts"] * FLOPS_PER_POINT / (streamed["ms"] / 1e3)
                                / 1e12 / fp32_peak},
            "fp64_fma_peak_tflops": fp64_peak,
            "per_sigma": per_sigma, "clocks": clk, "gpu_launches": 3 * (3 + queued(P)) * reps}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ small grid, one Magnus step (configuration 1)

SMALL_REPS = 200


def run_small32(a):
    """du = (1/2 u_vv + v u_x) dt + 1/2 u_v dW on a 32 x 32 grid over [-5, 5]^2, standard
    Gaussian u0, 100 Philox paths, T = 1: double-precision Magnus orders 1 and 2 with one
    step against Euler-Maruyama with 1000 steps, all against the closed-form solution.
    The target error is Euler's own (Err of Euler 1000); each method is timed on the 100
    paths, SMALL_REPS solves per timed step."""
    import torch

    import paper_2207_09776_b300 as msk
    from paper_2207_09776_b300 import build as mbuild
    from workloads import LANGEVIN_32

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    mbuild.build()
    msk.load_library()
    stream = torch.cuda.current_stream()
    w = LANGEVIN_32.with_(path_offset=rank * LANGEVIN_32.paths)
    s = msk.Solver(w, device=local)
    P = w.paths
    out = s.state(P, msk.MSK_F64)
    st = torch.zeros(P, dtype=torch.int32, device="cuda")
    methods = {"magnus_m1_K1": lambda: msk.msk_solve_magnus(s.ctx, 1, 1, P, msk.MSK_F64, out, st, stream),
               "magnus_m2_K1": lambda: msk.msk_solve_magnus(s.ctx, 2, 1, P, msk.MSK_F64, out, st, stream),
               "euler_N1000": lambda: msk.msk_solve_euler(s.ctx, 1000, P, msk.MSK_F64, out, st, stream)}
    res = {}
    clocks = ClockSampler(local)
    clocks.start()
    for name, fn in methods.items():
        fn()
        torch.cuda.synchronize()
        errs, em = s.error(out, msk.MSK_F64)
        e = float(em.cpu()[0])
        for _ in range(max(a.warmup, 1)):
            fn()
        t0, t1 = _events(torch, stream)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(a.steps * SMALL_REPS):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / (a.steps * SMALL_REPS)
        res[name] = {"err_vs_closed_form": e, "err_max_path": float(errs.max().cpu()),
                     "paths_per_s": P / (ms / 1e3), "ms_per_solve": ms}
    clk = clocks.stop()
    target = res["euler_N1000"]["err_vs_closed_form"]
    for v in res.values():
        v["meets_target"] = v["err_vs_closed_form"] <= target * (1 + 1e-12)
    best = "magnus_m2_K1"
    line = {"metric": METRIC, "value": world * res[best]["paths_per_s"], "unit": "paths/s", "n_gpus": world,
            "steps": a.steps, "warmup": max(a.warmup, 1), "ms_per_step": res[best]["ms_per_solve"] * SMALL_REPS,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "langevin_const_d32", "d": 32, "paths_per_gpu": P, "T": w.T,
                       "n_fine": w.n_fine, "reference": "closed-form solution (Gaussian)",
                       "err_target": "Err of Euler-Maruyama with 1000 steps",
                       "step": f"{SMALL_REPS} solves of the 100 paths",
                       "parallelism": f"replicas x{world} (path ranges)"},
            "methods": res, "err_target": target,
            "speedup_m2_over_euler": res[best]["paths_per_s"] / res["euler_N1000"]["paths_per_s"],
            "note": "order 1 carries no Ito correction (Stratonovich-consistent), so its error does not "
                    "shrink with the step", "clocks": clk, "gpu_launches": 4 * a.steps * SMALL_REPS}
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ step-size experiments (Section 3.1 / 3.2)

# Magnus steps per unit time of the sweeps: the constant-coefficient sweep resolves the
# paper's thresholds (m2: fluctuations above 0.065, explosion near 0.085; m3: above 0.1 and
# 0.33) on a fine Brownian grid divisible by every K; the variable-coefficient sweep keeps
# that workload's 10^5 fine cells (K must divide them; the Euler reference takes 10^4 steps)
SWEEP_K_CONST = (100, 50, 25, 20, 16, 15, 14, 13, 12, 11, 10, 8, 6, 5, 4, 3, 2)
SWEEP_NFINE_CONST = 1_201_200          # lcm of SWEEP_K_CONST
SWEEP_K_VAR = (100, 80, 50, 40, 32, 25, 20, 16, 10, 8, 5, 4, 2)
SWEEP_EULER_REF = 10_000               # Euler step 1e-4 (the reference of Fig. StepTestVar)


def run_step_sweep(a):
    """Fig. StepTest (Section 3.1) and Fig. StepTestVar (Section 3.2): d = 200, 100 paths,
    the paper's constant coefficients (a = 1.1, sigma = 1/sqrt(10), -v d_x, [-4, 4]^2,
    phi = exp(-(x^2 + v^2)/2)) and then the x profile psi = 1 + 1/(1 + x^2); Magnus orders 2
    and 3 over a range of step sizes.  Per step size: time per path, mean relative error on
    the central 1/16 of the grid (kappa = 4, the paper's measure) and on the central quarter
    (kappa = 1), and the number of exploding paths (MSK_PATH_BLOWUP or non-finite).
    References: the closed-form solution (constant coefficients), Euler-Maruyama with step
    1e-4 in double precision (x profile).  Float Taylor arithmetic on the variable-
    coefficient engine (d = 200 is not a multiple of 32; psi = 1 for the constant case)."""
    import torch

    import paper_2207_09776_b300 as msk
    from paper_2207_09776_b300 import build as mbuild
    from workloads import PAPER_CONST, PAPER_VAR

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mbuild.build()
    msk.load_library()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()

    def sweep(s, ref, Ks, P):
        res = {}
        for order in (2, 3):
            rows = {}
            for K in Ks:
                out = s.state(P, msk.MSK_F32)
                st = torch.zeros(P, dtype=torch.int32, device="cuda")
                msk.msk_solve_magnus(s.ctx, order, K, P, msk.MSK_F32, out, st, stream)   # warm
                t0, t1 = _events(torch, stream)
                t0.record(stream)
                msk.msk_solve_magnus(s.ctx, order, K, P, msk.MSK_F32, out, st, stream)
                t1.record(stream)
                torch.cuda.synchronize()
                ms = t0.elapsed_time(t1)
                bad = (st != 0).cpu()
                row = {"dt": 1.0 / K, "ms_per_path": ms / P, "exploded": int(bad.sum())}
                for kappa in (4, 1):
                    e, _ = s.error(out, msk.MSK_F32, ref=ref, ref_precision=msk.MSK_F64, kappa=kappa)
                    e = e.cpu()
                    good = ~bad & torch.isfinite(e)
                    row[f"err_k{kappa}"] = float(e.mean())
                    row[f"err_k{kappa}_unexploded"] = float(e[good].mean()) if bool(good.any()) else None
                rows[f"K{K}"] = row
            res[f"m{order}"] = rows
        return res

    out_line = {}
    # ---- constant coefficients, closed-form reference ---------------------------------
    wc = PAPER_CONST.with_(d=200, n_fine=SWEEP_NFINE_CONST, paths=100)
    sref = msk.Solver(wc, device=local)
    ref_c = sref.explicit()
    s = msk.Solver(wc, device=local)
    msk.msk_set_x_profile(s.ctx, msk.MSK_XPROF_VALUES, psi=[1.0] * wc.d)
    out_line["constant"] = sweep(s, ref_c, SWEEP_K_CONST, wc.paths)
    s.close()
    sref.close()
    # ---- x profile, Euler 1e-4 reference (double) ---------------------------------------
    wv = PAPER_VAR[1].with_(paths=100)
    s = msk.Solver(wv, device=local)
    ref_v = s.euler(SWEEP_EULER_REF, precision=msk.MSK_F64)
    out_line["x_profile"] = sweep(s, ref_v, SWEEP_K_VAR, wv.paths)
    s.close()
    clk = clocks.stop()

    m3 = out_line["constant"]["m3"]["K10"]
    line = {"metric": METRIC, "value": 1e3 / m3["ms_per_path"], "unit": "paths/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": m3["ms_per_path"] * 100, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper_step_sweep_d200", "d": 200, "paths_per_gpu": 100,
                       "value_is": "order 3, step 0.1, constant coefficients",
                       "n_fine_constant": SWEEP_NFINE_CONST, "n_fine_x_profile": PAPER_VAR[1].n_fine,
                       "reference": {"constant": "closed form", "x_profile": "Euler-Maruyama, step 1e-4, double"}},
            "sweeps": out_line, "clocks": clk, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ variable coefficients (Table errorsVar)

VAR_STEPS = {100: 20, 200: 40, 300: 100}       # the paper's Magnus step sizes 0.05, 0.025, 0.01
VAR_PATHS = {100: 4096, 200: 1024, 300: 512}   # paths per timed solve (outputs > 126 MB L2)
VAR_REF_PATHS = 16
VAR_EM_REF = 100_000                           # Euler-Maruyama with step 1e-5 (the paper's reference)
VAR_EM_CMP = 10_000                            # Euler-Maruyama with step 1e-4 (the paper's comparator)
# floating-point operations per grid point and Taylor term of the variable-coefficient
# engine: pass A (a, b at the point and its four neighbours, A0 a, A0 b, B a, B b, p, q)
# 71, pass B (B p + A0 q - mu t, scaled, accumulated) 14; a fused multiply-add counts 2
VAR_FLOPS_PER_POINT = 85
PAPER_VAR_TABLE = {   # Table errorsVar: seconds per simulation on the paper's V100 (MATLAB)
    100: {"M2": 0.13, "M3": 0.24, "EM_1e-4": 4.24, "EM_1e-5": 42.24},
    200: {"M2": 1.66, "M3": 1.83, "EM_1e-4": 21.02, "EM_1e-5": 209.02},
    300: {"M2": 4.28, "M3": 5.0, "EM_1e-4": 58.41, "EM_1e-5": 582.88}}


def _oracle_var_paths(args):
    w, order, K, paths = args
    from oracle import magnus
    from oracle.discretization import LangevinOperators
    ops = LangevinOperators(w)
    for p in paths:
        magnus.solve_path(w, order, K, p, ops)
    return len(paths)


def general_coefficients(w):
    """The paper's variable-coefficient Langevin problem (x profile psi) written as the nine
    general coefficient grids h, f^x, f^v, g^xx, g^xv, g^vv, sigma, sigma^x, sigma^v."""
    import numpy as np
    d = w.d
    xs = w.ax + (w.bx - w.ax) / (d + 1) * np.arange(1, d + 1)
    X, V = np.meshgrid(xs, xs, indexing="xy")
    psi = 1.0 + w.x_profile_c / (1.0 + X * X)
    z = np.zeros_like(X)
    return np.stack([z, w.drift_sign * V, z, z, z, w.a0 * psi, z, z, w.s0 * np.sqrt(psi)])


def run_paper_var(a):
    """The paper's variable-coefficient experiment (Section 3.2, Table errorsVar): d = 100,
    200, 300 on [-4, 4]^2, g^vv = 1.1 (1 + 1/(x^2+1)), sigma^v = 10^-1/2 sqrt(1 + 1/(x^2+1)),
    -v d_x drift, phi = exp(-(x^2+v^2)/2), T = 1, 10^5 fine Brownian cells.  Per grid: the
    double Euler-Maruyama solution with step 1e-5 on 16 paths is the reference; Magnus orders 2
    and 3 at the paper's steps (float and double) and Euler-Maruyama with step 1e-4 report Err
    against it; the timed step is one float order-3 solve of each grid's batch."""
    import torch

    import paper_2207_09776_b300 as msk
    from paper_2207_09776_b300 import build as mbuild
    from workloads import PAPER_VAR

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    mbuild.build()
    msk.load_library()
    stream = torch.cuda.current_stream()
    peaks, peak_src = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    fp32_peak = fma_peak(msk, local, stream, msk.MSK_F32)   # measured
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    reps = max(1, a.steps // 3)
    clocks = ClockSampler(local)
    per_grid, total_ms, total_paths, total_flops, launches = {}, 0.0, 0, 0.0, 0
    e2e_ms, d2h = 0.0, 0
    started = False
    for w0 in PAPER_VAR:
        d, K = w0.d, VAR_STEPS[w0.d]
        P = VAR_PATHS[d]
        w = w0.with_(paths=P, path_offset=rank * P)
        s = msk.Solver(w, device=local)
        R = VAR_REF_PATHS
        # ---- accuracy (untimed): errors on R paths against Euler-Maruyama with step 1e-5
        t0 = time.perf_counter()
        ref = s.euler(VAR_EM_REF, paths=R, precision=msk.MSK_F64)
        torch.cuda.synchronize()
        ref_s = time.perf_counter() - t0
        acc = {}

        def err(u, prec):
            e, m = s.error(u, prec, ref=ref, ref_precision=msk.MSK_F64)
            e1, _ = s.error(u, prec, ref=ref, ref_precision=msk.MSK_F64, kappa=1)
            return {"err": float(m.cpu()[0]), "err_kappa1": float(e1.mean().cpu())}
        for order in (2, 3):
            for prec, nm in ((msk.MSK_F32, "f32"), (msk.MSK_F64, "f64")):
                u, st = s.magnus(order, K, paths=R, precision=prec, status=True)
                acc[f"M{order}_{nm}"] = dict(err(u, prec), flagged_paths=int((st != 0).sum()))
        for n_em, nm in ((VAR_EM_CMP, "EM_1e-4_f64"), (VAR_EM_CMP // 10, "EM_1e-3_f64")):
            u = s.euler(n_em, paths=R, precision=msk.MSK_F64)
            e = err(u, msk.MSK_F64)
            acc[nm] = {k: (v if math.isfinite(v) else None) for k, v in e.items()}
        # ---- timed: float order-3 solves of P paths (L2 flushed between solves)
        out = s.state(P, msk.MSK_F32)
        st = torch.zeros(P, dtype=torch.int32, device="cuda")
        for _ in range(max(a.warmup, 1)):
            msk.msk_solve_magnus(s.ctx, ORDER, K, P, msk.MSK_F32, out, st, stream)
        torch.cuda.synchronize()
        msk.msk_work_counter(s.ctx, reset=True, stream=stream)
        if not started:
            clocks.start()
            started = True
        ms = 0.0
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            msk.msk_solve_magnus(s.ctx, ORDER, K, P, msk.MSK_F32, out, st, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        ms /= reps
        mv = msk.msk_work_counter(s.ctx, reset=True, stream=stream) / reps
        # order 2 and the Euler comparators on the same batch (one solve each)
        extra = {}
        for nm, fn in (("M2_f32", lambda: msk.msk_solve_magnus(s.ctx, 2, K, P, msk.MSK_F32, out, st, stream)),
                       ("EM_1e-4_f32", lambda: msk.msk_solve_euler(s.ctx, VAR_EM_CMP, P, msk.MSK_F32, out, st,
                                                                   stream))):
            flush.fill_(1)
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            extra[nm] = {"paths_per_s": P / (e0.elapsed_time(e1) / 1e3)}
        if d in (100, 200):
            # the same problem through the general-coefficient path (nine-point B, five-point
            # A with per-point coefficients): the cost of generality, and agreement
            coef = general_coefficients(w)
            msk.msk_solve_magnus(s.ctx, ORDER, K, P, msk.MSK_F32, out, st, stream)   # variable engine
            ref_var = out.clone()
            msk.msk_set_general_coefficients(s.ctx, coef)
            msk.msk_solve_magnus(s.ctx, ORDER, K, P, msk.MSK_F32, out, st, stream)   # warm
            flush.fill_(1)
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            msk.msk_solve_magnus(s.ctx, ORDER, K, P, msk.MSK_F32, out, st, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            diff = float(((out - ref_var).norm() / ref_var.norm()).cpu())
            extra["general_coefficients_engine"] = {"paths_per_s": P / (e0.elapsed_time(e1) / 1e3),
                                                    "rel_l2_vs_variable_engine": diff}
            msk.msk_set_general_coefficients(s.ctx, None)
            msk.msk_set_x_profile(s.ctx, w.x_profile, w.x_profile_c)
        # end to end: the same float solve with the solution read back to pinned host memory
        host = torch.empty(P * d * d, dtype=torch.float32, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        msk.msk_solve_magnus(s.ctx, ORDER, K, P, msk.MSK_F32, out, st, stream)
        host.copy_(out.view(-1), non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        d2h += host.numel() * 4
        flops = mv * d * d * VAR_FLOPS_PER_POINT
        per_grid[f"d{d}"] = {
            "paths": P, "K": K, "h": w.T / K, "paths_per_s": P / (ms / 1e3), "ms": ms,
            "s_per_path": ms / 1e3 / P, "matvecs_per_path": mv / P,
            "tflops": flops / (ms / 1e3) / 1e12, "flagged_paths": int((st != 0).sum()),
            "errors_vs_EM_1e-5_on_16_paths": acc, "reference_solve_s": ref_s, "comparators": extra,
            "paper_V100_s_per_simulation": PAPER_VAR_TABLE[d]}
        total_ms += ms
        total_paths += P
        total_flops += flops
        launches += (3 + queued(P)) * reps
        s.close()
    clk = clocks.stop()
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    achieved = total_flops / (total_ms / 1e3) / 1e12
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cores = host_cores()
        w = PAPER_VAR[0].with_(paths=cores)
        chunks = [[c] for c in range(cores)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_var_paths, [(w.with_(n_fine=200), ORDER, 2, [0])] * cores)   # imports
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_var_paths, [(w, ORDER, VAR_STEPS[100], c) for c in chunks]))
            secs = time.perf_counter() - t0
        cpu = {"value": done / secs, "unit": "paths/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} paths of the d = 100 grid (FP64 oracle, order 3, K = 20), {secs:.1f} s"}
    line = {"metric": METRIC, "value": world * total_paths / (total_ms / 1e3), "unit": "paths/s", "n_gpus": world,
            "steps": reps, "warmup": max(a.warmup, 1), "ms_per_step": total_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper_langevin_var_d100_d200_d300", "grids": [100, 200, 300],
                       "paths_per_gpu": total_paths, "order": ORDER, "n_fine": PAPER_VAR[0].n_fine,
                       "step": "one float order-3 solve of each grid's batch at the paper's step size",
                       "reference": "double Euler-Maruyama, step 1e-5, 16 paths per grid",
                       "l2": "L2 flushed (256 MB write) before every timed solve",
                       "parallelism": f"replicas x{world} (path ranges)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": None,
                         "kernel": "var_engine2_kernel<float> (two columns per thread, one cluster barrier per term; d = 100 one CTA per path, d = 200 / 300 clusters of 4 / 9); B and A0 composed",
                         "flops_per_point_per_term": VAR_FLOPS_PER_POINT,
                         "peak_note": f"FP32 FMA peak 148 SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz ({peak_src} clock)"},
            "cpu_baseline": cpu,
            "e2e": {"value": world * total_paths / (e2e_ms / 1e3), "unit": "paths/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": d2h},
            "per_grid": per_grid, "clocks": clk, "gpu_launches": launches}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_surrogate_profile_case(a):
    """Two serves of PATHS paths by a surrogate with random parameters (kernel timing only)."""
    import torch

    import paper_2207_09776_b300 as msk
    from paper_2207_09776_b300 import build as mbuild
    mbuild.build()
    msk.load_library()
    P = a.surrogate_profile_case
    w = LANGEVIN_TRIG_128
    solver = msk.Solver(w)
    cfg = dict(SURR_CFG, infer_batch=P)
    s = msk.msk_surrogate_create(solver.ctx, ref_order=ORDER, ref_steps=K_CANDIDATES[0], init_seed=1, **cfg)
    n, r = w.d * w.d, SURR_CFG["rank"]
    g = torch.Generator(device="cuda").manual_seed(3)
    phi = torch.linalg.qr(torch.randn(n, r, device="cuda", generator=g))[0].T.contiguous()
    mean = torch.randn(n, device="cuda", generator=g) * 1e-3
    msk.msk_surrogate_set_pod(s, mean, phi, 1e-2)
    U = torch.empty(P, n, device="cuda")
    for _ in range(2):
        msk.msk_surrogate_infer(s, 0, P, U)
    msk.msk_surrogate_sync_status(s)
    print(json.dumps({"surrogate_profile_case": P, "finite": bool(torch.isfinite(U).all())}))
    msk.msk_surrogate_destroy(s)
    solver.close()


def run_profile_case(a):
    """Two solves (functionals, weights, engine) of the workload on a small path count."""
    import torch

    import paper_2207_09776_b300 as msk
    from paper_2207_09776_b300 import build as mbuild
    mbuild.build()
    msk.load_library()
    P = a.profile_case
    if a.profile_grid == 512:
        from workloads import LARGE_512
        w, K, order = LARGE_512[1].with_(paths=P), 64, 2
    elif a.profile_grid in VAR_STEPS:
        from workloads import PAPER_VAR
        w = PAPER_VAR[(100, 200, 300).index(a.profile_grid)].with_(paths=P)
        K, order = VAR_STEPS[a.profile_grid], ORDER
    else:
        w, K, order = LANGEVIN_TRIG_128.with_(paths=P), K_CANDIDATES[0], ORDER
    s = msk.Solver(w)
    if a.profile_general and a.profile_grid in VAR_STEPS:
        msk.msk_set_general_coefficients(s.ctx, general_coefficients(w))
    msk.msk_set_engine(s.ctx, {"auto": msk.MSK_ENGINE_AUTO, "resident": msk.MSK_ENGINE_RESIDENT,
                               "streamed": msk.MSK_ENGINE_STREAMED}[a.profile_engine])
    prec = msk.MSK_F32 if a.profile_precision == "f32" else msk.MSK_F64
    F = torch.empty(P * K * msk.MSK_NF, dtype=torch.float64, device="cuda")
    Wt = torch.empty(P * K * msk.MSK_NWT, dtype=torch.float64, device="cuda")
    out = torch.empty(P * w.d * w.d, dtype=torch.float32 if prec == msk.MSK_F32 else torch.float64, device="cuda")
    for _ in range(2):
        msk.msk_brownian_functionals_ex(s.ctx, K, P, prec, F)
        msk.msk_omega_weights(s.ctx, order, K, P, prec, F, Wt)
        msk.msk_magnus_from_weights(s.ctx, K, P, prec, Wt, out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": P, "matvecs": msk.msk_work_counter(s.ctx)}))
    s.close()


def main():
    a = parse()
    ClockSampler.csv_dir = a.clock_csv_dir
    if a.profile_case:
        run_profile_case(a)
        return
    if a.surrogate_profile_case:
        run_surrogate_profile_case(a)
        return
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "surrogate":
        run_surrogate(a)
    elif a.workload == "large512":
        run_large512(a)
    elif a.workload == "paper_var":
        run_paper_var(a)
    elif a.workload == "small32":
        run_small32(a)
    elif a.workload == "step_sweep":
        run_step_sweep(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()

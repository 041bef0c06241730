// Per-grid launches of the stencil engine (engine_core.cuh): a persistent grid
// of clusters, each solving paths cid, cid + ncl, ... of one context.
#include "engine_core.cuh"

extern const double kMskScaleCap;

namespace {

// The dynamic-queue kernels keep the next path index in 16 bytes past the slab.
__host__ __device__ constexpr size_t queue_slot_offset(size_t slab) { return (slab + 15) / 16 * 16; }

template <typename T, int D, int C, int NT, bool EULER, bool QUEUE>
__global__ void __launch_bounds__(NT, 1) engine_kernel(const EngineArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x;
  int rank = 0;
  if constexpr (C > 1) rank = (int)cg::this_cluster().block_rank();
  const int64_t cid = blockIdx.x / C, ncl = gridDim.x / C;
  // Every cluster of a launch is resident at once (the grid is sized to one wave): a
  // kernel launched as this one's programmatic dependent (the streamed share of a
  // split solve) may start on the SMs that the clusters leave free.  Without such
  // a dependent this has no effect.
  if constexpr (C > 1) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if constexpr (C > 1 && QUEUE) {
    // dynamic assignment on a cluster: rank 0 takes the queue position and publishes
    // the path in its slot; every CTA reads it through the cluster, and a second
    // cluster barrier keeps rank 0 from rewriting the slot or exiting while another
    // CTA still reads it (a CTA's shared memory must not be accessed after it exits)
    const ClusterSync sync;
    slab_init<T, D, C, NT>(sm, tid, rank, sync);
    volatile long long* slot = reinterpret_cast<long long*>(smem_raw + queue_slot_offset(Cfg<T, D, C, NT>::SMEM));
    const uint32_t slot0 = dsmem_addr(const_cast<long long*>(slot), 0);
    for (;;) {
      if (rank == 0 && tid == 0) {
        const unsigned long long q = atomicAdd(a.queue, 1ull);
        *slot = q < (unsigned long long)(a.qlen > 0 ? a.qlen : a.paths) ? a.order[q] : -1;
      }
      sync();
      const long long path = dsmem_ld_s64(slot0);
      sync();
      if (path < 0) break;
      solve_path<T, D, C, NT, EULER>(a, path, sm, tid, rank, sync);
    }
  } else if constexpr (C > 1) {
    const ClusterSync sync;
    slab_init<T, D, C, NT>(sm, tid, rank, sync);
    for (int64_t path = cid; path < a.paths; path += ncl) solve_path<T, D, C, NT, EULER>(a, path, sm, tid, rank, sync);
  } else if constexpr (QUEUE) {
    // dynamic assignment: queue position q -> path order[q]
    const CtaSync sync;
    slab_init<T, D, C, NT>(sm, tid, rank, sync);
    // the next path lives just past the slab (launch_one adds 16 bytes of dynamic shared memory)
    volatile long long* next_path = reinterpret_cast<long long*>(smem_raw + queue_slot_offset(Cfg<T, D, C, NT>::SMEM));
    for (;;) {
      if (tid == 0) {
        const unsigned long long q = atomicAdd(a.queue, 1ull);
        *next_path = q < (unsigned long long)(a.qlen > 0 ? a.qlen : a.paths) ? a.order[q] : -1;
      }
      sync();
      const long long path = *next_path;   // rewritten only after solve_path's closing barrier
      if (path < 0) break;
      solve_path<T, D, C, NT, EULER>(a, path, sm, tid, rank, sync);
    }
  } else {
    const CtaSync sync;
    slab_init<T, D, C, NT>(sm, tid, rank, sync);
    for (int64_t path = cid; path < a.paths; path += ncl) solve_path<T, D, C, NT, EULER>(a, path, sm, tid, rank, sync);
  }
}

// The kernel of one configuration, its dynamic shared memory and attributes, and
// how many of its clusters (CTAs when C = 1) are resident on the device at once.
template <typename T, int D, int C, int NT, bool EULER>
struct Launch {
  using K = Cfg<T, D, C, NT>;
  // the dynamic path queue (Magnus solves) needs 16 bytes past the slab
  static constexpr bool kQ = !EULER && queue_slot_offset(K::SMEM) + 16 <= 232448;
  void (*kern)(const EngineArgs) = nullptr;
  size_t smem = 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  int64_t capacity = 0;

  msk_status prepare(msk_ctx* ctx, bool queued, cudaStream_t stream) {
    queued = queued && kQ;
    kern = queued ? engine_kernel<T, D, C, NT, EULER, kQ> : engine_kernel<T, D, C, NT, EULER, false>;
    smem = queued ? queue_slot_offset(K::SMEM) + 16 : K::SMEM;
    msk_status st = msk_cuda(
        ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "smem attribute");
    if (st != MSK_OK) return st;
    if (C > 8) {
      st = msk_cuda(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1),
                    "cluster attribute");
      if (st != MSK_OK) return st;
    }
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    if (C > 1) {
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cfg.gridDim = dim3(C, 1, 1);
      int nc = 0;
      st = msk_cuda(ctx, cudaOccupancyMaxActiveClusters(&nc, kern, &cfg), "occupancy clusters");
      if (st != MSK_OK) return st;
      if (nc < 1) return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "cluster configuration cannot be scheduled");
      capacity = nc;
    } else {
      int per_sm = 0;
      st = msk_cuda(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem),
                    "occupancy");
      if (st != MSK_OK) return st;
      if (per_sm < 1) return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "kernel does not fit on an SM");
      capacity = (int64_t)per_sm * ctx->num_sms;
    }
    return MSK_OK;
  }
};

template <typename T, int D, int C, int NT, bool EULER>
msk_status launch_one(msk_ctx* ctx, const EngineArgs& a, cudaStream_t stream) {
  Launch<T, D, C, NT, EULER> L;
  msk_status st = L.prepare(ctx, a.queue != nullptr, stream);
  if (st != MSK_OK) return st;
  // one wave: every cluster resident at once (a programmatic dependent relies on it)
  const int64_t clusters = std::min<int64_t>(L.capacity, a.order && a.qlen > 0 ? a.qlen : a.paths);
  L.cfg.gridDim = dim3((unsigned)(clusters * C), 1, 1);
  return msk_cuda(ctx, cudaLaunchKernelEx(&L.cfg, L.kern, a), "engine launch");
}

template <bool EULER>
msk_status dispatch(msk_ctx* ctx, int precision, const EngineArgs& a, cudaStream_t s) {
  const int d = ctx->d;
  if (precision == MSK_F32) {
    switch (d) {
      case 32: return launch_one<float, 32, 1, 32, EULER>(ctx, a, s);
      case 64: return launch_one<float, 64, 1, 128, EULER>(ctx, a, s);
      case 128: return launch_one<float, 128, 1, 512, EULER>(ctx, a, s);
      case 256: return launch_one<float, 256, 4, 256, EULER>(ctx, a, s);
      case 512: return launch_one<float, 512, 16, 256, EULER>(ctx, a, s);
    }
  } else {
    switch (d) {
      case 32: return launch_one<double, 32, 1, 32, EULER>(ctx, a, s);
      case 64: return launch_one<double, 64, 1, 128, EULER>(ctx, a, s);
      case 128: return launch_one<double, 128, 2, 256, EULER>(ctx, a, s);
      case 256: return launch_one<double, 256, 8, 256, EULER>(ctx, a, s);
    }
  }
  return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "grid size / precision combination not built");
}

__global__ void em_table_kernel(CoefDev c, double T, int steps, double* em_d, float* em_f) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= steps) return;
  const double dt = T / steps, tn = n * dt;
  const double al = alpha_t(c, tn) * dt, sg = sigma_t(c, tn);
  em_d[2 * n] = al;
  em_d[2 * n + 1] = sg;
  em_f[2 * n] = (float)al;
  em_f[2 * n + 1] = (float)sg;
}

}  // namespace

// SMs that the queued Magnus form of the resident engine occupies when it fills the
// device (its clusters x C); 0 where the configuration is not built.
static msk_status resident_sms(msk_ctx* ctx, int precision, int64_t* sms) {
  *sms = 0;
  msk_status st = MSK_OK;
  if (precision == MSK_F32 && ctx->d == 512) {
    Launch<float, 512, 16, 256, false> L;
    st = L.prepare(ctx, true, nullptr);
    *sms = L.capacity * 16;
  } else if (precision == MSK_F32 && ctx->d == 256) {
    Launch<float, 256, 4, 256, false> L;
    st = L.prepare(ctx, true, nullptr);
    *sms = L.capacity * 4;
  } else if (precision == MSK_F64 && ctx->d == 256) {
    Launch<double, 256, 8, 256, false> L;
    st = L.prepare(ctx, true, nullptr);
    *sms = L.capacity * 8;
  }
  return st;
}

msk_status launch_em_table(msk_ctx* ctx, int steps, double* em_d, float* em_f, cudaStream_t stream) {
  em_table_kernel<<<(steps + 255) / 256, 256, 0, stream>>>(coef_dev(ctx->coef), ctx->T, steps, em_d, em_f);
  return msk_cuda(ctx, cudaGetLastError(), "euler table");
}

bool resident_engine_available(int d, int precision) {
  if (precision == MSK_F32) return d == 32 || d == 64 || d == 128 || d == 256 || d == 512;
  return d == 32 || d == 64 || d == 128 || d == 256;
}

bool engine_is_streamed(const msk_ctx* ctx, int precision) {
  if (ctx->xprof || ctx->gen) return false;
  if (ctx->engine_mode == MSK_ENGINE_STREAMED) return true;
  if (ctx->engine_mode == MSK_ENGINE_RESIDENT) return false;
  // automatic (and the split mode, or the automatic split in float at 256^2 and 512^2,
  // wherever the solve does not split): the resident engine
  // wherever it holds the grid (at 512^2 in float its 16-CTA clusters of 256 threads
  // measured as fast as streaming or faster, with termination per Taylor term instead
  // of per sweep), the streamed engine where only it does (double at 512^2)
  return !resident_engine_available(ctx->d, precision) && stream_engine_available(ctx->d, precision);
}

// Speed of the streamed engine per SM relative to the resident clusters' per SM, for
// the split (float, 512^2, a = 1, sigma = 0.5, order 2, K = 64: 965 paths/s on 148
// SMs against 1,008 paths/s on the 112 SMs of seven 16-CTA clusters).
static constexpr double kStreamedPerSm = 0.72;

msk_status engine_split(msk_ctx* ctx, int precision, int64_t paths, int64_t* n_s, int64_t* free_sms) {
  *n_s = 0;
  *free_sms = 0;
  if (ctx->xprof || ctx->gen) return MSK_OK;
  const int d = ctx->d;
  const bool both = resident_engine_available(d, precision) && stream_engine_available(d, precision);
  const bool want = ctx->engine_mode == MSK_ENGINE_SPLIT ||
                    (ctx->engine_mode == MSK_ENGINE_AUTO && precision == MSK_F32 && (d == 512 || d == 256));
  if (!both || !want) return MSK_OK;
  int64_t used = 0;
  msk_status st = resident_sms(ctx, precision, &used);
  if (st != MSK_OK) return st;
  const int64_t fr = (int64_t)ctx->num_sms - used;
  if (used < 1 || fr < 1) return MSK_OK;
  // the streamed share by the two engines' throughput on their SMs, in whole paths
  // per streamed CTA (rounded down: its paths are long, so it should finish first)
  const double share = fr * kStreamedPerSm / (fr * kStreamedPerSm + (double)used);
  const int64_t per_cta = (int64_t)((double)paths * share / (double)fr);
  *n_s = std::min<int64_t>(per_cta * fr, paths - 1);
  *free_sms = fr;
  return MSK_OK;
}

msk_status launch_engine_split(msk_ctx* ctx, int steps, int64_t paths, int64_t n_s, int64_t free_sms, int precision,
                               const double* Wt, void* out, uint32_t* status, cudaStream_t stream,
                               long long* order_buf, unsigned long long* queue, unsigned long long* queue2) {
  const int64_t n_r = paths - n_s;
  // the term grids first: growing them frees memory, which would wait for the clusters
  msk_status st = ensure_stream_scratch(ctx, precision, free_sms);
  if (st == MSK_OK) st = launch_path_order(ctx, Wt, steps, n_r, order_buf, queue, stream, 0);
  if (st == MSK_OK) st = launch_path_order(ctx, Wt, steps, n_s, order_buf + n_r, queue2, stream, n_r);
  if (st != MSK_OK) return st;
  // paths 0 .. n_r - 1 on the resident clusters (engine_is_streamed is false here) ...
  EngineSnap x;
  x.order = order_buf;
  x.queue = queue;
  x.qlen = n_r;
  st = launch_engine_ex(ctx, false, steps, paths, precision, Wt, nullptr, out, status, stream, x);
  if (st != MSK_OK) return st;
  // ... and n_r .. paths - 1 on the streamed engine, one CTA per free SM, started
  // while the clusters run
  return launch_engine_stream(ctx, steps, paths, precision, Wt, out, status, stream, order_buf + n_r, queue2, n_s,
                              free_sms, true);
}

msk_status launch_engine(msk_ctx* ctx, bool euler, int steps, int64_t paths, int precision,
                         const double* Wt, const double* dW, void* out, uint32_t* status,
                         cudaStream_t stream) {
  return launch_engine_ex(ctx, euler, steps, paths, precision, Wt, dW, out, status, stream, EngineSnap{});
}

msk_status launch_engine_ex(msk_ctx* ctx, bool euler, int steps, int64_t paths, int precision,
                            const double* Wt, const double* dW, void* out, uint32_t* status,
                            cudaStream_t stream, const EngineSnap& x) {
  if (paths == 0) return MSK_OK;
  if (ctx->xprof || ctx->gen)
    return launch_engine_var(ctx, euler, steps, paths, precision, Wt, dW, out, status, stream, x);
  if (!euler && engine_is_streamed(ctx, precision)) {
    if (x.snap || x.u0_self)
      return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "output times are not built on the streamed engine");
    return launch_engine_stream(ctx, steps, paths, precision, Wt, out, status, stream, x.order, x.queue);
  }
  EngineArgs a{};
  a.snap = x.snap;
  a.snap_first = x.snap_first;
  a.snap_cnt = x.snap_cnt;
  a.n_out = x.n_out;
  a.u0_self = x.u0_self;
  a.em_d = x.em_d;
  a.em_f = x.em_f;
  a.order = x.order;
  a.queue = x.queue;
  a.qlen = x.qlen;
  a.band = ctx->band;
  a.u0 = ctx->u0;
  a.Wt = Wt;
  a.dW = dW;
  a.out = out;
  a.status = status;
  a.work = ctx->work;
  a.paths = paths;
  a.steps = steps;
  a.dx = ctx->dx;
  a.T = ctx->T;
  a.s_cap = kMskScaleCap;
  a.tol32 = 0x1p-20f;   // float Taylor tolerance (see gen_theta.py)
  a.tol64 = 0x1p-53;
  a.c = coef_dev(ctx->coef);
  return euler ? dispatch<true>(ctx, precision, a, stream) : dispatch<false>(ctx, precision, a, stream);
}

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
        *slot = q < (unsigned long long)a.paths ? a.order[q] : -1;
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
        *next_path = q < (unsigned long long)a.paths ? a.order[q] : -1;
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

template <typename T, int D, int C, int NT, bool EULER>
msk_status launch_one(msk_ctx* ctx, const EngineArgs& a, cudaStream_t stream) {
  using K = Cfg<T, D, C, NT>;
  // the dynamic path queue (Magnus solves) needs 16 bytes past the slab
  constexpr bool kQ = !EULER && queue_slot_offset(K::SMEM) + 16 <= 232448;
  const bool queued = kQ && a.queue;
  auto kern = queued ? engine_kernel<T, D, C, NT, EULER, kQ> : engine_kernel<T, D, C, NT, EULER, false>;
  const size_t smem = queued ? queue_slot_offset(K::SMEM) + 16 : K::SMEM;
  msk_status st = msk_cuda(
      ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
      "smem attribute");
  if (st != MSK_OK) return st;
  if (C > 8) {
    st = msk_cuda(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1),
                  "cluster attribute");
    if (st != MSK_OK) return st;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  int64_t clusters = 0;
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
    clusters = nc;
  } else {
    int per_sm = 0;
    st = msk_cuda(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem),
                  "occupancy");
    if (st != MSK_OK) return st;
    if (per_sm < 1) return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "kernel does not fit on an SM");
    clusters = (int64_t)per_sm * ctx->num_sms;
  }
  clusters = std::min<int64_t>(clusters, a.paths);
  cfg.gridDim = dim3((unsigned)(clusters * C), 1, 1);
  return msk_cuda(ctx, cudaLaunchKernelEx(&cfg, kern, a), "engine launch");
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
  // automatic: the resident engine wherever it holds the grid (at 512^2 in float its
  // 16-CTA clusters of 256 threads measured as fast as streaming or faster, with
  // termination per Taylor term instead of per sweep), the streamed engine where only
  // it does (double at 512^2)
  return !resident_engine_available(ctx->d, precision) && stream_engine_available(ctx->d, precision);
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

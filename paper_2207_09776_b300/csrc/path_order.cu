// Longest-processing-time-first path order for the engines' dynamic queue:
// a path's Taylor work is estimated from its step records (the expected number
// of Taylor terms of each step, or s_n m_n where none was estimated), the paths
// are counting-sorted
// by decreasing estimate, and the engine's CTAs take them in that order from an
// atomic counter, so the last paths handed out are the cheapest.
#include "msk_internal.cuh"

namespace {

// Counting sort of the paths by decreasing estimated cost, in one
// block: histogram of the (capped) costs in shared memory, a block-wide
// exclusive scan, then a scatter.  Paths of equal cost keep no particular order
// (the solution of a path does not depend on which CTA solves it).
constexpr int kOrderBuckets = 4096;
constexpr int kOrderThreads = 1024;
constexpr int kOrderCache = 8192;   // paths whose bucket is kept in shared memory between the passes

__device__ __forceinline__ int order_bucket(const double* Wt, int steps, int64_t p) {
  double c = 0.0;
#pragma unroll 4
  for (int n = 0; n < steps; ++n) {
    const double* o = Wt + ((size_t)p * steps + n) * MSK_NWT;
    // expected stencil applications when the weight kernel estimated them, else s m
    c += o[MSK_WT_WORK] > 0.0 ? o[MSK_WT_WORK] : o[MSK_WT_S] * o[MSK_WT_M];
  }
  const int ci = c < (double)(kOrderBuckets - 1) ? (int)c : kOrderBuckets - 1;   // NaN -> cap
  return kOrderBuckets - 1 - ci;   // costliest first
}

// Paths first .. first + paths - 1 (Wt points at path first's records).
__global__ void __launch_bounds__(kOrderThreads) path_order_kernel(const double* Wt, int steps, int64_t paths,
                                                                   int64_t first, long long* order,
                                                                   unsigned long long* queue) {
  __shared__ int cnt[kOrderBuckets];
  __shared__ int wsum[kOrderThreads / 32];
  __shared__ unsigned short cache[kOrderCache];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < kOrderBuckets; i += kOrderThreads) cnt[i] = 0;
  __syncthreads();
  for (int64_t p = tid; p < paths; p += kOrderThreads) {
    const int b = order_bucket(Wt, steps, p);
    if (p < kOrderCache) cache[p] = (unsigned short)b;
    atomicAdd(&cnt[b], 1);
  }
  __syncthreads();
  // exclusive scan: each thread owns kOrderBuckets / kOrderThreads consecutive buckets
  constexpr int PER = kOrderBuckets / kOrderThreads;
  int local[PER], tot = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    local[j] = cnt[tid * PER + j];
    tot += local[j];
  }
  int incl = tot;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = lane < kOrderThreads / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, off);
      if (lane >= off) v += u;
    }
    if (lane < kOrderThreads / 32) wsum[lane] = v;   // inclusive over warps
  }
  __syncthreads();
  int base = incl - tot + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    cnt[tid * PER + j] = base;
    base += local[j];
  }
  __syncthreads();
  for (int64_t p = tid; p < paths; p += kOrderThreads) {
    const int pos = atomicAdd(&cnt[p < kOrderCache ? (int)cache[p] : order_bucket(Wt, steps, p)], 1);
    order[pos] = first + p;
  }
  if (tid == 0) *queue = 0ull;
}

}  // namespace

msk_status launch_path_order(msk_ctx* ctx, const double* Wt, int steps, int64_t paths, long long* order,
                             unsigned long long* queue, cudaStream_t stream, int64_t first) {
  if (first + paths > (int64_t)INT32_MAX) return msk_fail(ctx, MSK_ERR_ARG, "too many paths for the path queue");
  path_order_kernel<<<1, kOrderThreads, 0, stream>>>(Wt + (size_t)first * steps * MSK_NWT, steps, paths, first,
                                                     order, queue);
  return msk_cuda(ctx, cudaGetLastError(), "path order");
}

// Whether p is page-locked host memory mapped into the device: the split solve's
// streamed share keeps its partial sums in the output, which it would then sweep
// over the bus for every group of Taylor terms.
static bool host_memory(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

msk_status launch_magnus_queued(msk_ctx* ctx, int steps, int64_t paths, int precision, const double* Wt, void* out,
                                uint32_t* status, cudaStream_t stream, long long* order_buf,
                                unsigned long long* queue, unsigned long long* queue2) {
  EngineSnap x;
  // the queue pays off once every CTA solves several paths of unequal cost
  if (order_buf && queue && paths > 2 * (int64_t)ctx->num_sms) {
    if (queue2 && out && !host_memory(out)) {
      int64_t n_s = 0, free_sms = 0;
      msk_status st = engine_split(ctx, precision, paths, &n_s, &free_sms);
      if (st != MSK_OK) return st;
      if (n_s > 0)
        return launch_engine_split(ctx, steps, paths, n_s, free_sms, precision, Wt, out, status, stream, order_buf,
                                   queue, queue2);
    }
    msk_status st = launch_path_order(ctx, Wt, steps, paths, order_buf, queue, stream);
    if (st != MSK_OK) return st;
    x.order = order_buf;
    x.queue = queue;
  }
  return launch_engine_ex(ctx, false, steps, paths, precision, Wt, nullptr, out, status, stream, x);
}

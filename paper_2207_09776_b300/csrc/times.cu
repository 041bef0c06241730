// Solutions at several output times (Section 3, "Implementation": within each
// sub-interval of the iterated scheme the Magnus expansion can be evaluated at
// every requested time, all times and trajectories in parallel).
//
// An output time t = T c / n_fine with t_n <= t < t_{n+1}, n = c / L (L =
// n_fine / steps cells), has the solution exp(Y(t_n, t)) U(t_n), with Y(t_n, t)
// the order-`order` logarithm over the cells n L .. c - 1 and U(t_n) the
// iterated solution after n full steps (a time on a sub-interval end is U(t_n)
// itself: an empty interval).  Two engine launches:
//   1. the iterated solve of every path, storing the state at the start of each
//      step that holds output times (and after the last step, for t = T) into
//      those outputs' slots (no final output);
//   2. one partial step per (path, output time): functionals and weights of its
//      interval, and the exponential action started from the slot's snapshot,
//      written over it (empty intervals: zero weights, no Taylor term, the
//      snapshot stays).  All paths x outputs run concurrently.
#include <algorithm>
#include <vector>

#include "msk_internal.cuh"

namespace {

__global__ void or_status_kernel(uint32_t* out, const uint32_t* main_st, int64_t paths, int n_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= paths * n_out) return;
  out[i] |= main_st[i / n_out];
}

}  // namespace

extern "C" msk_status msk_solve_magnus_times(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                                             const int64_t* times_cells, int n_times, void* u_out_dev,
                                             uint32_t* status_dev, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (order < 1 || order > 3) return msk_fail(ctx, MSK_ERR_ARG, "order must be 1, 2 or 3");
  if (precision != MSK_F64 && precision != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  if (steps < 1 || ctx->n_fine % steps != 0)
    return msk_fail(ctx, MSK_ERR_ARG, "steps must be >= 1 and divide n_fine");
  if (paths < 0) return msk_fail(ctx, MSK_ERR_ARG, "paths < 0");
  if (n_times < 1 || !times_cells) return msk_fail(ctx, MSK_ERR_ARG, "need at least one output time");
  for (int q = 0; q < n_times; ++q) {
    if (times_cells[q] < 1 || times_cells[q] > ctx->n_fine)
      return msk_fail(ctx, MSK_ERR_ARG, "output times (in fine cells) must lie in 1 .. n_fine");
    if (q > 0 && times_cells[q] <= times_cells[q - 1])
      return msk_fail(ctx, MSK_ERR_ARG, "output times must be strictly increasing");
  }
  if (paths == 0) return MSK_OK;
  if (!u_out_dev) return msk_fail(ctx, MSK_ERR_ARG, "null output");
  cudaStream_t s = (cudaStream_t)stream;
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;

  const int64_t L = ctx->n_fine / steps;
  const int64_t jobs = paths * n_times;
  const double delta = ctx->T / (double)ctx->n_fine;
  // host tables: step -> its outputs; (path, output) -> interval and (t0, h)
  std::vector<int> first(steps + 1, 0), cnt(steps + 1, 0);
  std::vector<int64_t> step_of(n_times);
  for (int q = 0; q < n_times; ++q) {
    const int64_t n = times_cells[q] / L;   // 0 .. steps
    step_of[q] = n;
    if (cnt[n] == 0) first[n] = q;
    ++cnt[n];
  }
  std::vector<int64_t> jt(3 * jobs);
  std::vector<double> th(2 * jobs);
  for (int64_t p = 0; p < paths; ++p)
    for (int q = 0; q < n_times; ++q) {
      const int64_t j = p * n_times + q, c0 = step_of[q] * L;
      jt[3 * j] = p;
      jt[3 * j + 1] = c0;
      jt[3 * j + 2] = times_cells[q] - c0;
      th[2 * j] = (double)c0 * delta;
      th[2 * j + 1] = (double)(times_cells[q] - c0) * delta;
    }

  // scratch: main functionals + weights, interval functionals + weights, tables, main status
  const size_t nF = (size_t)paths * steps * MSK_NF, nW = (size_t)paths * steps * MSK_NWT;
  const size_t nFj = (size_t)jobs * MSK_NF, nWj = (size_t)jobs * MSK_NWT;
  const size_t doubles = nF + nW + nFj + nWj + 2 * (size_t)jobs + 3 * (size_t)jobs   // jt as int64
                         + (size_t)steps + 1 + ((size_t)paths + 1) / 2 + 4;          // first/cnt, status
  st = msk_ensure_scratch(ctx, doubles * sizeof(double));
  if (st != MSK_OK) return st;
  double* F = reinterpret_cast<double*>(ctx->scratch);
  double* Wt = F + nF;
  double* Fj = Wt + nW;
  double* Wtj = Fj + nFj;
  double* thd = Wtj + nWj;
  int64_t* jtd = reinterpret_cast<int64_t*>(thd + 2 * jobs);
  int* firstd = reinterpret_cast<int*>(jtd + 3 * jobs);
  int* cntd = firstd + steps + 1;
  uint32_t* main_st = reinterpret_cast<uint32_t*>(cntd + steps + 1);
  st = msk_cuda(ctx, cudaMemcpyAsync(thd, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice, s),
                "copy interval times");
  if (st == MSK_OK)
    st = msk_cuda(ctx, cudaMemcpyAsync(jtd, jt.data(), jt.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s),
                  "copy intervals");
  if (st == MSK_OK)
    st = msk_cuda(ctx, cudaMemcpyAsync(firstd, first.data(), (steps + 1) * sizeof(int), cudaMemcpyHostToDevice, s),
                  "copy step table");
  if (st == MSK_OK)
    st = msk_cuda(ctx, cudaMemcpyAsync(cntd, cnt.data(), (steps + 1) * sizeof(int), cudaMemcpyHostToDevice, s),
                  "copy step table");
  if (st != MSK_OK) return st;
  // the pageable copies above are staged before they return; the host tables may go out of scope

  const bool nf32 = precision == MSK_F32;
  // 1. iterated solve, snapshots at the starts of the steps holding output times
  st = launch_brownian(ctx, steps, paths, F, false, s, nf32);
  if (st == MSK_OK) st = launch_omega(ctx, order, steps, paths, precision, F, Wt, s);
  EngineSnap x;
  x.snap = u_out_dev;
  x.snap_first = firstd;
  x.snap_cnt = cntd;
  x.n_out = n_times;
  if (st == MSK_OK)
    st = launch_engine_ex(ctx, false, steps, paths, precision, Wt, nullptr, nullptr, status_dev ? main_st : nullptr,
                          s, x);
  // 2. one partial step per (path, output time), started from its snapshot
  if (st == MSK_OK) st = launch_brownian_jobs(ctx, jtd, jobs, Fj, s, nf32);
  if (st == MSK_OK) st = launch_omega_jobs(ctx, order, jobs, precision, Fj, thd, Wtj, s);
  EngineSnap y;
  y.u0_self = 1;
  if (st == MSK_OK) st = launch_engine_ex(ctx, false, 1, jobs, precision, Wtj, nullptr, u_out_dev, status_dev, s, y);
  if (st == MSK_OK && status_dev) {
    or_status_kernel<<<(unsigned)((jobs + 255) / 256), 256, 0, s>>>(status_dev, main_st, paths, n_times);
    st = msk_cuda(ctx, cudaGetLastError(), "status kernel");
  }
  return st;
}

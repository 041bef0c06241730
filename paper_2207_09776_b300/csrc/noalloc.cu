// msk_solve_magnus_noalloc: the iterated Magnus solve without any device
// allocation inside the call.
//
// msk_solve_magnus keeps the per-(path, step) Brownian functionals and Magnus
// weights in scratch that the library allocates (and grows) with cudaMalloc.
// Some callers cannot let a library do that: their device memory is owned by
// another allocator (a framework's caching allocator, or a fixed memory budget
// shared with other work), or they must not hit cudaMalloc / cudaFree inside a
// latency-bound loop because those calls synchronise the device.  This entry
// point takes its scratch from one file-scope __device__ array instead.
//
// Properties a caller has to know:
//  - The array holds kNoAllocScratchDoubles doubles (16 MiB).  Every GPU that
//    loads this library holds it from the moment the library's device code is
//    loaded there until the process exits.
//  - A request needs paths * steps * (MSK_NF + MSK_NWT) doubles, plus
//    6 * (n_fine + 1) for time-dependent coefficients and MSK_POW_J / 2 per
//    step for the power norms of the Taylor selection (recomputed by every
//    call, a few microseconds); larger requests are rejected with MSK_ERR_ARG
//    before any device work.
//  - The first call on a device looks up the array's device address (set-up,
//    once per device, with that device current); make that first call before
//    any stream capture.
//  - All calls share the array and it keeps the last call's contents; nothing
//    in it needs to start at zero (each call writes every element it reads
//    before reading it, on the caller's stream).  Calls whose work overlaps on
//    the GPU (different streams, or different contexts on the same device)
//    race on the array and must be serialised by the caller.
//  - Inputs live in the context (set up beforehand, which does allocate: also
//    the operator table of the x-profile and general-coefficient engines, which
//    msk_set_x_profile / msk_set_general_coefficients allocate), the outputs
//    are the caller's buffers, as for msk_solve_magnus.
#include <mutex>

#include "msk_internal.cuh"

msk_status launch_cell_table_into(msk_ctx* ctx, double* tab, cudaStream_t stream);
msk_status launch_brownian_with_table(msk_ctx* ctx, int steps, int64_t paths, double* out, const double* tab,
                                      cudaStream_t stream, bool nf32);

namespace {

constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 21;   // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the array on ctx->device (the device must be current).
msk_status scratch_address(msk_ctx* ctx, double** out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return msk_fail(ctx, MSK_ERR_ARG, "device index out of range for the static scratch");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[ctx->device]) {
    void* p = nullptr;
    msk_status st = msk_cuda(ctx, cudaGetSymbolAddress(&p, g_noalloc_scratch), "static scratch address");
    if (st != MSK_OK) return st;
    g_scratch_ptr[ctx->device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[ctx->device];
  return MSK_OK;
}

}  // namespace

extern "C" msk_status msk_solve_magnus_noalloc(msk_ctx* ctx, int order, int steps, int64_t paths,
                                               int precision, void* u_out_dev, uint32_t* path_status_dev,
                                               void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (order < 1 || order > 3) return msk_fail(ctx, MSK_ERR_ARG, "order must be 1, 2 or 3");
  if (precision != MSK_F64 && precision != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  if (steps < 1 || ctx->n_fine % steps != 0)
    return msk_fail(ctx, MSK_ERR_ARG, "steps must be >= 1 and divide n_fine");
  if (paths < 0) return msk_fail(ctx, MSK_ERR_ARG, "paths < 0");
  if (paths == 0) return MSK_OK;
  if (!u_out_dev) return msk_fail(ctx, MSK_ERR_ARG, "null output");
  if (engine_is_streamed(ctx, precision))
    return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "the streamed engine needs library scratch; msk_solve_magnus_noalloc "
                                              "runs the resident engines only");
  const bool trig = ctx->coef.kind == MSK_COEF_TRIG;
  // Bound check by division, so that no product of the caller's sizes can wrap
  // around: the cell table first (n_fine is at most the array size here), then
  // the per-path share (steps <= n_fine, so steps * 28 cannot overflow).
  const size_t per_path = (size_t)steps * (MSK_NF + MSK_NWT);
  const bool table_fits = (uint64_t)ctx->n_fine < kNoAllocScratchDoubles / 6;
  const size_t nT = trig && table_fits ? 6 * (size_t)(ctx->n_fine + 1) : 0;
  // power-norm table of the (s, m) selection: rows <= steps <= n_fine floats x MSK_POW_J
  const size_t nP = ((size_t)power_norm_rows(ctx, steps) * MSK_POW_J + 1) / 2;
  if ((trig && (!table_fits || nT > kNoAllocScratchDoubles)) || nP > kNoAllocScratchDoubles - nT ||
      (uint64_t)paths > (kNoAllocScratchDoubles - nT - nP) / per_path)
    return msk_fail(ctx, MSK_ERR_ARG,
                    "request of " + std::to_string(paths) + " paths x " + std::to_string(steps) +
                    " steps does not fit the static scratch of msk_solve_magnus_noalloc, which holds " +
                    std::to_string(kNoAllocScratchDoubles) + " doubles (paths * steps * " +
                    std::to_string(MSK_NF + MSK_NWT) + " + 6 (n_fine + 1) if time-dependent + " +
                    std::to_string(MSK_POW_J) + " / 2 per step of the Taylor selection)");
  const size_t nF = (size_t)paths * steps * MSK_NF, nW = (size_t)paths * steps * MSK_NWT;
  cudaStream_t s = (cudaStream_t)stream;
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  double* base = nullptr;
  st = scratch_address(ctx, &base);
  if (st != MSK_OK) return st;
  double* F = base;
  double* Wt = F + nF;
  double* tab = Wt + nW;
  float* pow_tab = reinterpret_cast<float*>(tab + nT);
  if (trig) st = launch_cell_table_into(ctx, tab, s);
  if (st == MSK_OK) st = launch_brownian_with_table(ctx, steps, paths, F, tab, s, precision == MSK_F32);
  if (st == MSK_OK) st = launch_power_norms(ctx, order, steps, pow_tab, s);
  if (st == MSK_OK) st = launch_omega_tab(ctx, order, steps, paths, precision, F, Wt, pow_tab, s);
  if (st == MSK_OK) st = launch_engine(ctx, false, steps, paths, precision, Wt, nullptr, u_out_dev, path_status_dev, s);
  return st;
}

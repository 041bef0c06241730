// Context management and the composite entry points of the C ABI.
#include <math.h>

#include <new>

#include "msk_internal.cuh"

// Message of the last failed msk_create on this thread (returned for ctx NULL).
static thread_local std::string t_create_err = "null context";

msk_status msk_fail(msk_ctx* ctx, msk_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

msk_status msk_cuda(msk_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MSK_OK;
  cudaGetLastError();   // clear a sticky launch error of this thread
  return msk_fail(ctx, e == cudaErrorMemoryAllocation ? MSK_ERR_OOM : MSK_ERR_CUDA,
                  std::string(what) + ": " + cudaGetErrorString(e));
}

msk_status msk_ensure_scratch(msk_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return MSK_OK;
  if (ctx->scratch) {
    // cudaFree waits for work that may still use the old buffer
    cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
  }
  const size_t want = bytes + bytes / 4;
  msk_status st = msk_cuda(ctx, cudaMalloc(&ctx->scratch, want), "scratch allocation");
  if (st != MSK_OK) return st;
  ctx->scratch_bytes = want;
  return MSK_OK;
}

bool msk_supported_d(int d) { return d >= 8 && d <= 512; }

static bool is_fin(double x) { return isfinite(x) != 0; }

extern "C" const char* msk_last_error(const msk_ctx* ctx) {
  if (!ctx) return t_create_err.c_str();
  return ctx->err.c_str();
}

extern "C" void msk_destroy(msk_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->u0) cudaFree(ctx->u0);
  if (ctx->band) cudaFree(ctx->band);
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->work) cudaFree(ctx->work);
  if (ctx->tab) cudaFree(ctx->tab);
  if (ctx->psi) cudaFree(ctx->psi);
  if (ctx->var_tab) cudaFree(ctx->var_tab);
  if (ctx->pow_tab) cudaFree(ctx->pow_tab);
  if (ctx->stream_scratch) cudaFree(ctx->stream_scratch);
  if (ctx->gen64) cudaFree(ctx->gen64);
  if (ctx->gen32) cudaFree(ctx->gen32);
  delete ctx;
}

extern "C" msk_status msk_create(msk_ctx** out, const msk_grid* g, int device) {
  if (!out) return MSK_ERR_ARG;
  *out = nullptr;
  if (!g) return MSK_ERR_ARG;
  if (g->nx != g->nv || !msk_supported_d(g->nx)) return MSK_ERR_ARG;
  if (!is_fin(g->ax) || !is_fin(g->bx) || !is_fin(g->av) || !is_fin(g->bv)) return MSK_ERR_NONFINITE;
  if (!(g->bx > g->ax) || !(g->bv > g->av)) return MSK_ERR_ARG;
  msk_ctx* ctx = new (std::nothrow) msk_ctx();
  if (!ctx) return MSK_ERR_OOM;
  ctx->device = device;
  ctx->d = g->nx;
  ctx->ax = g->ax;
  ctx->bx = g->bx;
  ctx->av = g->av;
  ctx->bv = g->bv;
  ctx->dx = (g->bx - g->ax) / (g->nx + 1);
  ctx->dv = (g->bv - g->av) / (g->nv + 1);
  ctx->coef = msk_coeffs{1, MSK_COEF_CONST, 1.0, 0.0, 0.5, 0.0};
  ctx->u0g = msk_gaussian{0.0, 0.0, 1.0, 0.0, 1.0, 1.0};
  msk_status st = msk_cuda(ctx, cudaSetDevice(device), "set device");
  if (st == MSK_OK) st = msk_cuda(ctx, cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device),
                                  "device attribute");
  const size_t dd = (size_t)ctx->d * ctx->d;
  if (st == MSK_OK) st = msk_cuda(ctx, cudaMalloc(&ctx->u0, dd * sizeof(double)), "u0 allocation");
  if (st == MSK_OK)
    st = msk_cuda(ctx, cudaMalloc(&ctx->band, (size_t)MSK_NOPS * ctx->d * MSK_BAND * sizeof(double)),
                  "band allocation");
  if (st == MSK_OK) st = msk_cuda(ctx, cudaMalloc(&ctx->aux, 32 * sizeof(double)), "aux allocation");
  if (st == MSK_OK) st = msk_cuda(ctx, cudaMalloc(&ctx->work, sizeof(unsigned long long)), "counter allocation");
  if (st == MSK_OK) st = msk_cuda(ctx, cudaMemset(ctx->work, 0, sizeof(unsigned long long)), "counter reset");
  if (st == MSK_OK) st = launch_band_tables(ctx, 0);
  if (st == MSK_OK) st = launch_gaussian_u0(ctx, 0);
  if (st != MSK_OK) {
    t_create_err = ctx->err;
    msk_destroy(ctx);
    return st;
  }
  *out = ctx;
  return MSK_OK;
}

extern "C" msk_status msk_set_coefficients(msk_ctx* ctx, const msk_coeffs* c) {
  if (!ctx || !c) return MSK_ERR_ARG;
  if (c->drift_sign != 1 && c->drift_sign != -1) return msk_fail(ctx, MSK_ERR_ARG, "drift_sign must be +-1");
  if (c->kind != MSK_COEF_CONST && c->kind != MSK_COEF_TRIG) return msk_fail(ctx, MSK_ERR_ARG, "bad kind");
  if (!is_fin(c->a0) || !is_fin(c->a1) || !is_fin(c->s0) || !is_fin(c->s1))
    return msk_fail(ctx, MSK_ERR_NONFINITE, "non-finite coefficient");
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  const bool rebuild = c->drift_sign != ctx->coef.drift_sign;
  if (rebuild || c->a0 != ctx->coef.a0 || c->kind != ctx->coef.kind) ctx->var_dirty = true;
  ctx->coef = *c;
  ++ctx->setup_gen;
  if (rebuild) return launch_band_tables(ctx, 0);
  return MSK_OK;
}

extern "C" msk_status msk_set_engine(msk_ctx* ctx, int mode) {
  if (!ctx) return MSK_ERR_ARG;
  if (mode != MSK_ENGINE_AUTO && mode != MSK_ENGINE_RESIDENT && mode != MSK_ENGINE_STREAMED &&
      mode != MSK_ENGINE_SPLIT)
    return msk_fail(ctx, MSK_ERR_ARG, "bad engine mode");
  ctx->engine_mode = mode;
  return MSK_OK;
}

extern "C" msk_status msk_set_initial_gaussian(msk_ctx* ctx, const msk_gaussian* g) {
  if (!ctx || !g) return MSK_ERR_ARG;
  const double v[6] = {g->mean_x, g->mean_v, g->cov_xx, g->cov_xv, g->cov_vv, g->scale};
  for (double x : v)
    if (!is_fin(x)) return msk_fail(ctx, MSK_ERR_NONFINITE, "non-finite initial datum");
  if (!(g->cov_xx > 0) || !(g->cov_vv > 0) || !(g->cov_xx * g->cov_vv - g->cov_xv * g->cov_xv > 0))
    return msk_fail(ctx, MSK_ERR_ARG, "covariance must be positive definite");
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  ctx->u0g = *g;
  return launch_gaussian_u0(ctx, 0);
}

extern "C" msk_status msk_set_initial(msk_ctx* ctx, const double* u0_dev, void* stream) {
  if (!ctx || !u0_dev) return MSK_ERR_ARG;
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  const size_t dd = (size_t)ctx->d * ctx->d;
  return msk_cuda(ctx, cudaMemcpyAsync(ctx->u0, u0_dev, dd * sizeof(double), cudaMemcpyDeviceToDevice,
                                       (cudaStream_t)stream), "copy u0");
}

extern "C" msk_status msk_set_seed(msk_ctx* ctx, uint64_t seed, uint64_t path_offset, int64_t n_fine, double T) {
  if (!ctx) return MSK_ERR_ARG;
  if (n_fine < 1 || n_fine > ((int64_t)1 << 32)) return msk_fail(ctx, MSK_ERR_ARG, "n_fine out of range");
  if (!is_fin(T)) return msk_fail(ctx, MSK_ERR_NONFINITE, "non-finite T");
  if (!(T > 0)) return msk_fail(ctx, MSK_ERR_ARG, "T must be positive");
  ctx->seed = seed;
  ctx->path_offset = path_offset;
  ctx->n_fine = n_fine;
  ctx->T = T;
  ++ctx->setup_gen;
  return MSK_OK;
}

static msk_status check_steps(msk_ctx* ctx, int steps, int64_t paths) {
  if (steps < 1 || ctx->n_fine % steps != 0) return msk_fail(ctx, MSK_ERR_ARG, "steps must be >= 1 and divide n_fine");
  if (paths < 0) return msk_fail(ctx, MSK_ERR_ARG, "paths < 0");
  return MSK_OK;
}

extern "C" msk_status msk_brownian_functionals(msk_ctx* ctx, int steps, int64_t paths, double* F_dev, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  msk_status st = check_steps(ctx, steps, paths);
  if (st != MSK_OK) return st;
  if (paths == 0) return MSK_OK;
  if (!F_dev) return msk_fail(ctx, MSK_ERR_ARG, "null buffer");
  st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  return launch_brownian(ctx, steps, paths, F_dev, false, (cudaStream_t)stream);
}

extern "C" msk_status msk_brownian_functionals_ex(msk_ctx* ctx, int steps, int64_t paths, int normals, double* F_dev,
                                                 void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (normals != MSK_F64 && normals != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "normals must be MSK_F64 or MSK_F32");
  msk_status st = check_steps(ctx, steps, paths);
  if (st != MSK_OK) return st;
  if (paths == 0) return MSK_OK;
  if (!F_dev) return msk_fail(ctx, MSK_ERR_ARG, "null buffer");
  st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  return launch_brownian(ctx, steps, paths, F_dev, false, (cudaStream_t)stream, normals == MSK_F32);
}

extern "C" msk_status msk_brownian_increments(msk_ctx* ctx, int steps, int64_t paths, double* dW_dev, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  msk_status st = check_steps(ctx, steps, paths);
  if (st != MSK_OK) return st;
  if (paths == 0) return MSK_OK;
  if (!dW_dev) return msk_fail(ctx, MSK_ERR_ARG, "null buffer");
  st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  return launch_brownian(ctx, steps, paths, dW_dev, true, (cudaStream_t)stream);
}

// out_on_host: u_out_dev is the device address of mapped host memory, which the split
// solve's streamed share would sweep over the bus for every group of Taylor terms; those
// solves keep every path on the resident engine.
static msk_status solve_magnus(msk_ctx* ctx, int order, int steps, int64_t paths, int precision, void* u_out_dev,
                               uint32_t* path_status_dev, void* stream, bool out_on_host) {
  if (!ctx) return MSK_ERR_ARG;
  if (order < 1 || order > 3) return msk_fail(ctx, MSK_ERR_ARG, "order must be 1, 2 or 3");
  if (precision != MSK_F64 && precision != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  msk_status st = check_steps(ctx, steps, paths);
  if (st != MSK_OK) return st;
  if (paths == 0) return MSK_OK;
  if (!u_out_dev) return msk_fail(ctx, MSK_ERR_ARG, "null output");
  cudaStream_t s = (cudaStream_t)stream;
  st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  // scratch: functionals, weights, then the path order and two queue counters of the engine
  const size_t nF = (size_t)paths * steps * MSK_NF, nW = (size_t)paths * steps * MSK_NWT;
  st = msk_ensure_scratch(ctx, (nF + nW + (size_t)paths + 2) * sizeof(double));
  if (st != MSK_OK) return st;
  double* F = reinterpret_cast<double*>(ctx->scratch);
  double* Wt = F + nF;
  long long* order_buf = reinterpret_cast<long long*>(Wt + nW);
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(order_buf + paths);
  st = launch_brownian(ctx, steps, paths, F, false, s, precision == MSK_F32);
  if (st == MSK_OK) st = launch_omega(ctx, order, steps, paths, precision, F, Wt, s);
  if (st == MSK_OK)
    st = launch_magnus_queued(ctx, steps, paths, precision, Wt, u_out_dev, path_status_dev, s, order_buf, queue,
                              out_on_host ? nullptr : queue + 1);
  return st;
}

extern "C" msk_status msk_solve_magnus(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                                       void* u_out_dev, uint32_t* path_status_dev, void* stream) {
  return solve_magnus(ctx, order, steps, paths, precision, u_out_dev, path_status_dev, stream, false);
}

// The device address of a page-locked, mapped host buffer (nullptr if it is not one).
static void* mapped_device_ptr(void* host) {
  if (!host) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost) return nullptr;
  void* dev = nullptr;
  if (cudaHostGetDevicePointer(&dev, host, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return dev;
}

extern "C" msk_status msk_solve_magnus_host(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                                            const double* u0_host, void* u_out_host, uint32_t* path_status_host,
                                            void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (order < 1 || order > 3) return msk_fail(ctx, MSK_ERR_ARG, "order must be 1, 2 or 3");
  if (precision != MSK_F64 && precision != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  msk_status st = check_steps(ctx, steps, paths);
  if (st != MSK_OK) return st;
  if (paths == 0) return MSK_OK;
  if (!u_out_host) return msk_fail(ctx, MSK_ERR_ARG, "null output");
  st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  void* out = mapped_device_ptr(u_out_host);
  if (!out) return msk_fail(ctx, MSK_ERR_ARG, "u_out_host is not page-locked host memory mapped into the device");
  uint32_t* status = nullptr;
  if (path_status_host) {
    status = static_cast<uint32_t*>(mapped_device_ptr(path_status_host));
    if (!status)
      return msk_fail(ctx, MSK_ERR_ARG, "path_status_host is not page-locked host memory mapped into the device");
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (u0_host) {
    const size_t dd = (size_t)ctx->d * ctx->d;
    st = msk_cuda(ctx, cudaMemcpyAsync(ctx->u0, u0_host, dd * sizeof(double), cudaMemcpyHostToDevice, s),
                  "copy u0 from the host");
    if (st != MSK_OK) return st;
  }
  return solve_magnus(ctx, order, steps, paths, precision, out, status, stream, true);
}

extern "C" msk_status msk_solve_euler(msk_ctx* ctx, int steps, int64_t paths, int precision, void* u_out_dev,
                                      uint32_t* path_status_dev, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (precision != MSK_F64 && precision != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  msk_status st = check_steps(ctx, steps, paths);
  if (st != MSK_OK) return st;
  if (paths == 0) return MSK_OK;
  if (!u_out_dev) return msk_fail(ctx, MSK_ERR_ARG, "null output");
  cudaStream_t s = (cudaStream_t)stream;
  st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  // scratch: increments [paths][steps], then the per-step coefficient table (2 doubles + 2 floats)
  st = msk_ensure_scratch(ctx, ((size_t)paths * steps + 3 * (size_t)steps) * sizeof(double));
  if (st != MSK_OK) return st;
  double* dW = reinterpret_cast<double*>(ctx->scratch);
  EngineSnap x;
  double* em_d = dW + (size_t)paths * steps;
  x.em_d = em_d;
  x.em_f = reinterpret_cast<float*>(em_d + 2 * (size_t)steps);
  st = launch_brownian(ctx, steps, paths, dW, true, s, precision == MSK_F32);
  if (st == MSK_OK) st = launch_em_table(ctx, steps, em_d, const_cast<float*>(x.em_f), s);
  if (st == MSK_OK)
    st = launch_engine_ex(ctx, true, steps, paths, precision, nullptr, dW, u_out_dev, path_status_dev, s, x);
  return st;
}

extern "C" msk_status msk_magnus_from_weights(msk_ctx* ctx, int steps, int64_t paths, int precision,
                                              const double* Wt_dev, void* u_out_dev, uint32_t* path_status_dev,
                                              void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (precision != MSK_F64 && precision != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  msk_status st = check_steps(ctx, steps, paths);
  if (st != MSK_OK) return st;
  if (paths == 0) return MSK_OK;
  if (!Wt_dev || !u_out_dev) return msk_fail(ctx, MSK_ERR_ARG, "null buffer");
  st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  // scratch: the engine's path order and two queue counters
  st = msk_ensure_scratch(ctx, ((size_t)paths + 2) * sizeof(double));
  if (st != MSK_OK) return st;
  long long* order_buf = reinterpret_cast<long long*>(ctx->scratch);
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(order_buf + paths);
  return launch_magnus_queued(ctx, steps, paths, precision, Wt_dev, u_out_dev, path_status_dev,
                              (cudaStream_t)stream, order_buf, queue, queue + 1);
}

extern "C" msk_status msk_work_counter(msk_ctx* ctx, uint64_t* matvecs_host, int reset, void* stream) {
  if (!ctx || !matvecs_host) return MSK_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  unsigned long long v = 0;
  st = msk_cuda(ctx, cudaMemcpyAsync(&v, ctx->work, sizeof(v), cudaMemcpyDeviceToHost, s), "read counter");
  if (st != MSK_OK) return st;
  st = msk_cuda(ctx, cudaStreamSynchronize(s), "sync counter");
  if (st != MSK_OK) return st;
  *matvecs_host = (uint64_t)v;
  if (reset) st = msk_cuda(ctx, cudaMemsetAsync(ctx->work, 0, sizeof(unsigned long long), s), "reset counter");
  return st;
}

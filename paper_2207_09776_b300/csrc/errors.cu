// S8/S9: closed-form solution, error norms and moments.
//
// Closed form (Section 3.1 gives the fundamental solution Gamma for constant
// 0 < sigma^2 < a and leaves the Gaussian-datum solution to the authors' code;
// re-derived by Fourier transform in (x, v) along the characteristics):
//   u_T(z) = c0 N(z; M_T m0 + c_T, M_T S0 M_T^T + C_T),  M_T = [[1, -kappa T], [0, 1]],
//   C_T = int_0^T (a - sigma^2)(t) m(T-t) m(T-t)^T dt,  m(tau) = (-kappa tau, 1),
//   c_T = (kappa int_0^T omega dt, -omega_T),  omega_t = int_0^t sigma dW,
// with omega_T and int omega dt the whole-interval functionals (one step).
// Err of Eq. meanErr is the per-path relative Frobenius error over the central
// 2^-kappa block, averaged over paths.
#include "msk_internal.cuh"

namespace {

__device__ __forceinline__ double sigma_t(const CoefDev& c, double t) {
  return c.s0 * (1.0 + c.s1 * cospi(2.0 * t));
}
__device__ __forceinline__ double a_t(const CoefDev& c, double t) { return c.a0 + c.a1 * sinpi(2.0 * t); }

// C_T by composite Simpson with 2^16 intervals (one block).
__global__ void diffusion_cov_kernel(CoefDev c, double kappa, double T, double* out) {
  constexpr int N = 1 << 16;
  const double hq = T / N;
  double sxx = 0, sxv = 0, svv = 0;
  for (int q = threadIdx.x; q <= N; q += blockDim.x) {
    const double t = q * hq;
    const double wq = (q == 0 || q == N) ? 1.0 : ((q & 1) ? 4.0 : 2.0);
    const double s = sigma_t(c, t);
    const double g = a_t(c, t) - s * s;
    const double tau = T - t;
    sxx += wq * g * kappa * kappa * tau * tau;
    sxv += wq * g * (-kappa * tau);
    svv += wq * g;
  }
  __shared__ double red[3][256];
  red[0][threadIdx.x] = sxx;
  red[1][threadIdx.x] = sxv;
  red[2][threadIdx.x] = svv;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int r = 0; r < 3; ++r) red[r][threadIdx.x] += red[r][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int r = 0; r < 3; ++r) out[r] = red[r][0] * hq / 3.0;
}

struct GaussArgs {
  int D;
  double ax, dx, av, dv, kappa, T;
  msk_gaussian g;
  const double* cT;   // C_T (xx, xv, vv)
};

// mean and covariance of u_T / c0 for one path from its whole-interval functionals
__device__ void terminal_gaussian(const GaussArgs& a, const double* F1, double m[2], double S[3]) {
  const double kT = a.kappa * a.T;
  // M m0
  m[0] = a.g.mean_x - kT * a.g.mean_v + a.kappa * F1[MSK_F_JOM];
  m[1] = a.g.mean_v - F1[MSK_F_OM];
  // M S0 M^T with M = [[1, -kT], [0, 1]]
  const double sxx = a.g.cov_xx, sxv = a.g.cov_xv, svv = a.g.cov_vv;
  S[0] = sxx - 2.0 * kT * sxv + kT * kT * svv + a.cT[0];
  S[1] = sxv - kT * svv + a.cT[1];
  S[2] = svv + a.cT[2];
}

__device__ __forceinline__ double gauss_at(double x, double v, const double m[2], const double S[3],
                                           double scale) {
  const double det = S[0] * S[2] - S[1] * S[1];
  const double ex = x - m[0], ev = v - m[1];
  const double q = (S[2] * ex * ex - 2.0 * S[1] * ex * ev + S[0] * ev * ev) / det;
  return scale * exp(-0.5 * q) / (2.0 * M_PI * sqrt(det));
}

__global__ void explicit_kernel(GaussArgs a, const double* F1, double* out) {
  const int64_t p = blockIdx.x;
  double m[2], S[3];
  terminal_gaussian(a, F1 + p * MSK_NF, m, S);
  const int D = a.D;
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int i = e % D, j = e / D;
    out[p * D * D + e] = gauss_at(a.ax + (i + 1) * a.dx, a.av + (j + 1) * a.dv, m, S, a.g.scale);
  }
}

template <typename TU, typename TR, bool EXPLICIT>
__global__ void error_kernel(GaussArgs a, const TU* u, const TR* ref, const double* F1, int lo, int len,
                             double* err) {
  const int64_t p = blockIdx.x;
  const int D = a.D;
  double m[2] = {0, 0}, S[3] = {1, 0, 1};
  if (EXPLICIT) terminal_gaussian(a, F1 + p * MSK_NF, m, S);
  double num = 0.0, den = 0.0;
  for (int e = threadIdx.x; e < len * len; e += blockDim.x) {
    const int i = lo + e % len, j = lo + e / len;
    const size_t off = (size_t)p * D * D + (size_t)j * D + i;
    double r;
    if (EXPLICIT) r = gauss_at(a.ax + (i + 1) * a.dx, a.av + (j + 1) * a.dv, m, S, a.g.scale);
    else r = (double)ref[off];
    const double d = r - (double)u[off];
    num += d * d;
    den += r * r;
  }
  __shared__ double rn[256], rd[256];
  rn[threadIdx.x] = num;
  rd[threadIdx.x] = den;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      rn[threadIdx.x] += rn[threadIdx.x + s];
      rd[threadIdx.x] += rd[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) err[p] = sqrt(rn[0] / rd[0]);
}

__global__ void mean_kernel(const double* x, int64_t n, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) s += x[q];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / (double)n;
}

template <typename TU>
__global__ void moments_kernel(GaussArgs a, const TU* u, double* mom) {
  const int64_t p = blockIdx.x;
  const int D = a.D;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int i = e % D, j = e / D;
    const double x = a.ax + (i + 1) * a.dx, v = a.av + (j + 1) * a.dv;
    const double w = (double)u[(size_t)p * D * D + e];
    s[0] += w;
    s[1] += w * x;
    s[2] += w * v;
    s[3] += w * x * x;
    s[4] += w * x * v;
    s[5] += w * v * v;
  }
  __shared__ double red[6][256];
  for (int r = 0; r < 6; ++r) red[r][threadIdx.x] = s[r];
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k)
      for (int r = 0; r < 6; ++r) red[r][threadIdx.x] += red[r][threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double cell = a.dx * a.dv;
    const double mass = red[0][0] * cell;
    const double ex = red[1][0] * cell / mass, ev = red[2][0] * cell / mass;
    double* o = mom + p * 6;
    o[0] = mass;
    o[1] = ex;
    o[2] = ev;
    o[3] = red[3][0] * cell / mass - ex * ex;
    o[4] = red[4][0] * cell / mass - ex * ev;
    o[5] = red[5][0] * cell / mass - ev * ev;
  }
}

GaussArgs gauss_args(msk_ctx* ctx) {
  GaussArgs a;
  a.D = ctx->d;
  a.ax = ctx->ax;
  a.dx = ctx->dx;
  a.av = ctx->av;
  a.dv = ctx->dv;
  a.kappa = (double)ctx->coef.drift_sign;
  a.T = ctx->T;
  a.g = ctx->u0g;
  a.cT = ctx->aux + MSK_NOPS;
  return a;
}

}  // namespace

msk_status launch_diffusion_cov(msk_ctx* ctx, cudaStream_t stream) {
  diffusion_cov_kernel<<<1, 256, 0, stream>>>(coef_dev(ctx->coef), (double)ctx->coef.drift_sign, ctx->T,
                                              ctx->aux + MSK_NOPS);
  return msk_cuda(ctx, cudaGetLastError(), "diffusion covariance");
}

// Whole-interval functionals (omega_T, int omega dt) into scratch, and C_T for the current T.
static msk_status whole_interval_functionals(msk_ctx* ctx, int64_t paths, double** F1, cudaStream_t s) {
  msk_status st = msk_ensure_scratch(ctx, (size_t)paths * MSK_NF * sizeof(double));
  if (st != MSK_OK) return st;
  st = launch_diffusion_cov(ctx, s);
  if (st != MSK_OK) return st;
  *F1 = reinterpret_cast<double*>(ctx->scratch);
  return launch_brownian(ctx, 1, paths, *F1, false, s);
}

extern "C" msk_status msk_explicit_solution(msk_ctx* ctx, int64_t paths, double* u_out_dev, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (paths < 0) return msk_fail(ctx, MSK_ERR_ARG, "paths < 0");
  if (paths == 0) return MSK_OK;
  if (!u_out_dev) return msk_fail(ctx, MSK_ERR_ARG, "null buffer");
  if (ctx->xprof || ctx->gen) return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "no closed form with variable coefficients");
  cudaStream_t s = (cudaStream_t)stream;
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  double* F1 = nullptr;
  st = whole_interval_functionals(ctx, paths, &F1, s);
  if (st != MSK_OK) return st;
  explicit_kernel<<<(unsigned)paths, 256, 0, s>>>(gauss_args(ctx), F1, u_out_dev);
  return msk_cuda(ctx, cudaGetLastError(), "explicit kernel");
}

extern "C" msk_status msk_error(msk_ctx* ctx, const void* u_dev, int u_precision, int64_t paths,
                                int ref_kind, const void* ref_dev, int ref_precision, int kappa,
                                double* err_per_path_dev, double* err_mean_dev, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (paths < 0) return msk_fail(ctx, MSK_ERR_ARG, "paths < 0");
  if ((u_precision != MSK_F64 && u_precision != MSK_F32) ||
      (ref_kind == MSK_REF_BUFFER && ref_precision != MSK_F64 && ref_precision != MSK_F32))
    return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  if (ref_kind != MSK_REF_EXPLICIT && ref_kind != MSK_REF_BUFFER)
    return msk_fail(ctx, MSK_ERR_ARG, "bad ref_kind");
  const int D = ctx->d;
  if (kappa < 0 || kappa > 20 || (D >> kappa) < 1) return msk_fail(ctx, MSK_ERR_ARG, "kappa out of range");
  if (paths == 0) return MSK_OK;
  if (!u_dev || !err_per_path_dev || (ref_kind == MSK_REF_BUFFER && !ref_dev))
    return msk_fail(ctx, MSK_ERR_ARG, "null buffer");
  if (ref_kind == MSK_REF_EXPLICIT && (ctx->xprof || ctx->gen))
    return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "no closed form with variable coefficients");
  cudaStream_t s = (cudaStream_t)stream;
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  // [lo, lo + floor(d / 2^kappa)), lo = floor(d/2 - d/2^(kappa+1))
  const int len = D >> kappa;
  const int lo2 = (int)(((int64_t)D * ((1 << kappa) - 1)) >> (kappa + 1));
  GaussArgs a = gauss_args(ctx);
  const unsigned grid = (unsigned)paths;
  if (ref_kind == MSK_REF_EXPLICIT) {
    double* F1 = nullptr;
    st = whole_interval_functionals(ctx, paths, &F1, s);
    if (st != MSK_OK) return st;
    if (u_precision == MSK_F64)
      error_kernel<double, double, true><<<grid, 256, 0, s>>>(a, (const double*)u_dev, nullptr, F1, lo2, len,
                                                             err_per_path_dev);
    else
      error_kernel<float, double, true><<<grid, 256, 0, s>>>(a, (const float*)u_dev, nullptr, F1, lo2, len,
                                                            err_per_path_dev);
  } else {
    if (u_precision == MSK_F64 && ref_precision == MSK_F64)
      error_kernel<double, double, false><<<grid, 256, 0, s>>>(a, (const double*)u_dev, (const double*)ref_dev,
                                                              nullptr, lo2, len, err_per_path_dev);
    else if (u_precision == MSK_F32 && ref_precision == MSK_F64)
      error_kernel<float, double, false><<<grid, 256, 0, s>>>(a, (const float*)u_dev, (const double*)ref_dev,
                                                             nullptr, lo2, len, err_per_path_dev);
    else if (u_precision == MSK_F64 && ref_precision == MSK_F32)
      error_kernel<double, float, false><<<grid, 256, 0, s>>>(a, (const double*)u_dev, (const float*)ref_dev,
                                                             nullptr, lo2, len, err_per_path_dev);
    else
      error_kernel<float, float, false><<<grid, 256, 0, s>>>(a, (const float*)u_dev, (const float*)ref_dev,
                                                            nullptr, lo2, len, err_per_path_dev);
  }
  st = msk_cuda(ctx, cudaGetLastError(), "error kernel");
  if (st != MSK_OK) return st;
  if (err_mean_dev) {
    mean_kernel<<<1, 256, 0, s>>>(err_per_path_dev, paths, err_mean_dev);
    st = msk_cuda(ctx, cudaGetLastError(), "mean kernel");
  }
  return st;
}

extern "C" msk_status msk_moments(msk_ctx* ctx, const void* u_dev, int precision, int64_t paths,
                                  double* mom_dev, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (paths < 0) return msk_fail(ctx, MSK_ERR_ARG, "paths < 0");
  if (precision != MSK_F64 && precision != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  if (paths == 0) return MSK_OK;
  if (!u_dev || !mom_dev) return msk_fail(ctx, MSK_ERR_ARG, "null buffer");
  cudaStream_t s = (cudaStream_t)stream;
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  if (precision == MSK_F64)
    moments_kernel<double><<<(unsigned)paths, 256, 0, s>>>(gauss_args(ctx), (const double*)u_dev, mom_dev);
  else
    moments_kernel<float><<<(unsigned)paths, 256, 0, s>>>(gauss_args(ctx), (const float*)u_dev, mom_dev);
  return msk_cuda(ctx, cudaGetLastError(), "moments kernel");
}

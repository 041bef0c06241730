// S3: Brownian increments and per-step functionals, generated in-kernel.
//
// The paper evaluates the Lebesgue integrals of Eq. MagnusFormulas by simple
// Riemann sums on a fine grid of mesh Delta^Leb (Section 3, "Implementation"
// and "Error and notations").  The rule is read as the exact integral of the
// piecewise-linear interpolant of W through the fine nodes; on a fine cell of
// width delta with end values w0, w1 (step-local W~, restarted at the step):
//     int W~    += delta (w0 + w1) / 2
//     int W~^2  += delta (w0^2 + w0 w1 + w1^2) / 3
//     int s W~  += delta (s0 (2 w0 + w1) + s1 (w0 + 2 w1)) / 6
// and, for time-dependent sigma, alpha = a/2 (dW = dW_k/delta ds on the cell):
//     omega~    += sigma(t_mid) dW_k                     (omega = int sigma dW)
//     int omega~ += delta (omega0 + omega1) / 2
//     G1 = int omega~ ds - sum s_mid sigma(t_mid) dW_k
//     G2 = delta/2 sum (alpha0 omega0 + alpha1 omega1) - sum alpha_bar(s_mid) sigma(t_mid) dW_k.
// One thread integrates one (path, step) pair sequentially over its fine cells.
#include "philox.cuh"
#include "msk_internal.cuh"

namespace {

struct BrownArgs {
  uint64_t seed, path_offset;
  int64_t n_fine, paths;
  int steps;
  double T;
  CoefDev c;
};

__device__ __forceinline__ double sigma_t(const CoefDev& c, double t) {
  return c.s0 * (1.0 + c.s1 * cospi(2.0 * t));
}
__device__ __forceinline__ double alpha_t(const CoefDev& c, double t) {
  return 0.5 * (c.a0 + c.a1 * sinpi(2.0 * t));
}
// int_{t0}^{t0+s} alpha
__device__ __forceinline__ double alpha_bar(const CoefDev& c, double t0, double s) {
  return 0.5 * (c.a0 * s + c.a1 * (cospi(2.0 * t0) - cospi(2.0 * (t0 + s))) / (2.0 * M_PI));
}

template <bool FULL, bool TRIG>
__global__ void brownian_kernel(BrownArgs a, double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.paths * a.steps) return;
  const int64_t p = idx / a.steps;
  const int n = (int)(idx % a.steps);
  const int64_t L = a.n_fine / a.steps;
  const double delta = a.T / (double)a.n_fine;
  const double sq = sqrt(delta);
  const double h = a.T / a.steps;
  const double tn = n * h;
  const uint64_t gpath = a.path_offset + (uint64_t)p;
  const int64_t f0 = (int64_t)n * L;

  double w0 = 0.0, I1 = 0.0, I2 = 0.0, I3 = 0.0;
  double om0 = 0.0, jom = 0.0, ssdw = 0.0, jaom = 0.0, abdw = 0.0;
  double z0 = 0.0, z1 = 0.0;
  for (int64_t k = 0; k < L; ++k) {
    const int64_t fi = f0 + k;
    if (k == 0 || (fi & 1) == 0) brownian_pair(a.seed, gpath, 0u, (uint64_t)(fi >> 1), z0, z1);
    const double dw = sq * ((fi & 1) ? z1 : z0);
    const double w1 = w0 + dw;
    if (FULL) {
      const double s0 = delta * (double)k, s1 = delta * (double)(k + 1);
      I1 += delta * (w0 + w1) / 2.0;
      I2 += delta * (w0 * w0 + w0 * w1 + w1 * w1) / 3.0;
      I3 += delta * (s0 * (2.0 * w0 + w1) + s1 * (w0 + 2.0 * w1)) / 6.0;
      const double smid = delta * ((double)k + 0.5);
      const double sig = TRIG ? sigma_t(a.c, tn + smid) : a.c.s0;
      const double om1 = om0 + sig * dw;
      jom += delta * (om0 + om1) / 2.0;
      ssdw += smid * sig * dw;
      if (TRIG) {
        jaom += delta * (alpha_t(a.c, tn + s0) * om0 + alpha_t(a.c, tn + s1) * om1) / 2.0;
        abdw += alpha_bar(a.c, tn, smid) * sig * dw;
      } else {
        const double al = 0.5 * a.c.a0;
        jaom += delta * (al * om0 + al * om1) / 2.0;
        abdw += al * smid * sig * dw;
      }
      om0 = om1;
    }
    w0 = w1;
  }
  if (FULL) {
    double* o = out + idx * MSK_NF;
    o[MSK_F_DW] = w0;
    o[MSK_F_I1] = I1;
    o[MSK_F_I2] = I2;
    o[MSK_F_I3] = I3;
    o[MSK_F_OM] = om0;
    o[MSK_F_JOM] = jom;
    o[MSK_F_G1] = jom - ssdw;
    o[MSK_F_G2] = jaom - abdw;
  } else {
    out[idx] = w0;
  }
}

}  // namespace

msk_status launch_brownian(msk_ctx* ctx, int steps, int64_t paths, double* out, bool increments_only,
                           cudaStream_t stream) {
  BrownArgs a{ctx->seed, ctx->path_offset, ctx->n_fine, paths, steps, ctx->T, coef_dev(ctx->coef)};
  const int64_t n = paths * steps;
  if (n == 0) return MSK_OK;
  const int threads = 128;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  const bool trig = ctx->coef.kind == MSK_COEF_TRIG;
  if (increments_only) brownian_kernel<false, false><<<blocks, threads, 0, stream>>>(a, out);
  else if (trig) brownian_kernel<true, true><<<blocks, threads, 0, stream>>>(a, out);
  else brownian_kernel<true, false><<<blocks, threads, 0, stream>>>(a, out);
  return msk_cuda(ctx, cudaGetLastError(), "brownian kernel");
}

// S1/S2: grid, finite-difference operators and the basis-operator band tables.
//
// The v-factors of the thirteen basis operators are products and commutators
// of three banded n_v x n_v matrices (Section 2, "Computation of A and B"):
//     Nv = diag(v_j),  T1 = D^v = tridiag(-1,0,1)/(2 dv),  T2 = D^vv = tridiag(1,-2,1)/dv^2,
// with v_j = av + (j+1) dv.  Products are evaluated entry-wise from the band
// structure of the truncated matrices, so boundary rows come out exactly as
// the products of the truncated matrices (the commutators of Eq.
// MagnusFormulas computed the way the paper computes them, as sparse matrix
// products).  Commutators with Nv use the exact difference v_j - v_l =
// (j - l) dv, so interior rows are bit-identical.  Products and sums use
// explicit round-to-nearest operations (no fused multiply-add contraction), so
// x y - y x cancels to an exact zero as it does in unfused arithmetic.
#include "philox.cuh"
#include "stencil.cuh"

namespace {

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

struct VPrims {
  int D;
  double dv, av, kappa;
  __device__ double nv(int j, int l) const { return j == l ? add(av, mul((double)(j + 1), dv)) : 0.0; }
  __device__ double t1(int j, int l) const {
    if (l < 0 || l >= D || j < 0 || j >= D) return 0.0;
    if (l == j + 1) return 0.5 / dv;
    if (l == j - 1) return -0.5 / dv;
    return 0.0;
  }
  __device__ double t2(int j, int l) const {
    if (l < 0 || l >= D || j < 0 || j >= D) return 0.0;
    if (l == j) return -2.0 / (dv * dv);
    if (l == j + 1 || l == j - 1) return 1.0 / (dv * dv);
    return 0.0;
  }
  // P = [Nv, T1], Q = [T2, T1]
  __device__ double P(int j, int l) const { return mul(mul((double)(j - l), dv), t1(j, l)); }
  __device__ double Q(int j, int l) const {
    if (j < 0 || j >= D || l < 0 || l >= D) return 0.0;
    double s = 0.0;
    for (int m = j - 1; m <= j + 1; ++m) s = add(s, sub(mul(t2(j, m), t1(m, l)), mul(t1(j, m), t2(m, l))));
    return s;
  }
  __device__ double entry(int op, int j, int l) const {
    if (j < 0 || j >= D || l < 0 || l >= D) return 0.0;
    switch (op) {
      case MSK_OP_BX: return mul(kappa, nv(j, l));
      case MSK_OP_BVV: return t2(j, l);
      case MSK_OP_A0: return t1(j, l);
      case MSK_OP_A0A0: {
        double s = 0.0;
        for (int m = j - 1; m <= j + 1; ++m) s = add(s, mul(t1(j, m), t1(m, l)));
        return s;
      }
      case MSK_OP_BX_A0: return mul(kappa, P(j, l));
      case MSK_OP_BVV_A0: return Q(j, l);
      case MSK_OP_BX_BVV: return mul(kappa, mul(mul((double)(j - l), dv), t2(j, l)));
      case MSK_OP_BXA0_A0: {
        double s = 0.0;
        for (int m = j - 1; m <= j + 1; ++m) s = add(s, sub(mul(P(j, m), t1(m, l)), mul(t1(j, m), P(m, l))));
        return mul(kappa, s);
      }
      case MSK_OP_BVVA0_A0: {
        double s = 0.0;
        for (int m = j - 2; m <= j + 2; ++m) s = add(s, sub(mul(Q(j, m), t1(m, l)), mul(t1(j, m), Q(m, l))));
        return s;
      }
      case MSK_OP_BXA0_BX: return mul(mul(kappa, kappa), mul(mul((double)(l - j), dv), P(j, l)));
      case MSK_OP_BXA0_BVV: {
        double s = 0.0;
        for (int m = j - 1; m <= j + 1; ++m) s = add(s, sub(mul(P(j, m), t2(m, l)), mul(t2(j, m), P(m, l))));
        return mul(kappa, s);
      }
      case MSK_OP_BVVA0_BX: return mul(kappa, mul(mul((double)(l - j), dv), Q(j, l)));
      case MSK_OP_BVVA0_BVV: {
        double s = 0.0;
        for (int m = j - 2; m <= j + 2; ++m) s = add(s, sub(mul(Q(j, m), t2(m, l)), mul(t2(j, m), Q(m, l))));
        return s;
      }
    }
    return 0.0;
  }
};

__global__ void band_tables_kernel(VPrims p, double* band) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = MSK_NOPS * p.D * MSK_BAND;
  if (idx >= total) return;
  const int o = idx % MSK_BAND;
  const int j = (idx / MSK_BAND) % p.D;
  const int k = idx / (MSK_BAND * p.D);
  band[idx] = p.entry(k, j, j + o - 2);
}

// Checks the structure the stencil kernels rely on and computes the traces.
// flags: bit 0 = a non-zero outside the 15-point stencil, bit 1 = an interior
// row differs from row 2 (other than the centre of a D^x-class operator),
// bit 2 = bandwidth 3 entries non-zero.
__global__ void band_check_kernel(VPrims p, const double* band, double dx, double* trace,
                                  int* flags) {
  const int k = blockIdx.x;
  const int D = p.D;
  const int xc = c_op_xclass[k];
  double tr = 0.0;
  for (int j = threadIdx.x; j < D; j += blockDim.x) {
    const double* b = band + ((size_t)k * D + j) * MSK_BAND;
    tr += b[2];
    if (xc == XC_DX && (b[0] != 0.0 || b[4] != 0.0)) atomicOr(flags, 1);
    if (xc == XC_DXX && (b[0] != 0.0 || b[2] != 0.0 || b[4] != 0.0)) atomicOr(flags, 1);
    if (p.entry(k, j, j + 3) != 0.0 || p.entry(k, j, j - 3) != 0.0) atomicOr(flags, 4);
    if (!is_special_row(j, D)) {
      const double* r2 = band + ((size_t)k * D + 2) * MSK_BAND;
      for (int o = 0; o < MSK_BAND; ++o) {
        if (o == 2 && xc == XC_DX) continue;
        if (b[o] != r2[o]) atomicOr(flags, 2);
      }
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = tr;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // trace(V (x) X) = trace(V) trace(X); trace(D^x) = 0,
    // trace((D^x)^2) = -(2 D - 2) / (4 dx^2) (centre -2 inside, -1 on the two edge rows)
    double tX = xc == XC_I ? (double)D : (xc == XC_DX ? 0.0 : -(2.0 * D - 2.0) / (4.0 * dx * dx));
    trace[k] = red[0] * tX;
  }
}

__global__ void gaussian_u0_kernel(int D, double ax, double dx, double av, double dv, msk_gaussian g,
                                   double* u0) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= D * D) return;
  const int i = idx % D, j = idx / D;
  const double x = ax + (i + 1) * dx, v = av + (j + 1) * dv;
  const double det = g.cov_xx * g.cov_vv - g.cov_xv * g.cov_xv;
  const double ex = x - g.mean_x, ev = v - g.mean_v;
  const double q = (g.cov_vv * ex * ex - 2.0 * g.cov_xv * ex * ev + g.cov_xx * ev * ev) / det;
  u0[idx] = g.scale * exp(-0.5 * q) / (2.0 * M_PI * sqrt(det));
}

// out = Omega u, one thread per grid point, with Omega's coefficients folded per row.
__global__ void apply_omega_kernel(const double* band, int D, double inv2dx, double inv4dx2,
                                   const double* weights, int64_t paths, const double* u,
                                   double* out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t pts = (int64_t)D * D;
  if (idx >= paths * pts) return;
  const int64_t p = idx / pts;
  const int rem = (int)(idx % pts);
  const int i = rem % D, j = rem / D;
  double w[MSK_NOPS];
  for (int k = 0; k < MSK_NOPS; ++k) w[k] = weights[p * MSK_NOPS + k];
  double c[MSK_NCOEF];
  fold_row(band, D, j, w, 0.0, inv2dx, inv4dx2, c);
  const double* U = u + p * pts;
  auto at = [&](int ii, int jj) -> double {
    return (ii < 0 || ii >= D || jj < 0 || jj >= D) ? 0.0 : U[(int64_t)jj * D + ii];
  };
  const bool edge = (i == 0 || i == D - 1);
  const double a1 = edge ? c[CF_AE + 0] : c[CF_A + 1];
  const double a3 = edge ? c[CF_AE + 1] : c[CF_A + 3];
  double v = c[CF_A + 0] * at(i, j - 2) + a1 * at(i, j - 1) + c[CF_A + 2] * at(i, j) +
             a3 * at(i, j + 1) + c[CF_A + 4] * at(i, j + 2);
  for (int o = -1; o <= 1; ++o) v += c[CF_B + o + 1] * (at(i + 1, j + o) - at(i - 1, j + o));
  v += c[CF_C + 0] * (at(i + 2, j - 1) + at(i - 2, j - 1));
  v += c[CF_C + 1] * (at(i + 2, j + 1) + at(i - 2, j + 1));
  out[idx] = v;
}

__global__ void philox_words_kernel(uint64_t seed, uint64_t path, uint32_t tag, int64_t first,
                                    int64_t n, uint32_t* out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const uint64_t j = (uint64_t)(first + q);
  const uint4 w = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)path, (uint32_t)(path >> 32), tag),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  out[4 * q + 0] = w.x;
  out[4 * q + 1] = w.y;
  out[4 * q + 2] = w.z;
  out[4 * q + 3] = w.w;
}

}  // namespace

msk_status launch_band_tables(msk_ctx* ctx, cudaStream_t stream) {
  VPrims p{ctx->d, ctx->dv, ctx->av, (double)ctx->coef.drift_sign};
  const int total = MSK_NOPS * ctx->d * MSK_BAND;
  band_tables_kernel<<<(total + 255) / 256, 256, 0, stream>>>(p, ctx->band);
  int* dflags = reinterpret_cast<int*>(ctx->aux + MSK_NOPS + 8);
  msk_status st = msk_cuda(ctx, cudaMemsetAsync(dflags, 0, sizeof(int), stream), "memset flags");
  if (st != MSK_OK) return st;
  band_check_kernel<<<MSK_NOPS, 256, 0, stream>>>(p, ctx->band, ctx->dx, ctx->aux, dflags);
  st = msk_cuda(ctx, cudaGetLastError(), "band tables");
  if (st != MSK_OK) return st;
  int flags = 0;
  double tr[MSK_NOPS];
  st = msk_cuda(ctx, cudaMemcpyAsync(&flags, dflags, sizeof(int), cudaMemcpyDeviceToHost, stream),
                "copy flags");
  if (st != MSK_OK) return st;
  st = msk_cuda(ctx, cudaMemcpyAsync(tr, ctx->aux, sizeof(tr), cudaMemcpyDeviceToHost, stream),
                "copy traces");
  if (st != MSK_OK) return st;
  st = msk_cuda(ctx, cudaStreamSynchronize(stream), "sync tables");
  if (st != MSK_OK) return st;
  if (flags != 0)
    return msk_fail(ctx, MSK_ERR_UNSUPPORTED,
                    "operator tables do not fit the 15-point widened stencil (flags " +
                        std::to_string(flags) + ")");
  for (int k = 0; k < MSK_NOPS; ++k) ctx->host_trace[k] = tr[k];
  return MSK_OK;
}

msk_status launch_gaussian_u0(msk_ctx* ctx, cudaStream_t stream) {
  const int n = ctx->d * ctx->d;
  gaussian_u0_kernel<<<(n + 255) / 256, 256, 0, stream>>>(ctx->d, ctx->ax, ctx->dx, ctx->av, ctx->dv,
                                                          ctx->u0g, ctx->u0);
  msk_status st = msk_cuda(ctx, cudaGetLastError(), "gaussian u0");
  if (st != MSK_OK) return st;
  return msk_cuda(ctx, cudaStreamSynchronize(stream), "sync u0");
}

extern "C" msk_status msk_apply_omega(msk_ctx* ctx, const double* weights_dev, int64_t paths,
                                      const double* u_dev, double* out_dev, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (paths < 0) return msk_fail(ctx, MSK_ERR_ARG, "paths < 0");
  if (paths == 0) return MSK_OK;
  if (!weights_dev || !u_dev || !out_dev) return msk_fail(ctx, MSK_ERR_ARG, "null buffer");
  if (ctx->xprof || ctx->gen)
    return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "the widened-stencil tables hold only the Langevin coefficients");
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  const int64_t n = paths * (int64_t)ctx->d * ctx->d;
  const int64_t blocks = (n + 255) / 256;
  apply_omega_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      ctx->band, ctx->d, 0.5 / ctx->dx, 0.25 / (ctx->dx * ctx->dx), weights_dev, paths, u_dev, out_dev);
  return msk_cuda(ctx, cudaGetLastError(), "apply omega");
}

extern "C" msk_status msk_philox_words(uint64_t seed, uint64_t path, uint32_t tag, int64_t first_pair,
                                       int64_t npairs, uint32_t* out_dev, void* stream) {
  if (npairs < 0 || first_pair < 0 || first_pair + npairs > (int64_t)0x100000000LL) return MSK_ERR_ARG;
  if (npairs == 0) return MSK_OK;
  if (!out_dev) return MSK_ERR_ARG;
  philox_words_kernel<<<(unsigned)((npairs + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      seed, path, tag, first_pair, npairs, out_dev);
  return cudaGetLastError() == cudaSuccess ? MSK_OK : MSK_ERR_CUDA;
}

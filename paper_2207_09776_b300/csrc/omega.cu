// S4 + S5a: Magnus weights, trace shift, norm bound and Taylor (s, m) per (path, step).
//
// Constant coefficients, B = Bx + alpha Bvv, A = sigma A0 (alpha = a/2), step h,
// functionals dW, I1, I2, I3 of the step (Eq. MagnusFormulas):
//   Y1: h B + dW A
//   Y2: - h/2 A^2 + (I1 - h dW / 2) [B,A]
//   Y3: + cA [[B,A],A] + cB [[B,A],B],
//       cA = I2/2 - dW I1/2 + h dW^2/12,  cB = I3 - h I1/2 - h^2 dW/12,
// expanded over the basis operators with [B,A] = sigma([Bx,A0] + alpha [Bvv,A0]) etc.
// Time-dependent coefficients: the order-2 extension obtained from the
// Appendix's Picard step with Y1_t = t Bx + alpha_bar_t Bvv + omega_t A0,
//   Y2 = h Bx + alpha_bar_h Bvv + omega_h A0 - (int sigma^2)/2 A0^2
//        + G1/2 [Bx,A0] + G2/2 [Bvv,A0] - G3/2 [Bx,Bvv],
// plus the two third-order terms with B, A frozen at the step midpoint.
//
// The exponential action uses a scaled truncated Taylor series; (s, m) follow
// Al-Mohy & Higham (2011): for ||Omega - mu I|| <= nrm, choose m minimising
// m ceil(nrm / theta_m) with theta_m the backward-error radius at the unit
// roundoff of the arithmetic, mu = trace(Omega)/n.  The norm is the exact
// infinity norm bound of the folded stencil (maximum absolute row sum).
#include <math.h>

#include "stencil.cuh"
#include "theta_tables.h"

namespace {

// reciprocals 1 / theta_m (one multiply per candidate degree instead of a double
// division, which is a long instruction sequence on this part's narrow double pipe)
__constant__ double c_inv_theta64[MSK_THETA_MMAX_F64];
__constant__ double c_inv_theta32[MSK_THETA_MMAX_F32];

struct OmegaArgs {
  const double* band;
  const double* trace;
  const double* var;   // x profile / general coefficients: traces [0, ops) and shifted norms [ops, 2 ops); else null
  int var_ops;         // 6: the six operators of constant coefficients; 13: the MSK_OP_* basis
  const double* job_th;   // interval mode: (t0, h) per record; else null (step n: t0 = n h, h = T / steps)
  int D, order, steps, precision;
  int64_t paths;
  double T, dx;
  CoefDev c;
  double s_cap;
};

__device__ __forceinline__ double sigma_t(const CoefDev& c, double t) {
  return c.s0 * (1.0 + c.s1 * cospi(2.0 * t));
}
__device__ __forceinline__ double alpha_t(const CoefDev& c, double t) {
  return 0.5 * (c.a0 + c.a1 * sinpi(2.0 * t));
}
__device__ __forceinline__ double alpha_bar(const CoefDev& c, double t0, double s) {
  return 0.5 * (c.a0 * s + c.a1 * (cospi(2.0 * t0) - cospi(2.0 * (t0 + s))) / (2.0 * M_PI));
}
// int_{t0}^{t0+h} sigma^2
__device__ double sigma_sq_int(const CoefDev& c, double t0, double h) {
  const double t1 = t0 + h, tp = 2.0 * M_PI;
  return c.s0 * c.s0 *
         (h + 2.0 * c.s1 * (sinpi(2.0 * t1) - sinpi(2.0 * t0)) / tp +
          c.s1 * c.s1 * (0.5 * h + (sinpi(4.0 * t1) - sinpi(4.0 * t0)) / (4.0 * tp)));
}
// int_0^h (s alpha(t0+s) - alpha_bar(t0, s)) ds = 2 int_0^h s alpha - h alpha_bar(h)
__device__ double g3_int(const CoefDev& c, double t0, double h) {
  const double t1 = t0 + h, cc = 2.0 * M_PI;
  const double trig = -h * cospi(2.0 * t1) / cc + (sinpi(2.0 * t1) - sinpi(2.0 * t0)) / (cc * cc);
  const double s_alpha = 0.5 * (c.a0 * h * h / 2.0 + c.a1 * trig);
  return 2.0 * s_alpha - h * alpha_bar(c, t0, h);
}

__device__ void magnus_weights(const OmegaArgs& a, double tn, double h, const double* f, double w[MSK_NOPS]) {
  for (int k = 0; k < MSK_NOPS; ++k) w[k] = 0.0;
  const double dW = f[MSK_F_DW], I1 = f[MSK_F_I1], I2 = f[MSK_F_I2], I3 = f[MSK_F_I3];
  const double cA = 0.5 * I2 - 0.5 * dW * I1 + h * dW * dW / 12.0;
  const double cB = I3 - 0.5 * h * I1 - h * h * dW / 12.0;
  if (a.c.kind == MSK_COEF_CONST) {
    const double al = 0.5 * a.c.a0, sg = a.c.s0;
    w[MSK_OP_BX] = h;
    w[MSK_OP_BVV] = al * h;
    w[MSK_OP_A0] = sg * dW;
    if (a.order >= 2) {
      const double c1 = I1 - 0.5 * h * dW;
      w[MSK_OP_A0A0] = -0.5 * sg * sg * h;
      w[MSK_OP_BX_A0] = sg * c1;
      w[MSK_OP_BVV_A0] = al * sg * c1;
    }
    if (a.order >= 3) {
      w[MSK_OP_BXA0_A0] = sg * sg * cA;
      w[MSK_OP_BVVA0_A0] = al * sg * sg * cA;
      w[MSK_OP_BXA0_BX] = sg * cB;
      w[MSK_OP_BXA0_BVV] = al * sg * cB;
      w[MSK_OP_BVVA0_BX] = al * sg * cB;
      w[MSK_OP_BVVA0_BVV] = al * al * sg * cB;
    }
  } else {
    w[MSK_OP_BX] = h;
    w[MSK_OP_BVV] = alpha_bar(a.c, tn, h);
    w[MSK_OP_A0] = f[MSK_F_OM];
    if (a.order >= 2) {
      w[MSK_OP_A0A0] = -0.5 * sigma_sq_int(a.c, tn, h);
      w[MSK_OP_BX_A0] = 0.5 * f[MSK_F_G1];
      w[MSK_OP_BVV_A0] = 0.5 * f[MSK_F_G2];
      w[MSK_OP_BX_BVV] = -0.5 * g3_int(a.c, tn, h);
    }
    if (a.order >= 3) {
      const double tm = tn + 0.5 * h;
      const double al = alpha_t(a.c, tm), sg = sigma_t(a.c, tm);
      w[MSK_OP_BXA0_A0] = sg * sg * cA;
      w[MSK_OP_BVVA0_A0] = al * sg * sg * cA;
      w[MSK_OP_BXA0_BX] = sg * cB;
      w[MSK_OP_BXA0_BVV] = al * sg * cB;
      w[MSK_OP_BVVA0_BX] = al * sg * cB;
      w[MSK_OP_BVVA0_BVV] = al * al * sg * cB;
    }
  }
}

__device__ double row_abs_sum(const double c[MSK_NCOEF]) {
  // interior-column sum; edge columns lose neighbours but may carry Ae instead of A[+-1]
  double s = fabs(c[CF_A + 0]) + fmax(fabs(c[CF_A + 1]), fabs(c[CF_AE + 0])) + fabs(c[CF_A + 2]) +
             fmax(fabs(c[CF_A + 3]), fabs(c[CF_AE + 1])) + fabs(c[CF_A + 4]);
  s += 2.0 * (fabs(c[CF_B + 0]) + fabs(c[CF_B + 1]) + fabs(c[CF_B + 2]));
  s += 2.0 * (fabs(c[CF_C + 0]) + fabs(c[CF_C + 1]));
  return s;
}

__global__ void omega_kernel(OmegaArgs a, const double* __restrict__ F, double* __restrict__ Wt) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.paths * a.steps) return;
  double tn, h;
  if (a.job_th) {
    tn = a.job_th[2 * idx];
    h = a.job_th[2 * idx + 1];
  } else {
    h = a.T / a.steps;
    tn = (double)(idx % a.steps) * h;
  }
  double w[MSK_NOPS];
  magnus_weights(a, tn, h, F + idx * MSK_NF, w);
  const int D = a.D;
  double mu, nrm = 0.0;
  if (a.var && a.var_ops == MSK_NOPS) {
    // x profile, time-dependent coefficients: the thirteen basis operators, each
    // with its exact trace and shifted norm
    double tr = 0.0;
    for (int k = 0; k < MSK_NOPS; ++k) {
      tr += w[k] * a.var[k];
      nrm += fabs(w[k]) * a.var[MSK_NOPS + k];
    }
    mu = tr / ((double)D * D);
  } else if (a.var) {
    // x profile (constant coefficients): Omega over the six operators B, A0, A0^2,
    // [B,A0], [[B,A0],A0], [[B,A0],B] with B = Bx + alpha Bvv; the bound is the sum
    // of |weight| x the exact norm of each operator minus its own trace shift
    const double w6[6] = {w[MSK_OP_BX],    w[MSK_OP_A0],      w[MSK_OP_A0A0],
                          w[MSK_OP_BX_A0], w[MSK_OP_BXA0_A0], w[MSK_OP_BXA0_BX]};
    double tr = 0.0;
    for (int k = 0; k < 6; ++k) {
      tr += w6[k] * a.var[k];
      nrm += fabs(w6[k]) * a.var[6 + k];
    }
    mu = tr / ((double)D * D);
  } else {
    double tr = 0.0;
    for (int k = 0; k < MSK_NOPS; ++k) tr += w[k] * a.trace[k];
    mu = tr / ((double)D * D);
    // infinity-norm bound of Omega - mu I over the row classes: the four boundary
    // rows and the two extreme interior rows (only V1's centre varies inside, linearly)
    const int rows[6] = {0, 1, 2, D - 3, D - 2, D - 1};
    for (int r = 0; r < 6; ++r) {
      double c[MSK_NCOEF];
      fold_row(a.band, D, rows[r], w, -mu, 0.5 / a.dx, 0.25 / (a.dx * a.dx), c);
      nrm = fmax(nrm, row_abs_sum(c));
    }
  }
  const double* ith = a.precision == MSK_F32 ? c_inv_theta32 : c_inv_theta64;
  const int mmax = a.precision == MSK_F32 ? MSK_THETA_MMAX_F32 : MSK_THETA_MMAX_F64;
  double best_s = 1.0, best_m = 0.0;
  if (nrm > 0.0) {
    double best_cost = INFINITY;
    for (int m = 1; m <= mmax; ++m) {
      const double s = fmax(1.0, ceil(nrm * ith[m - 1]));
      const double cost = m * s;
      if (cost < best_cost) {
        best_cost = cost;
        best_s = s;
        best_m = m;
      }
    }
    if (!(best_s <= a.s_cap)) best_s = a.s_cap;   // also catches a non-finite norm
  }
  double* o = Wt + idx * MSK_NWT;
  for (int k = 0; k < MSK_NOPS; ++k) o[k] = w[k];
  for (int k = MSK_NOPS; k < MSK_WT_MU; ++k) o[k] = 0.0;
  o[MSK_WT_MU] = mu;
  o[MSK_WT_NORM] = nrm;
  o[MSK_WT_S] = best_s;
  o[MSK_WT_M] = best_m;
}

bool g_theta_loaded[64] = {false};

// Coefficient profile of the weights: with general coefficients A already holds
// sigma and the coefficients are time-independent, so the weights are those of
// constant coefficients with sigma = 1.
CoefDev omega_coef(const msk_ctx* ctx) {
  CoefDev c = coef_dev(ctx->coef);
  if (ctx->gen) {
    c.kind = MSK_COEF_CONST;
    c.a0 = c.a1 = c.s1 = 0.0;
    c.s0 = 1.0;
  }
  return c;
}

}  // namespace

// Taylor scaling cap: beyond it the path is flagged MSK_PATH_SCALE_CAP.
extern const double kMskScaleCap = 16384.0;

// Upload the theta tables to this device's constant memory (once per device).
msk_status msk_prepare_omega(msk_ctx* ctx) {
  if (ctx->device >= 0 && ctx->device < 64 && !g_theta_loaded[ctx->device]) {
    double i64[MSK_THETA_MMAX_F64], i32[MSK_THETA_MMAX_F32];
    for (int m = 0; m < MSK_THETA_MMAX_F64; ++m) i64[m] = 1.0 / msk_theta_f64[m];
    for (int m = 0; m < MSK_THETA_MMAX_F32; ++m) i32[m] = 1.0 / msk_theta_f32[m];
    msk_status st = msk_cuda(ctx, cudaMemcpyToSymbol(c_inv_theta64, i64, sizeof(i64)), "theta64");
    if (st != MSK_OK) return st;
    st = msk_cuda(ctx, cudaMemcpyToSymbol(c_inv_theta32, i32, sizeof(i32)), "theta32");
    if (st != MSK_OK) return st;
    g_theta_loaded[ctx->device] = true;
  }
  return MSK_OK;
}

msk_status launch_omega(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                        const double* F, double* Wt, cudaStream_t stream) {
  msk_status st0 = msk_prepare_omega(ctx);
  if (st0 != MSK_OK) return st0;
  const int64_t n = paths * steps;
  if (n == 0) return MSK_OK;
  if (ctx->xprof || ctx->gen) {
    st0 = ensure_var_tables(ctx, stream);
    if (st0 != MSK_OK) return st0;
  }
  OmegaArgs a{ctx->band, ctx->aux, (ctx->xprof || ctx->gen) ? ctx->var_tab : nullptr, var_table_ops(ctx), nullptr,
              ctx->d, order, steps, precision, paths, ctx->T, ctx->dx, omega_coef(ctx), kMskScaleCap};
  omega_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(a, F, Wt);
  return msk_cuda(ctx, cudaGetLastError(), "omega kernel");
}

// Weight records of arbitrary intervals: job_th_dev[2 i], [2 i + 1] = (t0, h) of
// interval i, F its functionals (njobs records, one step each).
msk_status launch_omega_jobs(msk_ctx* ctx, int order, int64_t njobs, int precision, const double* F,
                             const double* job_th_dev, double* Wt, cudaStream_t stream) {
  msk_status st0 = msk_prepare_omega(ctx);
  if (st0 != MSK_OK) return st0;
  if (njobs == 0) return MSK_OK;
  if (ctx->xprof || ctx->gen) {
    st0 = ensure_var_tables(ctx, stream);
    if (st0 != MSK_OK) return st0;
  }
  OmegaArgs a{ctx->band, ctx->aux, (ctx->xprof || ctx->gen) ? ctx->var_tab : nullptr, var_table_ops(ctx),
              job_th_dev, ctx->d, order, 1, precision, njobs, ctx->T, ctx->dx, omega_coef(ctx), kMskScaleCap};
  omega_kernel<<<(unsigned)((njobs + 127) / 128), 128, 0, stream>>>(a, F, Wt);
  return msk_cuda(ctx, cudaGetLastError(), "omega kernel (intervals)");
}

extern "C" msk_status msk_omega_weights(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                                        const double* F_dev, double* Wt_dev, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (order < 1 || order > 3) return msk_fail(ctx, MSK_ERR_ARG, "order must be 1, 2 or 3");
  if (steps < 1 || ctx->n_fine % steps != 0)
    return msk_fail(ctx, MSK_ERR_ARG, "steps must be >= 1 and divide n_fine");
  if (paths < 0) return msk_fail(ctx, MSK_ERR_ARG, "paths < 0");
  if (precision != MSK_F64 && precision != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  if (paths == 0) return MSK_OK;
  if (!F_dev || !Wt_dev) return msk_fail(ctx, MSK_ERR_ARG, "null buffer");
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  return launch_omega(ctx, order, steps, paths, precision, F_dev, Wt_dev, (cudaStream_t)stream);
}

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
// The exponential action uses a scaled truncated Taylor series (T_m(A/s))^s with
// the backward-error radii theta_m of Al-Mohy & Higham (2011) at the unit
// roundoff of the arithmetic, A = Omega - mu I, mu = trace(Omega)/n.  Their
// Theorem 4.2 allows any p with p(p-1) <= m + 1 and
//   alpha_p(A) = max(||A^p||^(1/p), ||A^(p+1)||^(1/(p+1))) <= s theta_m,
// which is sharper than ||A|| <= s theta_m for these non-normal stencils.  Here
//   - ||A||_inf is exact (maximum absolute row sum of the folded stencil);
//   - A = X + E, X the deterministic part (every functional set to zero, shared
//     by all paths of a step) and E the Brownian part; ||X^q||_inf, q <= 9, are
//     computed exactly once per step by propagating unit rows (power_norm_kernel),
//     ||E||_inf per path, and expanding (X + E)^q into its 2^q words bounds
//     ||A^q|| <= T_q, T_0 = 1, T_q = ||X^q|| + ||E|| sum_{j<q} ||X^j|| T_{q-1-j};
//   - s is the smallest scaling count admissible for some p (the series stops
//     early once two consecutive terms are below the tolerance, so its cost is
//     about the number of terms until convergence, which grows with s), then m the
//     smallest degree admissible at that s; m <= 120.
#include <math.h>

#include "stencil.cuh"
#include "theta_tables.h"

// Largest norm of the Brownian part E of Omega - mu I per Taylor sub-step.  The
// deterministic part is dissipative and centred by the trace shift, so its terms
// grow only where the partial sum grows; E (Delta W A, the commutator terms) has
// oscillatory spectrum, and its terms can grow like e^{||E|| / s} while the sum
// stays bounded, so the rounding of the working precision is amplified by up to
// that factor.  s is at least ||E|| / MSK_THETA_E.  In float, 14 (about theta_55
// at the float tolerance) is where the large-step order-3 solves of the d = 200
// step-size experiment explode on exactly the paths the double solves explode on
// (without the bound, on up to 95 of 100 more); in double 24 changes no result.
#ifndef MSK_THETA_E_F32
#define MSK_THETA_E_F32 14.0
#endif
#ifndef MSK_THETA_E_F64
#define MSK_THETA_E_F64 24.0
#endif

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
  const float* pow_tab;   // ||X_n^q||, q = 1 .. MSK_POW_J, per step (pow_rows rows); null: plain norm bound
  int pow_rows;           // 1: X does not depend on the step
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

// ---- infinity norms of the powers of the deterministic part X_n ---------------
//
// X_n = V0 (x) I + V1 (x) D^x with the v-bands V0 (offsets -2..2, the shift -mu
// on the centre) and V1 (offsets -1..1) of the zero-functional weights of step n
// (no (D^x)^2 operator carries a deterministic weight).  Row (i0, j0) of X^q is
// e^T X^q, propagated as r <- r X in a window of v-rows j0 - 2q .. j0 + 2q and
// columns i0 - q .. i0 + q (zero outside the grid):
//   (r X)(i, j) = sum_o r(i, j-o) V0[j-o][o] + sum_o (r(i-1, j-o) - r(i+1, j-o)) V1[j-o][o] / (2 dx).
// Rows whose column lies J or more from both x edges never reach an edge within
// J products, so they share their row sums: one representative column per
// v-row suffices besides the J columns next to each edge.
constexpr int kPowJ = MSK_POW_J;
constexpr int kPowWV = 4 * kPowJ + 5;      // window v-rows: +-2J and a 2-row halo
constexpr int kPowWX = 2 * kPowJ + 3;      // window columns: +-J and a 1-column halo
constexpr int kPowThreads = 256;

struct PowArgs {
  OmegaArgs o;     // band, trace, D, order, steps, T, dx, c
  int nxc;         // column classes per v-row
  float* out;      // [rows][kPowJ], zeroed; maxima by atomicMax on the bit patterns
};

__device__ __forceinline__ int pow_class_col(int xc, int D) {
  if (D <= 2 * kPowJ + 1) return xc;           // every column its own class
  if (xc <= kPowJ) return xc;                  // J edge columns, then the representative column J
  return D - 1 - (xc - kPowJ - 1);
}

__global__ void __launch_bounds__(kPowThreads) power_norm_kernel(PowArgs pa) {
  const OmegaArgs& a = pa.o;
  const int D = a.D;
  const int j0 = blockIdx.x / pa.nxc, i0 = pow_class_col(blockIdx.x % pa.nxc, D);
  const int n = blockIdx.y;
  __shared__ float buf[2][kPowWV * kPowWX];
  __shared__ float V0[kPowWV][5], V1[kPowWV][3];
  __shared__ float red[kPowThreads / 32];
  const int tid = threadIdx.x;
  // zero-functional weights and shift of step n
  const double h = a.T / a.steps, tn = n * h;
  double w[MSK_NOPS], f0[MSK_NF];
  for (int k = 0; k < MSK_NF; ++k) f0[k] = 0.0;
  magnus_weights(a, tn, h, f0, w);
  double tr = 0.0;
  for (int k = 0; k < MSK_NOPS; ++k) tr += w[k] * a.trace[k];
  const double mu = tr / ((double)D * D), inv2dx = 0.5 / a.dx;
  // window row jw <-> grid row j0 - 2J - 2 + jw, window column iw <-> i0 - J - 1 + iw
  for (int jw = tid; jw < kPowWV; jw += kPowThreads) {
    const int j = j0 - 2 * kPowJ - 2 + jw;
    double v0[5] = {0, 0, 0, 0, 0}, v1[3] = {0, 0, 0};
    if (j >= 0 && j < D) {
      for (int k = 0; k < MSK_NOPS; ++k) {
        if (w[k] == 0.0) continue;
        const double* b = a.band + ((size_t)k * D + j) * MSK_BAND;
        if (c_op_xclass[k] == XC_I)
          for (int o = 0; o < 5; ++o) v0[o] += w[k] * b[o];
        else if (c_op_xclass[k] == XC_DX)
          for (int o = 0; o < 3; ++o) v1[o] += w[k] * b[o + 1];
      }
      v0[2] -= mu;
    }
    for (int o = 0; o < 5; ++o) V0[jw][o] = (float)v0[o];
    for (int o = 0; o < 3; ++o) V1[jw][o] = (float)(v1[o] * inv2dx);
  }
  for (int e = tid; e < 2 * kPowWV * kPowWX; e += kPowThreads) (&buf[0][0])[e] = 0.0f;
  __syncthreads();
  const int cj = 2 * kPowJ + 2, ci = kPowJ + 1;   // window position of (i0, j0)
  if (tid == 0) buf[0][cj * kPowWX + ci] = 1.0f;
  __syncthreads();
  int cur = 0;
  for (int q = 1; q <= kPowJ; ++q) {
    const int hv = 2 * q, hx = q, nv = 2 * hv + 1, nx = 2 * hx + 1;
    const float* src = buf[cur];
    float* dst = buf[cur ^ 1];
    float part = 0.0f;
    for (int e = tid; e < nv * nx; e += kPowThreads) {
      const int jw = cj - hv + e / nx, iw = ci - hx + e % nx;
      const int j = j0 - 2 * kPowJ - 2 + jw, i = i0 - kPowJ - 1 + iw;
      float v = 0.0f;
      if (j >= 0 && j < D && i >= 0 && i < D) {
#pragma unroll
        for (int o = -2; o <= 2; ++o) v = fmaf(src[(jw - o) * kPowWX + iw], V0[jw - o][o + 2], v);
#pragma unroll
        for (int o = -1; o <= 1; ++o)
          v = fmaf(src[(jw - o) * kPowWX + iw - 1] - src[(jw - o) * kPowWX + iw + 1], V1[jw - o][o + 1], v);
      }
      dst[jw * kPowWX + iw] = v;
      part += fabsf(v);
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      float t = 0.0f;
      for (int k = 0; k < kPowThreads / 32; ++k) t += red[k];
      atomicMax(reinterpret_cast<unsigned int*>(pa.out) + (size_t)n * kPowJ + q - 1, __float_as_uint(t));
    }
    cur ^= 1;
    __syncthreads();
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
  // norm (or bound) of the Brownian part E of Omega - mu I: the operators whose weights
  // vanish when every functional is zero
  double wd[MSK_NOPS], f0[MSK_NF];
  for (int k = 0; k < MSK_NF; ++k) f0[k] = 0.0;
  magnus_weights(a, tn, h, f0, wd);
  double eps = 0.0;
  if (a.var && a.var_ops == MSK_NOPS) {
    for (int k = 0; k < MSK_NOPS; ++k) eps += fabs(w[k] - wd[k]) * a.var[MSK_NOPS + k];
  } else if (a.var) {
    const int map6[6] = {MSK_OP_BX, MSK_OP_A0, MSK_OP_A0A0, MSK_OP_BX_A0, MSK_OP_BXA0_A0, MSK_OP_BXA0_BX};
    for (int k = 0; k < 6; ++k) eps += fabs(w[map6[k]] - wd[map6[k]]) * a.var[6 + k];
  }
  const double* ith = a.precision == MSK_F32 ? c_inv_theta32 : c_inv_theta64;
  const int mmax = a.precision == MSK_F32 ? MSK_THETA_MMAX_F32 : MSK_THETA_MMAX_F64;
  // d[q] >= ||(Omega - mu I)^q||^(1/q): d[1] the exact norm, d[2..J] from the
  // deterministic power norms (when available) and the norm of the Brownian part
  double dq[MSK_POW_J + 1];
  for (int q = 0; q <= MSK_POW_J; ++q) dq[q] = nrm;
  if (!a.var) {
    // Langevin operators: E = Omega - mu I - X exactly, X the zero-functional part with its
    // own shift (the infinity norm of its folded stencil)
    double we[MSK_NOPS], trd = 0.0;
    for (int k = 0; k < MSK_NOPS; ++k) {
      trd += wd[k] * a.trace[k];
      we[k] = w[k] - wd[k];
    }
    const double dmu = mu - trd / ((double)D * D);
    const int rows[6] = {0, 1, 2, D - 3, D - 2, D - 1};
    for (int r = 0; r < 6; ++r) {
      double c[MSK_NCOEF];
      fold_row(a.band, D, rows[r], we, -dmu, 0.5 / a.dx, 0.25 / (a.dx * a.dx), c);
      eps = fmax(eps, row_abs_sum(c));
    }
  }
  if (a.pow_tab && nrm > 0.0) {
    const int row = a.pow_rows == 1 ? 0 : (int)(idx % a.steps);
    const float* g = a.pow_tab + (size_t)row * MSK_POW_J;
    // the float table carries relative rounding far below 1e-4 (unit rows, at most
    // nine stencil products): inflate it by 2^-10 so it stays an upper bound
    double gx[MSK_POW_J + 1], Tq[MSK_POW_J + 1];
    gx[0] = 1.0;
    Tq[0] = 1.0;
    for (int q = 1; q <= MSK_POW_J; ++q) {
      gx[q] = (double)g[q - 1] * (1.0 + 0x1p-10);
      double t = gx[q];
      for (int j = 0; j < q; ++j) t += eps * gx[j] * Tq[q - 1 - j];
      Tq[q] = t;
      if (q >= 2) dq[q] = fmin(nrm, exp(log(t) / q));
    }
  }
  double best_s = 1.0, best_m = 0.0, amin = nrm, used = nrm;
  if (nrm > 0.0) {
    // alpha_p for p = 2 .. J - 1, usable at degree m when p (p - 1) <= m + 1
    double alpha[MSK_POW_J];
    alpha[1] = nrm;
    for (int p = 2; p < MSK_POW_J; ++p) alpha[p] = fmax(dq[p], dq[p + 1]);
    for (int p = 2; p < MSK_POW_J; ++p)
      if (p * (p - 1) <= mmax + 1) amin = fmin(amin, alpha[p]);
    best_s = fmax(1.0, ceil(amin * ith[mmax - 1]));
    best_s = fmax(best_s, ceil(eps / (a.precision == MSK_F32 ? MSK_THETA_E_F32 : MSK_THETA_E_F64)));
    if (!(best_s <= a.s_cap)) {   // also catches a non-finite norm
      best_s = a.s_cap;
      best_m = mmax;
      used = amin;
    } else {
      best_m = mmax;
      for (int m = 1; m <= mmax; ++m) {
        double am = nrm;
        for (int p = 2; p < MSK_POW_J && p * (p - 1) <= m + 1; ++p) am = fmin(am, alpha[p]);
        if (am * ith[m - 1] <= best_s) {
          best_m = m;
          used = am;
          break;
        }
      }
    }
  }
  double* o = Wt + idx * MSK_NWT;
  for (int k = 0; k < MSK_NOPS; ++k) o[k] = w[k];
  for (int k = MSK_NOPS; k < MSK_WT_MU; ++k) o[k] = 0.0;
  o[MSK_WT_ALPHA] = used;
  o[MSK_WT_EPS] = eps;
  // expected Taylor terms: per sub-step about x + sqrt(2 x ln(1/tol)) with x = alpha / s
  // (the terms x^k / k! fall below the tolerance), capped by the degree
  if (nrm > 0.0) {
    const double x = used / best_s, L = a.precision == MSK_F32 ? 13.9 : 36.7;
    o[MSK_WT_WORK] = best_s * fmin(best_m, ceil(x + sqrt(2.0 * x * L)) + 1.0);
  }
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

int power_norm_rows(const msk_ctx* ctx, int steps) {
  if (ctx->xprof || ctx->gen) return 0;      // those engines bound the norm over their operators
  // Steps so short that the plain norm already allows one sub-step gain nothing from the
  // power norms (the degree only caps an early-terminating series): an upper estimate
  // of ||h B|| + ||A^2 term|| against half of the smaller theta_120 (double) skips them.
  const double h = ctx->T / steps;
  const double vmax = fmax(fabs(ctx->av), fabs(ctx->bv));
  const double amax = fabs(ctx->coef.a0) + fabs(ctx->coef.kind == MSK_COEF_TRIG ? ctx->coef.a1 : 0.0);
  const double smax = fabs(ctx->coef.s0) * (1.0 + fabs(ctx->coef.kind == MSK_COEF_TRIG ? ctx->coef.s1 : 0.0));
  const double est = h * (vmax / ctx->dx + (amax + smax * smax) * 2.0 / (ctx->dv * ctx->dv));
  if (est < 0.5 * msk_theta_f64[MSK_THETA_MMAX_F64 - 1]) return 0;
  return ctx->coef.kind == MSK_COEF_CONST ? 1 : steps;
}

msk_status launch_power_norms(msk_ctx* ctx, int order, int steps, float* pow_tab, cudaStream_t stream) {
  const int rows = power_norm_rows(ctx, steps);
  if (rows == 0) return MSK_OK;
  msk_status st = msk_cuda(ctx, cudaMemsetAsync(pow_tab, 0, (size_t)rows * MSK_POW_J * sizeof(float), stream),
                           "power norm reset");
  if (st != MSK_OK) return st;
  PowArgs pa{};
  pa.o = OmegaArgs{ctx->band, ctx->aux, nullptr, 0, nullptr, nullptr, 0, ctx->d, order, steps, MSK_F64, 0,
                   ctx->T, ctx->dx, omega_coef(ctx), kMskScaleCap};
  pa.nxc = ctx->d <= 2 * kPowJ + 1 ? ctx->d : 2 * kPowJ + 1;
  pa.out = pow_tab;
  power_norm_kernel<<<dim3((unsigned)(ctx->d * pa.nxc), (unsigned)rows), kPowThreads, 0, stream>>>(pa);
  return msk_cuda(ctx, cudaGetLastError(), "power norm kernel");
}

// The context's cached table for (steps, order >= 2); recomputed when the
// operators, coefficients or time grid changed since it was built.
static msk_status ensure_power_norms(msk_ctx* ctx, int order, int steps, cudaStream_t stream, const float** out) {
  *out = nullptr;
  const int rows = power_norm_rows(ctx, steps);
  if (rows == 0) return MSK_OK;
  const int o2 = order >= 2;
  if (ctx->pow_tab && ctx->pow_gen == ctx->setup_gen && ctx->pow_steps == steps && ctx->pow_o2 == o2) {
    *out = ctx->pow_tab;
    return MSK_OK;
  }
  const int64_t need = (int64_t)rows * MSK_POW_J;
  if (need > ctx->pow_cap) {
    if (ctx->pow_tab) cudaFree(ctx->pow_tab);   // waits for work that may still read it
    ctx->pow_tab = nullptr;
    ctx->pow_cap = 0;
    msk_status st = msk_cuda(ctx, cudaMalloc(&ctx->pow_tab, need * sizeof(float)), "power norm table");
    if (st != MSK_OK) return st;
    ctx->pow_cap = need;
  }
  msk_status st = launch_power_norms(ctx, order, steps, ctx->pow_tab, stream);
  if (st != MSK_OK) return st;
  ctx->pow_gen = ctx->setup_gen;
  ctx->pow_steps = steps;
  ctx->pow_o2 = o2;
  *out = ctx->pow_tab;
  return MSK_OK;
}

msk_status launch_omega_tab(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                            const double* F, double* Wt, const float* pow_tab, cudaStream_t stream) {
  msk_status st0 = msk_prepare_omega(ctx);
  if (st0 != MSK_OK) return st0;
  const int64_t n = paths * steps;
  if (n == 0) return MSK_OK;
  if (ctx->xprof || ctx->gen) {
    st0 = ensure_var_tables(ctx, stream);
    if (st0 != MSK_OK) return st0;
  }
  const int rows = power_norm_rows(ctx, steps);
  OmegaArgs a{ctx->band, ctx->aux, (ctx->xprof || ctx->gen) ? ctx->var_tab : nullptr, var_table_ops(ctx), nullptr,
              rows ? pow_tab : nullptr, rows, ctx->d, order, steps, precision, paths, ctx->T, ctx->dx,
              omega_coef(ctx), kMskScaleCap};
  omega_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(a, F, Wt);
  return msk_cuda(ctx, cudaGetLastError(), "omega kernel");
}

msk_status launch_omega(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                        const double* F, double* Wt, cudaStream_t stream) {
  if (paths * steps == 0) return MSK_OK;
  const float* tab = nullptr;
  msk_status st = ensure_power_norms(ctx, order, steps, stream, &tab);
  if (st != MSK_OK) return st;
  return launch_omega_tab(ctx, order, steps, paths, precision, F, Wt, tab, stream);
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
              job_th_dev, nullptr, 0, ctx->d, order, 1, precision, njobs, ctx->T, ctx->dx, omega_coef(ctx),
              kMskScaleCap};
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

extern "C" msk_status msk_power_norms(msk_ctx* ctx, int order, int steps, float* out_dev, int* rows_out,
                                      void* stream) {
  if (!ctx || !rows_out) return MSK_ERR_ARG;
  if (order < 1 || order > 3) return msk_fail(ctx, MSK_ERR_ARG, "order must be 1, 2 or 3");
  if (steps < 1 || ctx->n_fine % steps != 0)
    return msk_fail(ctx, MSK_ERR_ARG, "steps must be >= 1 and divide n_fine");
  *rows_out = power_norm_rows(ctx, steps);
  if (*rows_out == 0 || !out_dev) return MSK_OK;   // null output: the row count only
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  return launch_power_norms(ctx, order, steps, out_dev, (cudaStream_t)stream);
}

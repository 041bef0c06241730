// Widened-stencil form of the Magnus logarithm.
//
// Every basis operator of the Langevin problem is one Kronecker product
// V (x) X with V a banded n_v x n_v matrix (bandwidth <= 2) and X one of
// I, D^x, (D^x)^2 (Section 2: x derivatives act from the left on the x index,
// v derivatives on the v index, and the commutators of Eq. MagnusFormulas
// multiply the factors separately).  Hence
//     Omega = V0 (x) I + V1 (x) D^x + V2 (x) (D^x)^2,   V_c = sum_{k in class c} w_k V_k,
// and one application at grid point (i, j) reads
//     sum_o V0[j][o] u(i, j+o)                              o = -2..2
//   + sum_o V1[j][o] (u(i+1, j+o) - u(i-1, j+o)) / (2 dx)   o = -1..1
//   + sum_o V2[j][o] ((D^x)^2 u(., j+o))(i)                 o = -1, +1
// with zero padding outside the grid, where the truncated (D^x)^2 =
// tridiag(-1,0,1)^2 / (4 dx^2) has centre -2 in the interior but -1 in its
// first and last rows (only one neighbour contributes).  Folding the centre of
// (D^x)^2 into the V0 coefficients gives twelve numbers per v-row:
//     A[0..4]  = V0[-2..2] - 2 V2[o]/(4dx^2) (o = +-1) + shift (o = 0)
//     Bc[0..2] = V1[-1..1] / (2 dx)
//     Cc[0..1] = V2[-1], V2[+1] / (4 dx^2)
//     Ae[0..1] = A[-1] + Cc[-1], A[+1] + Cc[+1]    (x-edge columns i = 0, n_x - 1)
// These are exact for the truncated matrices, including the boundary rows.
#pragma once

#include "msk_internal.cuh"

#define MSK_NCOEF 12
enum { CF_A = 0, CF_B = 5, CF_C = 8, CF_AE = 10 };

__constant__ int c_op_xclass[MSK_NOPS] = {XC_DX, XC_I,  XC_I,  XC_I,  XC_DX, XC_I, XC_DX,
                                          XC_DX, XC_I,  XC_DXX, XC_DX, XC_DX, XC_I};

// Fold the weighted basis tables of v-row j into the twelve stencil coefficients.
__device__ __forceinline__ void fold_row(const double* __restrict__ band, int D, int j,
                                         const double* w, double shift, double inv2dx,
                                         double inv4dx2, double out[MSK_NCOEF]) {
  double V0[MSK_BAND] = {0, 0, 0, 0, 0}, V1[MSK_BAND] = {0, 0, 0, 0, 0},
         V2[MSK_BAND] = {0, 0, 0, 0, 0};
  for (int k = 0; k < MSK_NOPS; ++k) {
    const double wk = w[k];
    if (wk == 0.0) continue;
    const double* b = band + ((size_t)k * D + j) * MSK_BAND;
    const int xc = c_op_xclass[k];
#pragma unroll
    for (int o = 0; o < MSK_BAND; ++o) {
      const double v = wk * b[o];
      if (xc == XC_I) V0[o] += v;
      else if (xc == XC_DX) V1[o] += v;
      else V2[o] += v;
    }
  }
#pragma unroll
  for (int o = 0; o < 5; ++o) out[CF_A + o] = V0[o];
  out[CF_A + 1] -= 2.0 * V2[1] * inv4dx2;
  out[CF_A + 3] -= 2.0 * V2[3] * inv4dx2;
  out[CF_A + 2] += shift;
#pragma unroll
  for (int o = 0; o < 3; ++o) out[CF_B + o] = V1[o + 1] * inv2dx;
  out[CF_C + 0] = V2[1] * inv4dx2;
  out[CF_C + 1] = V2[3] * inv4dx2;
  out[CF_AE + 0] = out[CF_A + 1] + out[CF_C + 0];
  out[CF_AE + 1] = out[CF_A + 3] + out[CF_C + 1];
}

// Only V1's centre varies across interior rows (Bx = kappa diag(v) (x) D^x).
__device__ __forceinline__ double fold_b0(const double* __restrict__ band, int D, int j,
                                          const double* w, double inv2dx) {
  double v = 0.0;
  for (int k = 0; k < MSK_NOPS; ++k) {
    if (c_op_xclass[k] != XC_DX || w[k] == 0.0) continue;
    v += w[k] * band[((size_t)k * D + j) * MSK_BAND + 2];
  }
  return v * inv2dx;
}

// Rows whose coefficients differ from the interior pattern: the boundary
// corrections of the truncated-matrix products reach two rows into the grid.
__host__ __device__ __forceinline__ bool is_special_row(int j, int D) { return j < 2 || j >= D - 2; }
__host__ __device__ __forceinline__ int special_index(int j, int D) { return j < 2 ? j : j - (D - 2) + 2; }
__host__ __device__ __forceinline__ int special_row(int idx, int D) { return idx < 2 ? idx : D - 2 + (idx - 2); }

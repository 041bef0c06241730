// Device kernels of the learned surrogate: Brownian features, the BF16 MLP
// (tensor-core GEMMs with fused epilogues, loss, Adam), the randomized POD
// and the decode / audit kernels.
#pragma once

#include <cuda_bf16.h>

#include "msk_internal.cuh"
#include "philox.cuh"

namespace sgk {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ features
// Standard normals of fine cells 2j, 2j+1 in single precision: the same Philox
// words as the double-precision generator (stream tag 0), uniforms
// (hi + 1/2) 2^-32 from the high word of each pair, Box-Muller.
__device__ __forceinline__ void normal_pair_f32(uint64_t seed, uint64_t path, uint64_t j, float& z0, float& z1) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)path, (uint32_t)(path >> 32), 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float u1 = fmaf((float)w.y, 0x1p-32f, 0x1p-33f);
  const float u2 = fmaf((float)w.w, 0x1p-32f, 0x1p-33f);
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per (path, step).  With m = n_fine / K fine cells of width delta in
// the step, dw_i = sqrt(delta) z_i, the features are
//   dW / sqrt(h)          = A / sqrt(m)
//   int W ds / s3         = sqrt(3) (m A - B) / m^1.5
//   int s dW / s3         = sqrt(3) B / m^1.5
// with A = sum z_i, B = sum (i + 1/2) z_i (piecewise-linear W in each cell),
// h = m delta, s3 = h^1.5 / sqrt(3).  Output bf16 [paths][K][3].
__global__ void __launch_bounds__(256) features_kernel(uint64_t seed, uint64_t first, uint64_t stride,
                                                       int64_t paths, int K, int64_t n_fine, bf16* __restrict__ X) {
  const int lane = threadIdx.x & 31;
  const int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (idx >= paths * K) return;                       // whole warp leaves together
  const int64_t p = idx / K;
  const int k = (int)(idx % K);
  const uint64_t gpath = first + (uint64_t)p * stride;
  const int64_t m = n_fine / K, c0 = (int64_t)k * m, c1 = c0 + m;
  float A = 0.f, B = 0.f;
  for (int64_t j = (c0 >> 1) + lane; 2 * j < c1; j += 32) {
    float z0, z1;
    normal_pair_f32(seed, gpath, (uint64_t)j, z0, z1);
    const int64_t a = 2 * j;
    if (a >= c0) {
      A += z0;
      B = fmaf(z0, (float)(a - c0) + 0.5f, B);
    }
    if (a + 1 < c1) {
      A += z1;
      B = fmaf(z1, (float)(a + 1 - c0) + 0.5f, B);
    }
  }
  A = warp_sum_f(A);
  B = warp_sum_f(B);
  if (lane == 0) {
    const float mf = (float)m, rs = rsqrtf(mf), c3 = 1.7320508075688772f * rs / mf;
    bf16* x = X + idx * 3;
    x[0] = __float2bfloat16(A * rs);
    x[1] = __float2bfloat16(fmaf(mf, A, -B) * c3);
    x[2] = __float2bfloat16(B * c3);
  }
}

// ------------------------------------------------------------------ GELU
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

// ------------------------------------------------------------------ BF16 GEMM (mma.sync)
// C[M][N] = sum_k A(m, k) B(n, k): bf16 operands, fp32 accumulation.
// A_KC: A stored [M][K] (row stride lda), else [K][M]; B_KC: B stored [N][K], else [K][N].
// Shared-memory tiles keep the global layout; ldmatrix (.trans for the [K][.]
// layouts) builds the m16n8k16 fragments.
enum { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_GELU = 2, EPI_GELU_BWD = 3 };

struct GemmArgs {
  const bf16* A;
  const bf16* B;
  int M, N, K, lda, ldb;
  int kchunk;             // K range per blockIdx.z (multiple of 32)
  int vecA, vecB;         // 16-byte loads allowed (aligned base, ld % 8 == 0)
  float* C;               // fp32 output; EPI_F32 with split-K: C + z * split_stride
  int ldc;
  int64_t split_stride;
  bf16* C16;              // bf16 output (EPI_BIAS_GELU: GELU(z); EPI_GELU_BWD: dz)
  int ldc16;
  const float* bias;      // [N]
  const float* aux;       // EPI_GELU_BWD: pre-activation z [M][ldaux]
  int ldaux;
};

constexpr int GBM = 128, GBN = 64, GBK = 32;
constexpr int KC_LD = GBK + 8;            // [rows][k] tiles: 80-byte rows
constexpr int A_T_LD = GBM + 8;           // [k][m] tile: 272-byte rows
constexpr int B_T_LD = GBN + 8;           // [k][n] tile: 144-byte rows

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <bool TRANS>
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16* p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  if (TRANS)
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
  else
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}

// Copy the (ROWS x GBK) tile at (r0, k0) of an operand into shared memory in
// its own layout: KC -> sm[ROWS][KC_LD] (k fastest), else sm[GBK][ROWS + 8]
// (rows fastest).  Elements outside [0, rows) x [k0, k1) are zero.
template <int ROWS, bool KC>
__device__ __forceinline__ void fill_tile(bf16* sm, const bf16* __restrict__ G, int ld, int rows, int r0, int k0,
                                          int k1, bool vec, int tid) {
  constexpr int CH = KC ? ROWS * (GBK / 8) : GBK * (ROWS / 8);   // 16-byte chunks
  const bf16 zero = __float2bfloat16(0.f);
  for (int c = tid; c < CH; c += 256) {
    int rr, kk;
    if (KC) {
      rr = c / (GBK / 8);
      kk = (c % (GBK / 8)) * 8;
    } else {
      kk = c / (ROWS / 8);
      rr = (c % (ROWS / 8)) * 8;
    }
    const int gr = r0 + rr, gk = k0 + kk;
    bf16* dst = KC ? sm + rr * KC_LD + kk : sm + kk * (ROWS + 8) + rr;
    const bool full = KC ? (gr < rows && gk + 8 <= k1) : (gk < k1 && gr + 8 <= rows);
    if (vec && full) {
      const bf16* src = KC ? G + (size_t)gr * ld + gk : G + (size_t)gk * ld + gr;
      *reinterpret_cast<uint4*>(dst) = __ldg(reinterpret_cast<const uint4*>(src));
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int r = KC ? gr : gr + e, k = KC ? gk + e : gk;
        dst[e] = (r < rows && k < k1) ? (KC ? G[(size_t)r * ld + k] : G[(size_t)k * ld + r]) : zero;
      }
    }
  }
}

template <bool A_KC, bool B_KC, int EPI>
__global__ void __launch_bounds__(256) gemm_bf16_kernel(const GemmArgs g) {
  constexpr int A_ELEMS = A_KC ? GBM * KC_LD : GBK * A_T_LD;
  constexpr int B_ELEMS = B_KC ? GBN * KC_LD : GBK * B_T_LD;
  __shared__ __align__(128) bf16 As[A_ELEMS];
  __shared__ __align__(128) bf16 Bs[B_ELEMS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp & 3, wn = warp >> 2;     // 4 x 2 warps, 32 x 32 outputs per warp
  const int gid = lane >> 2, tig = lane & 3;
  const int mi = lane >> 3, rr = lane & 7;     // ldmatrix: matrix and row served by this lane
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int kbeg = blockIdx.z * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
    fill_tile<GBM, A_KC>(As, g.A, g.lda, g.M, m0, k0, kend, g.vecA, tid);
    fill_tile<GBN, B_KC>(Bs, g.B, g.ldb, g.N, n0, k0, kend, g.vecB, tid);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t a[2][4], b[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        // matrices: (m 0-7, k 0-7), (m 8-15, k 0-7), (m 0-7, k 8-15), (m 8-15, k 8-15)
        const int mo = wm * 32 + i * 16 + (mi & 1) * 8, ko = kk + (mi >> 1) * 8;
        if (A_KC) ldsm_x4<false>(a[i], As + (mo + rr) * KC_LD + ko);
        else ldsm_x4<true>(a[i], As + (ko + rr) * A_T_LD + mo);
      }
#pragma unroll
      for (int jp = 0; jp < 2; ++jp) {
        // matrices: (n-tile 2jp, k 0-7), (2jp, k 8-15), (2jp+1, k 0-7), (2jp+1, k 8-15)
        const int no = wn * 32 + jp * 16 + (mi >> 1) * 8, ko = kk + (mi & 1) * 8;
        if (B_KC) ldsm_x4<false>(b[jp], Bs + (no + rr) * KC_LD + ko);
        else ldsm_x4<true>(b[jp], Bs + (ko + rr) * B_T_LD + no);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j >> 1][(j & 1) * 2], b[j >> 1][(j & 1) * 2 + 1]);
    }
    __syncthreads();
  }
  float* Cz = (EPI == EPI_F32) ? g.C + (size_t)blockIdx.z * g.split_stride : g.C;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = m0 + wm * 32 + i * 16 + gid + (q >= 2 ? 8 : 0);
        const int c = n0 + wn * 32 + j * 8 + tig * 2 + (q & 1);
        if (r >= g.M || c >= g.N) continue;
        float v = acc[i][j][q];
        if (EPI == EPI_F32) {
          Cz[(size_t)r * g.ldc + c] = v;
        } else if (EPI == EPI_BIAS_F32) {
          g.C[(size_t)r * g.ldc + c] = v + g.bias[c];
        } else if (EPI == EPI_BIAS_GELU) {
          v += g.bias[c];
          if (g.C) g.C[(size_t)r * g.ldc + c] = v;
          g.C16[(size_t)r * g.ldc16 + c] = __float2bfloat16(gelu(v));
        } else {
          const float dz = v * gelu_prime(g.aux[(size_t)r * g.ldaux + c]);
          g.C[(size_t)r * g.ldc + c] = dz;
          g.C16[(size_t)r * g.ldc16 + c] = __float2bfloat16(dz);
        }
      }
}

// out[i] = sum_z ws[z][i] (split-K reduction, fixed order).
__global__ void reduce_splits_kernel(const float* __restrict__ ws, int splits, int64_t n, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += ws[(size_t)z * n + i];
  out[i] = s;
}

// ------------------------------------------------------------------ loss, bias gradients, Adam
__device__ __forceinline__ double block_sum_d(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  const double s = red[0];
  __syncthreads();
  return s;
}

// g = 2 (out - target) / B as fp32 and bf16; per-block partial sums of (out - target)^2.
__global__ void __launch_bounds__(256) loss_grad_kernel(const float* __restrict__ out, const float* __restrict__ target,
                                                        int64_t n, float inv_b, float* __restrict__ g,
                                                        bf16* __restrict__ g16, double* __restrict__ partial) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float d = out[e] - target[e];
    s += (double)d * d;
    const float gv = 2.0f * d * inv_b;
    if (g) g[e] = gv;
    if (g16) g16[e] = __float2bfloat16(gv);
  }
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) loss_final_kernel(const double* __restrict__ partial, int n, double inv_b,
                                                         float* __restrict__ loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) *loss = (float)(s * inv_b);
}

// db[c] = sum_r g[r][c]: 32 columns per block, 8 row lanes, fixed order.
__global__ void colsum_kernel(const float* __restrict__ g, int rows, int cols, float* __restrict__ db) {
  __shared__ float red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float s = 0.f;
  if (c < cols)
    for (int r = threadIdx.y; r < rows; r += 8) s += g[(size_t)r * cols + c];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
    db[c] = t;
  }
}

// One Adam step on the flat parameter vector; refreshes its bf16 copy.
__global__ void adam_kernel(float* __restrict__ w, bf16* __restrict__ w16, const float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gr = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gr;
  const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  w16[i] = __float2bfloat16(wi);
}

__global__ void to_bf16_kernel(const float* __restrict__ x, bf16* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
}

// He initialisation of one weight block: w = N(0, 2 / fan_in) from Philox
// (stream tag 4, counter offset base), double-precision Box-Muller.
__global__ void init_weights_kernel(float* __restrict__ w, int64_t n, int64_t fan_in, uint64_t seed, uint64_t base) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double z0, z1;
  brownian_pair(seed, base + (uint64_t)(i >> 1), 4u, 0, z0, z1);
  w[i] = (float)(((i & 1) ? z1 : z0) * sqrt(2.0 / (double)fan_in));
}

// ------------------------------------------------------------------ POD
// Column sums of S (N x n) per chunk of rows, in double.
__global__ void colsum_partial_kernel(const float* __restrict__ S, int64_t N, int n, int64_t rows_per_chunk,
                                      double* __restrict__ partial) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk, r1 = min(N, r0 + rows_per_chunk);
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) s += S[r * n + f];
  partial[(size_t)blockIdx.y * n + f] = s;
}

__global__ void colmean_final_kernel(const double* __restrict__ partial, int chunks, int n, int64_t N,
                                     float* __restrict__ mean) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += partial[(size_t)c * n + f];
  mean[f] = (float)(s / (double)N);
}

// Gaussian test matrix G [N][Q] (Philox stream tag 3, double Box-Muller).
__global__ void gaussian_kernel(float* __restrict__ G, int64_t count, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double z0, z1;
  brownian_pair(seed, (uint64_t)(i >> 1), 3u, 0, z0, z1);
  G[i] = (float)((i & 1) ? z1 : z0);
}

// Sketch: Yt[z][q][f] = sum_{rows n of chunk z} G[n][q] (S[n][f] - mean[f]),  q < Q <= 80.
// Block: 128 columns x one row chunk, 256 threads (32 columns x 8 q-lanes).
constexpr int SK_Q = 80, SK_F = 128, SK_R = 32;
__global__ void __launch_bounds__(256) sketch_kernel(const float* __restrict__ S, const float* __restrict__ mean,
                                                     const float* __restrict__ G, int64_t N, int n, int Q,
                                                     int64_t rows_per_chunk, float* __restrict__ Yt) {
  __shared__ float Gs[SK_R][SK_Q];
  __shared__ float Ss[SK_R][SK_F];
  const int tid = threadIdx.x;
  const int f0 = blockIdx.x * SK_F;
  const int tf = tid & 31, tq = tid >> 5;   // columns f0 + tf + 32 c (c < 4); rows q = tq + 8 k (k < 10)
  const int64_t rbeg = (int64_t)blockIdx.y * rows_per_chunk, rend = min(N, rbeg + rows_per_chunk);
  float acc[10][4];
#pragma unroll
  for (int k = 0; k < 10; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[k][c] = 0.f;
  for (int64_t r0 = rbeg; r0 < rend; r0 += SK_R) {
    for (int e = tid; e < SK_R * SK_Q; e += 256) {
      const int r = e / SK_Q, q = e % SK_Q;
      Gs[r][q] = (r0 + r < rend && q < Q) ? G[(r0 + r) * Q + q] : 0.f;
    }
    for (int e = tid; e < SK_R * SK_F; e += 256) {
      const int r = e / SK_F, ff = e % SK_F, f = f0 + ff;
      Ss[r][ff] = (r0 + r < rend && f < n) ? S[(r0 + r) * n + f] - mean[f] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < SK_R; ++r) {
      float s[4], gq[10];
#pragma unroll
      for (int c = 0; c < 4; ++c) s[c] = Ss[r][tf + 32 * c];
#pragma unroll
      for (int k = 0; k < 10; ++k) gq[k] = Gs[r][tq + 8 * k];
#pragma unroll
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[k][c] = fmaf(gq[k], s[c], acc[k][c]);
    }
    __syncthreads();
  }
  float* Y = Yt + (size_t)blockIdx.y * Q * n;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const int q = tq + 8 * k;
    if (q >= Q) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int f = f0 + tf + 32 * c;
      if (f < n) Y[(size_t)q * n + f] = acc[k][c];
    }
  }
}

// Out[r][i] = sum_f (S[r][f] - mean[f]) Bm[i][f],  i < I <= 80.  Block: 32 rows x all I.
constexpr int PR_R = 32, PR_I = 80, PR_F = 64;
__global__ void __launch_bounds__(256) rows_dot_kernel(const float* __restrict__ S, const float* __restrict__ mean,
                                                       int64_t N, int n, const float* __restrict__ Bm, int I,
                                                       float* __restrict__ Out) {
  __shared__ float Ss[PR_R][PR_F + 1];
  __shared__ float Bs[PR_I][PR_F + 1];
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * PR_R;
  const int tr = tid & 31, ti = tid >> 5;   // row r0 + tr, outputs i = ti + 8 k (k < 10)
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
  for (int f0 = 0; f0 < n; f0 += PR_F) {
    for (int e = tid; e < PR_R * PR_F; e += 256) {
      const int r = e / PR_F, ff = e % PR_F, f = f0 + ff;
      Ss[r][ff] = (r0 + r < N && f < n) ? S[(r0 + r) * n + f] - mean[f] : 0.f;
    }
    for (int e = tid; e < PR_I * PR_F; e += 256) {
      const int ii = e / PR_F, ff = e % PR_F, f = f0 + ff;
      Bs[ii][ff] = (ii < I && f < n) ? Bm[(size_t)ii * n + f] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int ff = 0; ff < PR_F; ++ff) {
      const float sv = Ss[tr][ff];
#pragma unroll
      for (int k = 0; k < 10; ++k) acc[k] = fmaf(sv, Bs[ti + 8 * k][ff], acc[k]);
    }
    __syncthreads();
  }
  if (r0 + tr < N)
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const int i = ti + 8 * k;
      if (i < I) Out[(r0 + tr) * I + i] = acc[k];
    }
}

// Gram of the rows of Y (Q x n): Gm[i][j] = sum_f Y[i][f] Y[j][f] in double; one block per pair i >= j.
__global__ void __launch_bounds__(256) gram_rows_kernel(const float* __restrict__ Y, int Q, int n,
                                                        double* __restrict__ Gm) {
  const int i = blockIdx.x, j = blockIdx.y;
  if (j > i) return;   // whole block leaves together
  __shared__ double red[256];
  double s = 0.0;
  for (int f = threadIdx.x; f < n; f += blockDim.x) s += (double)Y[(size_t)i * n + f] * (double)Y[(size_t)j * n + f];
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) Gm[i * Q + j] = Gm[j * Q + i] = s;
}

// Partial Gram of the columns of Z (N x Q), one chunk of rows per block:
// float sums over 32-row slabs, double across slabs.  part[block][Q][Q].
constexpr int GC_R = 32;
constexpr int GC_PAIRS = (SK_Q * SK_Q + 255) / 256;   // 25 (i, j) pairs per thread
__global__ void __launch_bounds__(256) gram_cols_partial_kernel(const float* __restrict__ Z, int64_t N, int Q,
                                                                int64_t rows_per_block, double* __restrict__ part) {
  __shared__ float Zs[GC_R][SK_Q + 1];
  double acc[GC_PAIRS];
  float slab[GC_PAIRS];
#pragma unroll
  for (int t = 0; t < GC_PAIRS; ++t) acc[t] = 0.0;
  const int64_t rbeg = (int64_t)blockIdx.x * rows_per_block, rend = min(N, rbeg + rows_per_block);
  for (int64_t r0 = rbeg; r0 < rend; r0 += GC_R) {
    for (int e = threadIdx.x; e < GC_R * SK_Q; e += 256) {
      const int r = e / SK_Q, q = e % SK_Q;
      Zs[r][q] = (r0 + r < rend && q < Q) ? Z[(r0 + r) * Q + q] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < GC_PAIRS; ++t) slab[t] = 0.f;
    for (int r = 0; r < GC_R; ++r) {
#pragma unroll
      for (int t = 0; t < GC_PAIRS; ++t) {
        const int pidx = threadIdx.x + 256 * t;
        if (pidx < SK_Q * SK_Q) slab[t] = fmaf(Zs[r][pidx / SK_Q], Zs[r][pidx % SK_Q], slab[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < GC_PAIRS; ++t) acc[t] += (double)slab[t];
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < GC_PAIRS; ++t) {
    const int pidx = threadIdx.x + 256 * t;
    if (pidx >= SK_Q * SK_Q) continue;
    const int i = pidx / SK_Q, j = pidx % SK_Q;
    if (i < Q && j < Q) part[(size_t)blockIdx.x * Q * Q + i * Q + j] = acc[t];
  }
}

__global__ void sum_partials_d_kernel(const double* __restrict__ part, int parts, int64_t n, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int p = 0; p < parts; ++p) s += part[(size_t)p * n + i];
  out[i] = s;
}

// Symmetric eigendecomposition of a Q x Q matrix (Q <= 80) by cyclic Jacobi
// rotations in one block (Golub & Van Loan, "Matrix Computations", Sec. 8.5),
// followed by the post-processing the POD needs:
//   mode 0 (orthonormalise): kept = #{lambda_i > rel_keep lambda_max};
//           Mout[i][:] = w_i^T / sqrt(lambda_i), i < kept (descending lambda)
//   mode 1 (POD):            kept = min(r, #{lambda_i > rel_keep lambda_max});
//           Mout[i][:] = w_i^T, sv[i] = sqrt(max(lambda_i, 0)) for all i
// Dynamic shared memory: 2 Q^2 doubles + Q ints.
__global__ void __launch_bounds__(128) sym_eig_kernel(const double* __restrict__ Ain, int Q, int mode,
                                                      double rel_keep, int r, double* __restrict__ Mout,
                                                      int* __restrict__ kept_out, double* __restrict__ sv) {
  extern __shared__ double esm[];
  double* A = esm;
  double* V = esm + Q * Q;
  int* order = reinterpret_cast<int*>(V + Q * Q);
  __shared__ double red[128];
  __shared__ int s_kept;
  const int t = threadIdx.x;
  for (int e = t; e < Q * Q; e += blockDim.x) {
    A[e] = Ain[e];
    V[e] = (e / Q == e % Q) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int e = t; e < Q * Q; e += blockDim.x) {
      const double a = A[e];
      if (e / Q == e % Q) dia += a * a;
      else off += a * a;
    }
    off = block_sum_d(off, red);
    dia = block_sum_d(dia, red);
    if (off <= 1e-30 * dia || off == 0.0) break;   // same decision in all threads
    for (int p = 0; p < Q - 1; ++p)
      for (int q = p + 1; q < Q; ++q) {
        const double apq = A[p * Q + q];
        const double app = A[p * Q + p], aqq = A[q * Q + q];
        // skip negligible entries (same decision in all threads: all read the same values)
        if (fabs(apq) <= 1e-300 || fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq))) continue;
        const double theta = (aqq - app) / (2.0 * apq);
        const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
        __syncthreads();   // every thread has read A[p][q], A[p][p], A[q][q]
        for (int k = t; k < Q; k += blockDim.x) {   // A <- A J, V <- V J (columns p, q)
          const double akp = A[k * Q + p], akq = A[k * Q + q];
          A[k * Q + p] = c * akp - s * akq;
          A[k * Q + q] = s * akp + c * akq;
          const double vkp = V[k * Q + p], vkq = V[k * Q + q];
          V[k * Q + p] = c * vkp - s * vkq;
          V[k * Q + q] = s * vkp + c * vkq;
        }
        __syncthreads();
        for (int k = t; k < Q; k += blockDim.x) {   // A <- J^T A (rows p, q)
          const double apk = A[p * Q + k], aqk = A[q * Q + k];
          A[p * Q + k] = c * apk - s * aqk;
          A[q * Q + k] = s * apk + c * aqk;
        }
        __syncthreads();
      }
  }
  if (t == 0) {
    for (int i = 0; i < Q; ++i) order[i] = i;
    for (int i = 0; i < Q; ++i) {            // selection sort, descending eigenvalue
      int b = i;
      for (int j = i + 1; j < Q; ++j)
        if (A[order[j] * Q + order[j]] > A[order[b] * Q + order[b]]) b = j;
      const int tmp = order[i];
      order[i] = order[b];
      order[b] = tmp;
    }
    const double lmax = A[order[0] * Q + order[0]];
    int kept = 0;
    while (kept < Q && lmax > 0 && A[order[kept] * Q + order[kept]] > rel_keep * lmax) ++kept;
    if (mode == 1 && kept > r) kept = r;
    s_kept = kept;
    *kept_out = kept;
  }
  __syncthreads();
  const int kept = s_kept;
  for (int e = t; e < kept * Q; e += blockDim.x) {
    const int i = e / Q, j = e % Q, col = order[i];
    const double lam = A[col * Q + col];
    Mout[e] = mode == 0 ? V[j * Q + col] / sqrt(lam) : V[j * Q + col];
  }
  if (mode == 1 && sv)
    for (int i = t; i < Q; i += blockDim.x) sv[i] = sqrt(fmax(A[order[i] * Q + order[i]], 0.0));
}

// Out[i][f] = sum_j M[i][j] In[j][f]  (M small, I x J row-major, double).
__global__ void small_left_mul_kernel(const double* __restrict__ M, int I, int J, const float* __restrict__ In,
                                      int n, float* __restrict__ Out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (f >= n || i >= I) return;
  double s = 0.0;
  for (int j = 0; j < J; ++j) s += M[i * J + j] * (double)In[(size_t)j * n + f];
  Out[(size_t)i * n + f] = (float)s;
}

// Sign convention of each POD mode: its entry of largest magnitude (lowest
// index on ties) is positive.  One block of 256 threads per mode.
__global__ void __launch_bounds__(256) fix_sign_kernel(float* __restrict__ Phi, int n) {
  __shared__ float bv[256];
  __shared__ int bi[256];
  float* row = Phi + (size_t)blockIdx.x * n;
  float best = -1.f;
  int idx = 0x7fffffff;
  for (int f = threadIdx.x; f < n; f += blockDim.x) {
    const float a = fabsf(row[f]);
    if (a > best) {
      best = a;
      idx = f;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = idx;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      const float o = bv[threadIdx.x + k];
      const int oi = bi[threadIdx.x + k];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const bool flip = bi[0] < n && row[bi[0]] < 0.f;
  __syncthreads();
  if (flip)
    for (int f = threadIdx.x; f < n; f += blockDim.x) row[f] = -row[f];
}

// U[p][f] = mean[f] + sum_j C[p][j] Phi[j][f]; block: 8 paths x 1024 columns,
// float4 per thread (n % 4 == 0, r <= 80); streaming stores.
__global__ void __launch_bounds__(256) decode_kernel(const float* __restrict__ C, int64_t P, int r,
                                                     const float* __restrict__ Phi, const float* __restrict__ mean,
                                                     int n, float* __restrict__ U) {
  __shared__ float Cs[8][SK_Q];
  const int64_t p0 = (int64_t)blockIdx.y * 8;
  for (int e = threadIdx.x; e < 8 * r; e += blockDim.x) {
    const int pp = e / r, j = e % r;
    Cs[pp][j] = (p0 + pp < P) ? C[(p0 + pp) * r + j] : 0.f;
  }
  __syncthreads();
  const int f = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (f >= n) return;
  const float4 m = *reinterpret_cast<const float4*>(mean + f);
  float4 acc[8];
#pragma unroll
  for (int pp = 0; pp < 8; ++pp) acc[pp] = m;
  for (int j = 0; j < r; ++j) {
    const float4 ph = __ldg(reinterpret_cast<const float4*>(Phi + (size_t)j * n + f));
#pragma unroll
    for (int pp = 0; pp < 8; ++pp) {
      const float c = Cs[pp][j];
      acc[pp].x = fmaf(c, ph.x, acc[pp].x);
      acc[pp].y = fmaf(c, ph.y, acc[pp].y);
      acc[pp].z = fmaf(c, ph.z, acc[pp].z);
      acc[pp].w = fmaf(c, ph.w, acc[pp].w);
    }
  }
#pragma unroll
  for (int pp = 0; pp < 8; ++pp)
    if (p0 + pp < P) __stcs(reinterpret_cast<float4*>(U + (p0 + pp) * n + f), acc[pp]);
}

// Audit of local path j * every: relative L2 distance of the surrogate solution
// to the Magnus solution (double sums); above tol (or non-finite) the Magnus
// solution replaces it.  One block per audited path.  Flags: bit 0 audited, bit 1 replaced.
__global__ void __launch_bounds__(256) audit_kernel(float* __restrict__ U, const float* __restrict__ Uref, int64_t na,
                                                    int64_t every, int n, double tol, double* __restrict__ err,
                                                    uint32_t* __restrict__ flags) {
  __shared__ double red[256];
  const int64_t j = blockIdx.x;
  float* u = U + (size_t)(j * every) * n;
  const float* ur = Uref + (size_t)j * n;
  double dd = 0.0, rr = 0.0;
  for (int f = threadIdx.x; f < n; f += blockDim.x) {
    const double a = u[f], b = ur[f];
    dd += (a - b) * (a - b);
    rr += b * b;
  }
  dd = block_sum_d(dd, red);
  rr = block_sum_d(rr, red);
  double e = rr > 0 ? sqrt(dd / rr) : sqrt(dd);
  if (!(e == e)) e = INFINITY;   // NaN in the surrogate output counts as a failure
  const bool bad = !(e <= tol);
  if (bad)
    for (int f = threadIdx.x; f < n; f += blockDim.x) u[f] = ur[f];
  if (threadIdx.x == 0) {
    err[j] = e;
    if (flags) flags[j * every] |= 1u | (bad ? 2u : 0u);
  }
}

__global__ void or_flags_kernel(uint32_t* __restrict__ flags, int64_t n, uint32_t bits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flags[i] |= bits;
}

}  // namespace sgk

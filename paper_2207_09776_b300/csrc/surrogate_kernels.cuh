// Device kernels of the learned surrogate: Brownian features, the BF16 MLP
// (tensor-core GEMMs with fused epilogues, loss, Adam), the randomized POD
// and the decode / audit kernels.
#pragma once

#include <cuda_bf16.h>

#include "msk_internal.cuh"
#include "philox.cuh"
#include "umma.cuh"

namespace sgk {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ features
// Standard normals of fine cells 2j, 2j+1 in single precision: the same Philox
// words as the double-precision generator (stream tag 0), uniforms
// (hi + 1/2) 2^-32 from the high word of each pair, Box-Muller with the
// hardware approximations of log2, sin and cos (absolute errors ~1e-6, far
// below the bf16 rounding of the features).  The angle is evaluated in
// (-pi, pi], where the hardware sin/cos are accurate: cos(2 pi u) =
// -cos(2 pi (u - 1/2)) and sin(2 pi u) = -sin(2 pi (u - 1/2)).
__device__ __forceinline__ void normal_pair_f32(uint64_t seed, uint64_t path, uint64_t j, float& z0, float& z1) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)path, (uint32_t)(path >> 32), 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float u1 = fmaf((float)w.y, 0x1p-32f, 0x1p-33f);
  const float u2 = fmaf((float)w.w, 0x1p-32f, 0x1p-33f);
  const float r = sqrtf(-1.3862943611198906f * __log2f(u1));   // -2 ln u1 = -2 ln2 log2 u1
  const float a = 6.283185307179586f * (u2 - 0.5f);
  float s, c;
  __sincosf(a, &s, &c);
  z0 = -r * c;
  z1 = -r * s;
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
  // 32-bit cell arithmetic (n_fine <= 2^32): a 64-bit integer to float
  // conversion would run on the double-precision pipe.
  const uint32_t m = (uint32_t)(n_fine / K), c0 = (uint32_t)k * m;
  const int odd = (int)(c0 & 1u);                     // cell c0 is the second of its pair
  const uint32_t npair = (m + odd + 1) >> 1;          // pairs touching [c0, c0 + m)
  float A = 0.f, B = 0.f;
  for (uint32_t q = lane; q < npair; q += 32) {
    float z0, z1;
    normal_pair_f32(seed, gpath, (uint64_t)((c0 >> 1) + q), z0, z1);
    const int i0 = 2 * (int)q - odd;                  // cell index within the step of z0
    const float t0 = (float)i0 + 0.5f;
    if (i0 >= 0) {
      A += z0;
      B = fmaf(z0, t0, B);
    }
    if (i0 + 1 < (int)m) {
      A += z1;
      B = fmaf(z1, t0 + 1.0f, B);
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

// ------------------------------------------------------------------ BF16 GEMM (tcgen05)
// C[M][N] = sum_k A[m][k] B[n][k]: both operands K-major bf16 in global memory
// (row strides multiples of 8 elements), fp32 accumulation in tensor memory,
// 128 x BN output tiles fed by TMA (128-byte swizzle) and tcgen05.mma
// (128 x BN x 16 per instruction); see gemm_tc_kernel below.  With split-K the
// K range is divided into `splits` parts and EPI_F32 writes part z to
// C + z * split_stride.
enum { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_GELU = 2, EPI_GELU_BWD = 3, EPI_BIAS_SPLIT = 4, EPI_ADD_MEAN = 5 };

struct TcArgs {
  int M, N, K, kchunk;
  float* C;              // fp32 row-major [M][ldc] (EPI_BIAS_GELU: z, optional; EPI_GELU_BWD: dz, optional)
  int ldc;
  int64_t split_stride;
  bf16* C16;             // bf16 row-major [M][ldc16] (EPI_BIAS_GELU: GELU(z); EPI_GELU_BWD: dz;
                         // EPI_BIAS_SPLIT: [hi | hi | lo] of the output, 3N columns), optional
  int ldc16;
  bf16* CT;              // bf16 transposed [N][ldct] copy of the bf16 output, optional
  int ldct;
  const float* bias;     // [N] (EPI_ADD_MEAN: the POD mean)
  const float* aux;      // EPI_GELU_BWD: pre-activation z [M][ldaux]
  int ldaux;
  uint32_t* err;         // bit 0 set if a pipeline wait ran out
  int wait_test;         // test hook: the epilogue first waits on a barrier nothing arrives at
};

constexpr int TC_BM = 128, TC_BK = 64;
constexpr uint32_t kTcWaitLimit = 1u << 24;   // polls of one mbarrier before giving up
constexpr uint32_t kTcTestPolls = 1u << 10;    // polls of the test hook's wait (it never completes)

// EPI_ADD_MEAN stages each epilogue warp's 32 x 32 float chunks in two 4 KB
// buffers (128-byte swizzle) for TMA stores.
constexpr int TC_STAGE_BYTES = 8 * 2 * 4096;

__host__ __device__ constexpr size_t tc_smem_bytes(int BN, int stages, int epi) {
  return 1024 + (size_t)stages * (TC_BM + BN) * TC_BK * 2 + 1024 + (epi == EPI_ADD_MEAN ? TC_STAGE_BYTES : 0);
}

__device__ __forceinline__ void store_row_f32(float* dst, const float (&v)[32], int nn) {
  if (nn == 32 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < nn) dst[j] = v[j];
  }
}

__device__ __forceinline__ void store_row_bf16(bf16* dst, const float (&v)[32], int nn) {
  if (nn == 32 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
    uint32_t pk[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
      pk[q] = *reinterpret_cast<const uint32_t*>(&b2);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      reinterpret_cast<uint4*>(dst)[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < nn) dst[j] = __float2bfloat16(v[j]);
  }
}

__device__ __forceinline__ void store_row_f32_stream(float* dst, const float (&v)[32], int nn) {
  if (nn == 32 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      __stcs(reinterpret_cast<float4*>(dst) + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < nn) __stcs(dst + j, v[j]);
  }
}

// Column j of the chunk goes to CT[(nb + j) * ldct + m]: the 32 lanes of a warp
// hold consecutive rows m, so each j is one coalesced 64-byte store.
__device__ __forceinline__ void store_col_bf16(bf16* CT, int ldct, int nb, int m, const float (&v)[32], int nn) {
#pragma unroll
  for (int j = 0; j < 32; ++j)
    if (j < nn) CT[(size_t)(nb + j) * ldct + m] = __float2bfloat16(v[j]);
}

template <int EPI>
__device__ __forceinline__ void tc_epilogue_chunk(const TcArgs& g, float (&v)[32], int m, int nb, int nn, int z) {
  if (EPI == EPI_F32) {
    store_row_f32(g.C + (size_t)z * g.split_stride + (size_t)m * g.ldc + nb, v, nn);
  } else if (EPI == EPI_BIAS_F32) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < nn) v[j] += __ldg(g.bias + nb + j);
    store_row_f32(g.C + (size_t)m * g.ldc + nb, v, nn);
  } else if (EPI == EPI_BIAS_GELU) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < nn) v[j] += __ldg(g.bias + nb + j);
    if (g.C) store_row_f32(g.C + (size_t)m * g.ldc + nb, v, nn);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = gelu(v[j]);
    if (g.C16) store_row_bf16(g.C16 + (size_t)m * g.ldc16 + nb, v, nn);
    if (g.CT) store_col_bf16(g.CT, g.ldct, nb, m, v, nn);
  } else if (EPI == EPI_BIAS_SPLIT) {
    // network output c = acc + bias, and its two-term bf16 split c ~ hi + lo
    // laid out [hi | hi | lo] so that one K = 3N contraction with the split
    // basis [Phi_hi | Phi_lo | Phi_hi] gives hi Phi_hi + hi Phi_lo + lo Phi_hi.
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < nn) v[j] += __ldg(g.bias + nb + j);
    if (g.C) store_row_f32(g.C + (size_t)m * g.ldc + nb, v, nn);
    float hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      hi[j] = __bfloat162float(__float2bfloat16(v[j]));
      lo[j] = v[j] - hi[j];
    }
    bf16* row = g.C16 + (size_t)m * g.ldc16;
    store_row_bf16(row + nb, hi, nn);
    store_row_bf16(row + g.N + nb, hi, nn);
    store_row_bf16(row + 2 * g.N + nb, lo, nn);
  } else if (EPI == EPI_ADD_MEAN) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < nn) v[j] += __ldg(g.bias + nb + j);
    store_row_f32_stream(g.C + (size_t)m * g.ldc + nb, v, nn);
  } else {
    const float* z = g.aux + (size_t)m * g.ldaux + nb;
    if (nn == 32 && (reinterpret_cast<uintptr_t>(z) & 15) == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 zz = __ldg(reinterpret_cast<const float4*>(z) + q);
        v[4 * q] *= gelu_prime(zz.x);
        v[4 * q + 1] *= gelu_prime(zz.y);
        v[4 * q + 2] *= gelu_prime(zz.z);
        v[4 * q + 3] *= gelu_prime(zz.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < nn) v[j] *= gelu_prime(z[j]);
    }
    if (g.C) store_row_f32(g.C + (size_t)m * g.ldc + nb, v, nn);
    if (g.C16) store_row_bf16(g.C16 + (size_t)m * g.ldc16 + nb, v, nn);
    if (g.CT) store_col_bf16(g.CT, g.ldct, nb, m, v, nn);
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(bar)) : "memory");
}

// Persistent, warp-specialised tcgen05 GEMM.  The grid holds at most one CTA
// per resident slot; CTA b computes tiles b, b + gridDim.x, ... of the
// (split, m-tile, n-tile) enumeration (n fastest).  Warps:
//   0       TMA producer (lane 0): 128 x 64 and BN x 64 operand boxes through a
//           TC_STAGES-deep shared-memory ring (full/empty mbarriers);
//   1       TMEM owner and MMA issuer (lane 0): tcgen05.mma into one of two
//           BN-column accumulators (double buffer), commit to tmem_full[b];
//   2 .. 9  epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its tile rows)
//           and half of the tile's columns, then frees the accumulator
//           (tmem_empty[b], eight arrivals), so the next tile's MMAs overlap
//           this tile's epilogue.
// Every mbarrier wait is bounded (kTcWaitLimit polls); on expiry the thread sets
// g.err, an epilogue warp skips its remaining tiles (releasing each accumulator),
// the producer waits for its issued loads and the MMA issuer for its issued MMAs,
// so no CTA leaves with a bulk copy or an MMA in flight.
constexpr int TC_THREADS = 320;

template <int BN, int EPI, int TC_STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1) gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                 const __grid_constant__ CUtensorMap tmB,
                                                                 const __grid_constant__ CUtensorMap tmC,
                                                                 const TcArgs g, int tiles_m, int tiles_n,
                                                                 int splits) {
  static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
  static_assert(TC_STAGES >= 2 && TC_STAGES <= 6, "pipeline depth");
  constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2, B_BYTES = BN * TC_BK * 2;
  extern __shared__ uint8_t tc_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + TC_STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + TC_STAGES * B_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* tfull = empty + TC_STAGES;     // [2]
  uint64_t* tempty = tfull + 2;            // [2]
  uint64_t* never = tempty + 2;            // test hook: no thread ever arrives here
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  uint8_t* stage_out = sB + TC_STAGES * B_BYTES + 1024;   // EPI_ADD_MEAN: [8 warps][2][32 rows x 128 B]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_split = tiles_m * tiles_n, ntiles = per_split * splits;

  if (threadIdx.x == 0) {
    umma::prefetch_tensormap(&tmA);
    umma::prefetch_tensormap(&tmB);
    if (EPI == EPI_ADD_MEAN) umma::prefetch_tensormap(&tmC);
    for (int s = 0; s < TC_STAGES; ++s) {
      umma::mbar_init(full + s, 1);
      umma::mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      umma::mbar_init(tfull + b, 1);
      umma::mbar_init(tempty + b, 8);
    }
    umma::mbar_init(never, 1);
    umma::fence_barrier_init();
  }
  if (warp == 1) umma::tmem_alloc(tmem_slot, 2 * BN);
  umma::tc_fence_before();
  __syncthreads();
  umma::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto k_range = [&](int z, int& kbeg, int& nk) {
    kbeg = z * g.kchunk;
    const int kend = min(g.K, kbeg + g.kchunk);
    nk = (kend - kbeg + TC_BK - 1) / TC_BK;   // >= 1: every split owns a non-empty K range
  };

  bool fail = false;
  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      uint32_t it = 0;
      for (int t = blockIdx.x; t < ntiles && !fail; t += gridDim.x) {
        const int z = t / per_split, rem = t % per_split;
        const int m0 = (rem / tiles_n) * TC_BM, n0 = (rem % tiles_n) * BN;
        int kbeg, nk;
        k_range(z, kbeg, nk);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % TC_STAGES;
          if (!umma::mbar_wait(empty + s, ((it / TC_STAGES) & 1) ^ 1, kTcWaitLimit)) {
            fail = true;
            break;
          }
          umma::mbar_arrive_expect_tx(full + s, A_BYTES + B_BYTES);
          const int kc = kbeg + kb * TC_BK;
          umma::tma_load_2d(sA + s * A_BYTES, &tmA, full + s, kc, m0);
          umma::tma_load_2d(sB + s * B_BYTES, &tmB, full + s, kc, n0);
        }
      }
      // the last load of every stage has landed before the CTA can leave
      for (uint32_t j = it > (uint32_t)TC_STAGES ? it - TC_STAGES : 0; j < it; ++j)
        if (!umma::mbar_wait(full + j % TC_STAGES, (j / TC_STAGES) & 1, kTcWaitLimit)) fail = true;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      constexpr uint32_t idesc = umma::idesc_bf16_f32(TC_BM, BN);
      uint32_t it = 0, i = 0;
      int last0 = -1, last1 = -1;   // tile of the last commit on accumulators 0 and 1
      for (int t = blockIdx.x; t < ntiles && !fail; t += gridDim.x, ++i) {
        const int z = t / per_split;
        int kbeg, nk;
        k_range(z, kbeg, nk);
        const uint32_t ab = i & 1;
        if (!umma::mbar_wait(tempty + ab, ((i >> 1) & 1) ^ 1, kTcWaitLimit)) {
          fail = true;
          break;
        }
        umma::tc_fence_after();
        const uint32_t d = tmem + ab * BN;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % TC_STAGES;
          if (!umma::mbar_wait(full + s, (it / TC_STAGES) & 1, kTcWaitLimit)) {
            fail = true;
            break;
          }
          umma::tc_fence_after();
          const uint64_t da = umma::desc_sw128_kmajor(sA + s * A_BYTES);
          const uint64_t db = umma::desc_sw128_kmajor(sB + s * B_BYTES);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk)   // 16 bf16 = 32 bytes along K inside the swizzle atom
            umma::mma_bf16(d, da + 2 * kk, db + 2 * kk, idesc, (kb | kk) ? 1u : 0u);
          umma::mma_commit(empty + s);
        }
        umma::mma_commit(tfull + ab);   // arrives when this tile's MMAs are complete
        if (ab) last1 = (int)i;
        else last0 = (int)i;
      }
      // every MMA issued has completed before TMEM can be freed, also when the epilogue
      // gave up on a tile and no longer waits for it (bounded like every wait)
      if (last0 >= 0 && !umma::mbar_wait(tfull + 0, ((uint32_t)last0 >> 1) & 1, kTcWaitLimit)) fail = true;
      if (last1 >= 0 && !umma::mbar_wait(tfull + 1, ((uint32_t)last1 >> 1) & 1, kTcWaitLimit)) fail = true;
    }
  } else {
    // ---- epilogue warps
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    constexpr int CH = BN / 32 / 2;                     // 32-column chunks per warp
    uint8_t* my_stage = stage_out + (warp - 2) * 2 * 4096;
    uint32_t i = 0, nchunk = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int z = t / per_split, rem = t % per_split;
      const int m0 = (rem / tiles_n) * TC_BM, n0 = (rem % tiles_n) * BN;
      const uint32_t ab = i & 1;
      // after a wait has run out the warp waits no more: it skips its tiles but still
      // releases each accumulator, so the MMA issuer and the TMA producer run to the end
      bool ok = !fail;
      if (ok && g.wait_test) ok = umma::mbar_wait(never, 0, kTcTestPolls);
      if (ok) ok = umma::mbar_wait(tfull + ab, (i >> 1) & 1, kTcWaitLimit);
      const bool ready = __all_sync(0xffffffffu, ok);
      umma::tc_fence_after();
      if (!ready) fail = true;
      const int m = m0 + quarter * 32 + lane;
#pragma unroll 1
      for (int c = half * CH; ready && c < (half + 1) * CH; ++c) {
        const int nb = n0 + c * 32;
        if (nb >= g.N) break;                                 // same for the whole warp
        uint32_t r[32];
        umma::tmem_ld32(tmem + ab * BN + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(c * 32), r);
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
        if constexpr (EPI == EPI_ADD_MEAN) {
          // u = acc + mean, staged row-per-lane in a 128B-swizzled 32 x 32 box and
          // written by one TMA store (rows beyond M are clipped by the tensor map)
          const float4* mv = reinterpret_cast<const float4*>(g.bias + nb);
          uint8_t* sb = my_stage + (nchunk & 1) * 4096;
          if (lane == 0) umma::bulk_wait_read<1>();     // the store issued from this buffer two chunks ago
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 mm = __ldg(mv + q);
            const float4 o = make_float4(v[4 * q] + mm.x, v[4 * q + 1] + mm.y, v[4 * q + 2] + mm.z,
                                         v[4 * q + 3] + mm.w);
            *reinterpret_cast<float4*>(sb + lane * 128 + ((q ^ (lane & 7)) << 4)) = o;
          }
          umma::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            umma::tma_store_2d(&tmC, sb, nb, m0 + quarter * 32);
            umma::bulk_commit();
          }
          ++nchunk;
        } else {
          if (m < g.M) tc_epilogue_chunk<EPI>(g, v, m, nb, min(32, g.N - nb), z);
        }
      }
      umma::tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + ab);
    }
    if (EPI == EPI_ADD_MEAN && lane == 0) umma::bulk_wait_all();
  }
  if (fail) atomicOr(g.err, 1u);
  __syncwarp();
  umma::tc_fence_before();
  __syncthreads();
  if (warp == 1) umma::tmem_dealloc(tmem, 2 * BN);
}

// A' [P][ld] = [hi | hi | lo] of fp32 coefficients C [P][r] (see EPI_BIAS_SPLIT).
__global__ void split_coef_kernel(const float* __restrict__ C, int64_t P, int r, bf16* __restrict__ A, int ld) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P * r) return;
  const int64_t p = e / r;
  const int j = (int)(e % r);
  const float v = C[e];
  const bf16 hi = __float2bfloat16(v);
  const bf16 lo = __float2bfloat16(v - __bfloat162float(hi));
  bf16* row = A + p * ld;
  row[j] = hi;
  row[r + j] = hi;
  row[2 * r + j] = lo;
}

// Split decode basis B' [n][ld] = [Phi_hi | Phi_lo | Phi_hi] (K-major) from Phi [r][n].
__global__ void split_basis_kernel(const float* __restrict__ phi, int r, int n, bf16* __restrict__ B, int ld) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)r * n) return;
  const int j = (int)(e / n), f = (int)(e % n);
  const float v = phi[e];
  const bf16 hi = __float2bfloat16(v);
  const bf16 lo = __float2bfloat16(v - __bfloat162float(hi));
  bf16* row = B + (size_t)f * ld;
  row[j] = hi;
  row[r + j] = lo;
  row[2 * r + j] = hi;
}

// out[c][ld_out] = in[r][ld_in]^T for a rows x cols bf16 matrix (32 x 32 tiles).
__global__ void transpose_bf16_kernel(const bf16* __restrict__ in, int rows, int cols, int ld_in,
                                      bf16* __restrict__ out, int ld_out) {
  __shared__ bf16 t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * ld_in + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[(size_t)c * ld_out + r] = t[threadIdx.x][i];
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
// out, target, g, g16: [B][r]; g16T: [r][ldt] (transposed bf16 copy).
__global__ void __launch_bounds__(256) loss_grad_kernel(const float* __restrict__ out, const float* __restrict__ target,
                                                        int64_t n, int r, float inv_b, float* __restrict__ g,
                                                        bf16* __restrict__ g16, bf16* __restrict__ g16T, int ldt,
                                                        double* __restrict__ partial) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float d = out[e] - target[e];
    s += (double)d * d;
    const float gv = 2.0f * d * inv_b;
    const bf16 gq = __float2bfloat16(gv);
    g[e] = gv;
    g16[e] = gq;
    g16T[(size_t)(e % r) * ldt + e / r] = gq;
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

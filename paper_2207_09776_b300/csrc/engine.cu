// S5b/S6/S7: the shared-memory-resident stencil engine.
//
// Iterated Magnus (Section 2, "Iterated Magnus expansion"): on each of K
// sub-intervals U <- exp(Omega_n) U, with the exponential action evaluated as
// (T_m((Omega_n - mu I)/s))^s e^{mu} U by a scaled truncated Taylor series
// whose terms are widened-stencil matvecs (stencil.cuh), stopped early when two
// consecutive terms fall below the unit roundoff relative to the partial sum
// (the termination test of Al-Mohy & Higham 2011).  Euler-Maruyama
// (Eq. EulerMaruyama) is the same engine with one matvec per step by
// I + dt B(t_n) + dW_n A(t_n).
//
// Data layout.  One path's d x d state lives entirely in shared memory, split
// into C row slabs of d/C v-rows, one slab per CTA of a thread-block cluster
// (C = 1 for d <= 128 in float).  Each slab is double-buffered (ping-pong): a
// matvec reads buffer `cur` and writes buffer `cur ^ 1`, so one cluster-wide
// barrier per matvec suffices.  The two v-rows above and below a slab (the
// stencil's halo) are read directly from the neighbouring CTA's shared memory
// (distributed shared memory); rows outside the grid read as zero (Dirichlet).
// Each buffer row carries two zero columns on each side, so x neighbours need
// no bounds checks.
//
// Thread mapping.  Lane l of warp w owns grid column i = 32 (w mod d/32) + l
// and a strip of R consecutive v-rows; it keeps the Taylor partial sum of its
// R points in registers and slides a 5-row window over its strip, so each
// point costs five shared-memory loads (the new rows of columns i, i+-1, i+-2)
// and one store.  Interior-row coefficients sit in registers; only the four
// boundary rows (where the truncated-matrix commutators differ) and the centre
// of the V1 band (which carries v_j) are read from shared memory.
//
// Norms for early termination are reduced per warp with shuffles, published
// per warp in shared memory and gathered by every thread after the barrier,
// so all CTAs of a cluster take identical decisions.
#include <cooperative_groups.h>

#include <algorithm>

#include "stencil.cuh"

namespace cg = cooperative_groups;

extern const double kMskScaleCap;
msk_status msk_refresh_u0max(msk_ctx* ctx, cudaStream_t stream);

namespace {

struct EngineArgs {
  const double* band;
  const double* u0;
  const double* Wt;   // Magnus: [paths][steps][MSK_NWT]
  const double* dW;   // Euler:  [paths][steps]
  void* out;
  uint32_t* status;
  unsigned long long* work;
  int64_t paths;
  int steps;
  double dx, dv, av, T, tol, u0max, s_cap;
  CoefDev c;
};

template <typename T, int D, int C, int NT>
struct Cfg {
  static constexpr int RS = D / C;         // v-rows per CTA
  static constexpr int W = D + 4;          // padded row width
  static constexpr int NW = NT / 32;       // warps per CTA
  static constexpr int NWC = D / 32;       // warps across one row
  static constexpr int G = NW / NWC;       // row groups per CTA
  static constexpr int R = RS / G;         // rows per thread
  static_assert(D % 32 == 0, "d must be a multiple of 32");
  static_assert(NW % NWC == 0 && G >= 1, "thread count must cover whole rows");
  static_assert(RS % G == 0 && R >= 2, "slab rows must split evenly");
  static constexpr size_t BUF = (size_t)RS * W;
  static constexpr size_t OFF_ZERO = 2 * BUF;
  static constexpr size_t OFF_COEF = OFF_ZERO + W;               // 5 x 12 (4 boundary rows + interior)
  static constexpr size_t OFF_B0 = OFF_COEF + 5 * MSK_NCOEF;      // RS
  static constexpr size_t OFF_SLOT = OFF_B0 + RS;                 // 2 x NW x 2
  static constexpr size_t NELEM = OFF_SLOT + 4 * NW;
  static constexpr size_t SMEM = NELEM * sizeof(T);
};

template <typename T>
__device__ __forceinline__ T absnan(T x) {
  return (x == x) ? (x < T(0) ? -x : x) : T(INFINITY);
}
template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

template <int C>
__device__ __forceinline__ void sync_all() {
  if constexpr (C == 1) {
    __syncthreads();
  } else {
    cg::this_cluster().sync();
  }
}

__device__ __forceinline__ double sigma_t(const CoefDev& c, double t) {
  return c.s0 * (1.0 + c.s1 * cospi(2.0 * t));
}
__device__ __forceinline__ double alpha_t(const CoefDev& c, double t) {
  return 0.5 * (c.a0 + c.a1 * sinpi(2.0 * t));
}

template <typename T, int D, int C, int NT, bool EULER>
__global__ void __launch_bounds__(NT, 1) engine_kernel(const EngineArgs a) {
  using K = Cfg<T, D, C, NT>;
  constexpr int RS = K::RS, W = K::W, NW = K::NW, NWC = K::NWC, R = K::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* zrow = sm + K::OFF_ZERO;
  T* coef = sm + K::OFF_COEF;
  T* b0row = sm + K::OFF_B0;
  T* slots = sm + K::OFF_SLOT;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = (warp % NWC) * 32 + lane;   // grid column (x index)
  const int j0 = (warp / NWC) * R;          // first local v-row of this thread
  int rank = 0;
  if constexpr (C > 1) rank = (int)cg::this_cluster().block_rank();
  const int r0 = rank * RS;                 // first global v-row of this CTA
  const int64_t cid = blockIdx.x / C, ncl = gridDim.x / C;
  const bool edge = (i == 0) || (i == D - 1);
  const double inv2dx = 0.5 / a.dx, inv4dx2 = 0.25 / (a.dx * a.dx);

  // zero row and the two zero columns on each side of both buffers
  for (int e = tid; e < W; e += NT) zrow[e] = T(0);
  for (int e = tid; e < 2 * RS * 4; e += NT) {
    const int b = e / (RS * 4), rem = e % (RS * 4), row = rem / 4, cc = rem % 4;
    sm[b * K::BUF + (size_t)row * W + (cc < 2 ? cc : D + cc)] = T(0);
  }
  sync_all<C>();

  // value of column `col` (may be -2..D+1) of global v-row jg in buffer `b`
  auto ld = [&](int b, int jg, int col) -> T {
    if (jg >= r0 && jg < r0 + RS) return sm[b * K::BUF + (size_t)(jg - r0) * W + col + 2];
    if (jg < 0 || jg >= D) return T(0);
    if constexpr (C > 1) {
      const int pr = jg / RS;
      const T* peer = cg::this_cluster().map_shared_rank(sm, pr);
      return peer[b * K::BUF + (size_t)(jg - pr * RS) * W + col + 2];
    }
    return T(0);
  };

  // gather the per-warp maxima of all CTAs of the cluster (identical in every thread)
  auto gather = [&](int par, T& gn, T& ga) {
    gn = T(0);
    ga = T(0);
    for (int q = lane; q < C * NW; q += 32) {
      const int cr = q / NW, wq = q % NW;
      const T* sl = slots;
      if constexpr (C > 1) {
        if (cr != rank) sl = cg::this_cluster().map_shared_rank(slots, cr);
      }
      gn = tmax(gn, sl[(par * NW + wq) * 2 + 0]);
      ga = tmax(ga, sl[(par * NW + wq) * 2 + 1]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      gn = tmax(gn, __shfl_xor_sync(0xffffffffu, gn, off));
      ga = tmax(ga, __shfl_xor_sync(0xffffffffu, ga, off));
    }
  };

  for (int64_t path = cid; path < a.paths; path += ncl) {
    T acc[R];
    int cur = 0, par = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int jg = r0 + j0 + r;
      acc[r] = (T)a.u0[(size_t)jg * D + i];
      sm[(size_t)(j0 + r) * W + i + 2] = acc[r];
    }
    T unorm = (T)a.u0max;   // running infinity norm of the state
    bool scale_cap = false;
    unsigned long long nmv = 0;   // stencil applications of this path
    sync_all<C>();

    for (int n = 0; n < a.steps; ++n) {
      // ---- coefficients of this step's operator ----------------------------------
      double w[MSK_NOPS];
      double shift;
      int s_steps = 1, m_terms = 1;
      double eta = 1.0;
      if constexpr (EULER) {
        const double dt = a.T / a.steps, tn = n * dt;
        const double dWn = a.dW[path * a.steps + n];
        for (int k = 0; k < MSK_NOPS; ++k) w[k] = 0.0;
        w[MSK_OP_BX] = dt;
        w[MSK_OP_BVV] = alpha_t(a.c, tn) * dt;
        w[MSK_OP_A0] = sigma_t(a.c, tn) * dWn;
        shift = 1.0;
      } else {
        const double* rec = a.Wt + ((size_t)path * a.steps + n) * MSK_NWT;
        for (int k = 0; k < MSK_NOPS; ++k) w[k] = rec[k];
        const double mu = rec[MSK_WT_MU];
        s_steps = (int)rec[MSK_WT_S];
        m_terms = (int)rec[MSK_WT_M];
        if (rec[MSK_WT_S] >= a.s_cap) scale_cap = true;
        shift = -mu;
        eta = exp(mu / s_steps);
      }
      if (tid < 5) {
        const int jr = tid < 4 ? special_row(tid, D) : 2;
        double cf[MSK_NCOEF];
        fold_row(a.band, D, jr, w, shift, inv2dx, inv4dx2, cf);
#pragma unroll
        for (int q = 0; q < MSK_NCOEF; ++q) coef[tid * MSK_NCOEF + q] = (T)cf[q];
      }
      for (int jl = tid - 5; jl >= 0 && jl < RS; jl += NT) b0row[jl] = (T)fold_b0(a.band, D, r0 + jl, w, inv2dx);
      __syncthreads();
      T cI[MSK_NCOEF];
#pragma unroll
      for (int q = 0; q < MSK_NCOEF; ++q) cI[q] = coef[4 * MSK_NCOEF + q];
      const T cIa1 = edge ? cI[CF_AE + 0] : cI[CF_A + 1];
      const T cIa3 = edge ? cI[CF_AE + 1] : cI[CF_A + 3];

      for (int sub = 0; sub < s_steps; ++sub) {
        T c1 = unorm;   // norm of the previous Taylor term (term 0 = the state)
        for (int k = 1; k <= m_terms; ++k) {
          const T scale = EULER ? T(1) : (T)(1.0 / ((double)s_steps * k));
          const int nxt = cur ^ 1;
          T* dst = sm + nxt * K::BUF;
          T mn = T(0), ma = T(0);
          // sliding window over rows jg-2 .. jg+2
          int jg = r0 + j0;
          T cc0 = ld(cur, jg - 2, i), cc1 = ld(cur, jg - 1, i), cc2 = ld(cur, jg, i), cc3 = ld(cur, jg + 1, i);
          T l1a = ld(cur, jg - 1, i - 1), l1b = ld(cur, jg, i - 1);
          T r1a = ld(cur, jg - 1, i + 1), r1b = ld(cur, jg, i + 1);
          T l2a = ld(cur, jg - 1, i - 2), l2b = ld(cur, jg, i - 2);
          T r2a = ld(cur, jg - 1, i + 2), r2b = ld(cur, jg, i + 2);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            jg = r0 + j0 + r;
            const T cc4 = ld(cur, jg + 2, i);
            const T l1c = ld(cur, jg + 1, i - 1), r1c = ld(cur, jg + 1, i + 1);
            const T l2c = ld(cur, jg + 1, i - 2), r2c = ld(cur, jg + 1, i + 2);
            T A0, A1, A2, A3, A4, B0, B1, B2, C0, C1;
            if (is_special_row(jg, D)) {
              const T* cs = coef + special_index(jg, D) * MSK_NCOEF;
              A0 = cs[CF_A + 0];
              A1 = edge ? cs[CF_AE + 0] : cs[CF_A + 1];
              A2 = cs[CF_A + 2];
              A3 = edge ? cs[CF_AE + 1] : cs[CF_A + 3];
              A4 = cs[CF_A + 4];
              B0 = cs[CF_B + 0];
              B1 = cs[CF_B + 1];
              B2 = cs[CF_B + 2];
              C0 = cs[CF_C + 0];
              C1 = cs[CF_C + 1];
            } else {
              A0 = cI[CF_A + 0];
              A1 = cIa1;
              A2 = cI[CF_A + 2];
              A3 = cIa3;
              A4 = cI[CF_A + 4];
              B0 = cI[CF_B + 0];
              B1 = b0row[jg - r0];
              B2 = cI[CF_B + 2];
              C0 = cI[CF_C + 0];
              C1 = cI[CF_C + 1];
            }
            T v = A0 * cc0;
            v = fma(A1, cc1, v);
            v = fma(A2, cc2, v);
            v = fma(A3, cc3, v);
            v = fma(A4, cc4, v);
            v = fma(B0, r1a - l1a, v);
            v = fma(B1, r1b - l1b, v);
            v = fma(B2, r1c - l1c, v);
            v = fma(C0, r2a + l2a, v);
            v = fma(C1, r2c + l2c, v);
            if constexpr (EULER) {
              acc[r] = v;
              dst[(size_t)(jg - r0) * W + i + 2] = v;
              ma = tmax(ma, absnan(v));
            } else {
              const T t = v * scale;
              dst[(size_t)(jg - r0) * W + i + 2] = t;
              acc[r] += t;
              mn = tmax(mn, absnan(t));
              ma = tmax(ma, absnan(acc[r]));
            }
            cc0 = cc1; cc1 = cc2; cc2 = cc3; cc3 = cc4;
            l1a = l1b; l1b = l1c; r1a = r1b; r1b = r1c;
            l2a = l2b; l2b = l2c; r2a = r2b; r2b = r2c;
          }
          ++nmv;
          if constexpr (EULER) {
            sync_all<C>();
            cur = nxt;
            break;
          } else {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
              mn = tmax(mn, __shfl_xor_sync(0xffffffffu, mn, off));
              ma = tmax(ma, __shfl_xor_sync(0xffffffffu, ma, off));
            }
            if (lane == 0) {
              slots[(par * NW + warp) * 2 + 0] = mn;
              slots[(par * NW + warp) * 2 + 1] = ma;
            }
            sync_all<C>();
            T gn, ga;
            gather(par, gn, ga);
            par ^= 1;
            cur = nxt;
            unorm = ga;
            if (c1 + gn <= (T)a.tol * ga) break;
            c1 = gn;
          }
        }
        if constexpr (!EULER) {
          // u <- e^{mu/s} (partial sum); written into the buffer not holding the last term
          const T te = (T)eta;
          T* dst = sm + (cur ^ 1) * K::BUF;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            acc[r] *= te;
            dst[(size_t)(j0 + r) * W + i + 2] = acc[r];
          }
          unorm = unorm * te;
          sync_all<C>();
          cur ^= 1;
        }
      }
    }

    // ---- write the solution and the path status ----------------------------------
    T ma = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int jg = r0 + j0 + r;
      ma = tmax(ma, absnan(acc[r]));
      reinterpret_cast<T*>(a.out)[(size_t)path * D * D + (size_t)jg * D + i] = acc[r];
    }
    if (a.work && rank == 0 && tid == 0) atomicAdd(a.work, nmv);
    if (a.status) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) ma = tmax(ma, __shfl_xor_sync(0xffffffffu, ma, off));
      if (lane == 0) {
        slots[(par * NW + warp) * 2 + 0] = ma;
        slots[(par * NW + warp) * 2 + 1] = ma;
      }
      sync_all<C>();
      T gn, ga;
      gather(par, gn, ga);
      par ^= 1;
      if (rank == 0 && tid == 0) {
        uint32_t st = 0;
        if (!(ga < T(INFINITY))) st |= MSK_PATH_NONFINITE;
        if (scale_cap) st |= MSK_PATH_SCALE_CAP;
        if (!((double)ga <= 10.0 * a.u0max)) st |= MSK_PATH_BLOWUP;
        a.status[path] = st;
      }
    }
    sync_all<C>();   // nobody may still read this path's buffers or slots
  }
}

template <typename T, int D, int C, int NT, bool EULER>
msk_status launch_one(msk_ctx* ctx, const EngineArgs& a, cudaStream_t stream) {
  using K = Cfg<T, D, C, NT>;
  auto kern = engine_kernel<T, D, C, NT, EULER>;
  msk_status st = msk_cuda(
      ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM),
      "smem attribute");
  if (st != MSK_OK) return st;
  if (C > 8) {
    st = msk_cuda(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1),
                  "cluster attribute");
    if (st != MSK_OK) return st;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = K::SMEM;
  cfg.stream = stream;
  int64_t clusters = 0;
  if (C > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(C, 1, 1);
    int nc = 0;
    st = msk_cuda(ctx, cudaOccupancyMaxActiveClusters(&nc, kern, &cfg), "occupancy clusters");
    if (st != MSK_OK) return st;
    if (nc < 1) return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "cluster configuration cannot be scheduled");
    clusters = nc;
  } else {
    int per_sm = 0;
    st = msk_cuda(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, K::SMEM),
                  "occupancy");
    if (st != MSK_OK) return st;
    if (per_sm < 1) return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "kernel does not fit on an SM");
    clusters = (int64_t)per_sm * ctx->num_sms;
  }
  clusters = std::min<int64_t>(clusters, a.paths);
  cfg.gridDim = dim3((unsigned)(clusters * C), 1, 1);
  st = msk_cuda(ctx, cudaLaunchKernelEx(&cfg, kern, a), "engine launch");
  return st;
}

template <bool EULER>
msk_status dispatch(msk_ctx* ctx, int precision, const EngineArgs& a, cudaStream_t s) {
  const int d = ctx->d;
  if (precision == MSK_F32) {
    switch (d) {
      case 32: return launch_one<float, 32, 1, 128, EULER>(ctx, a, s);
      case 64: return launch_one<float, 64, 1, 256, EULER>(ctx, a, s);
      case 128: return launch_one<float, 128, 1, 512, EULER>(ctx, a, s);
      case 256: return launch_one<float, 256, 4, 512, EULER>(ctx, a, s);
      case 512: return launch_one<float, 512, 16, 1024, EULER>(ctx, a, s);
    }
  } else {
    switch (d) {
      case 32: return launch_one<double, 32, 1, 128, EULER>(ctx, a, s);
      case 64: return launch_one<double, 64, 1, 256, EULER>(ctx, a, s);
      case 128: return launch_one<double, 128, 2, 512, EULER>(ctx, a, s);
      case 256: return launch_one<double, 256, 8, 512, EULER>(ctx, a, s);
    }
  }
  return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "grid size / precision combination not built");
}

}  // namespace

msk_status launch_engine(msk_ctx* ctx, bool euler, int steps, int64_t paths, int precision,
                         const double* Wt, const double* dW, void* out, uint32_t* status,
                         cudaStream_t stream) {
  if (paths == 0) return MSK_OK;
  EngineArgs a;
  a.band = ctx->band;
  a.u0 = ctx->u0;
  a.Wt = Wt;
  a.dW = dW;
  a.out = out;
  a.status = status;
  a.work = ctx->work;
  a.paths = paths;
  a.steps = steps;
  a.dx = ctx->dx;
  a.dv = ctx->dv;
  a.av = ctx->av;
  a.T = ctx->T;
  a.tol = precision == MSK_F32 ? 0x1p-24 : 0x1p-53;
  a.u0max = ctx->host_u0max;
  a.s_cap = kMskScaleCap;
  a.c = coef_dev(ctx->coef);
  return euler ? dispatch<true>(ctx, precision, a, stream) : dispatch<false>(ctx, precision, a, stream);
}

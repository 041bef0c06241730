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
// into C slabs of d/C v-rows, one slab per CTA of a thread-block cluster
// (C = 1 for d <= 128 in float).  Each slab is double-buffered (ping-pong): a
// matvec reads buffer `cur` and writes buffer `cur ^ 1`, so one cluster-wide
// barrier per matvec suffices.  A slab buffer holds its rows plus two halo
// rows above and below and four padding columns on each side (zero): halo
// rows at the grid boundary stay zero (Dirichlet), halo rows facing another
// CTA are written by that CTA through distributed shared memory as it stores
// its own edge rows, so every load of the inner loop is a local, unguarded,
// 16-byte-aligned shared-memory load.
//
// Thread mapping.  A thread owns four consecutive grid columns (one 128-bit
// load per row in float) and a strip of R consecutive v-rows, keeps the Taylor
// partial sum of its 4R points in registers and slides a five-row window down
// its strip.  The x-neighbours at distance 1 and 2 come from the adjacent
// threads of the same row by warp shuffles (from shared memory only across a
// warp boundary).  Interior-row coefficients sit in registers, scaled by
// 1/(s k) once per Taylor term; only the four boundary rows (where the
// truncated-matrix commutators differ) and the centre of the V1 band (which
// carries v_j) are read from shared memory.  No double-precision arithmetic
// runs inside the matvec loop of the float engine.
//
// Norms for early termination are reduced per warp with shuffles, published
// per warp in shared memory and gathered by every thread after the barrier,
// so all CTAs of a cluster take identical decisions.
#include <cooperative_groups.h>

#include <algorithm>

#include "stencil.cuh"

namespace cg = cooperative_groups;

extern const double kMskScaleCap;

namespace {

constexpr int kMaxTerms = 64;   // >= the largest Taylor degree of either theta table

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
  double dx, T, s_cap;
  float tol32;
  double tol64;
  CoefDev c;
};

template <typename T, int D, int C, int NT>
struct Cfg {
  static constexpr int RS = D / C;         // v-rows per CTA
  static constexpr int TPR = D / 4;        // threads per grid row (4 columns each)
  static constexpr int NG = NT / TPR;      // row groups per CTA
  static constexpr int R = RS / NG;        // rows per thread
  static constexpr int NW = NT / 32;       // warps per CTA
  static constexpr int W = D + 8;          // padded row width: 4 zero columns each side
  static constexpr int ROWS = RS + 4;      // 2 halo rows each side
  static_assert(D % 32 == 0, "d must be a multiple of 32");
  static_assert(NT % TPR == 0 && NG >= 1, "threads must cover whole rows");
  static_assert(TPR <= 32 ? (32 % TPR == 0) : (TPR % 32 == 0), "rows must align with warps");
  static_assert(RS % NG == 0 && R >= 2, "slab rows must split evenly");
  static constexpr size_t BUF = (size_t)ROWS * W;
  static constexpr size_t OFF_COEF = 2 * BUF;                     // 5 x 12: 4 boundary rows + interior
  static constexpr size_t OFF_B0 = OFF_COEF + 5 * MSK_NCOEF;      // RS: centre of V1 per local row
  static constexpr size_t OFF_SCALE = OFF_B0 + RS;                // kMaxTerms + 1: 1/(s k)
  static constexpr size_t OFF_SLOT = OFF_SCALE + kMaxTerms + 1;   // 2 x NW x 2 norm slots
  static constexpr size_t NELEM = OFF_SLOT + 4 * NW;
  static constexpr size_t SMEM = NELEM * sizeof(T);
  static_assert(SMEM <= 232448, "slab does not fit the 227 KB of shared memory per CTA");
};

template <typename T> struct V4 { T x, y, z, w; };

__device__ __forceinline__ V4<float> ld4(const float* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.z, v.w);
}
template <typename T> __device__ __forceinline__ T get(const V4<T>& v, int p) {
  return p == 0 ? v.x : (p == 1 ? v.y : (p == 2 ? v.z : v.w));
}
template <typename T> __device__ __forceinline__ void set(V4<T>& v, int p, T x) {
  if (p == 0) v.x = x; else if (p == 1) v.y = x; else if (p == 2) v.z = x; else v.w = x;
}

// max(|x|) helpers: fmax/fabs map to one min/max instruction with an |x| operand;
// NaN is ignored here (non-finite paths are caught by absnan at the end).
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
template <typename T> __device__ __forceinline__ T tabs(T x) { return fabs(x); }
template <typename T> __device__ __forceinline__ T amax4(const V4<T>& v) {
  return tmax(tmax(tabs(v.x), tabs(v.y)), tmax(tabs(v.z), tabs(v.w)));
}
template <typename T> __device__ __forceinline__ T absnan(T x) { return (x == x) ? tabs(x) : T(INFINITY); }

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

// Twelve stencil coefficients of one row (see stencil.cuh), already scaled.
// a1q0/a3q0 and a1q3/a3q3 are the centre-row coefficients of the thread's first
// and last column (the x-edge variants where that column is 0 or d-1).
template <typename T> struct RowCoef { T a0, a1, a2, a3, a4, b0, b1, b2, c0, c1, a1q0, a3q0, a1q3, a3q3; };

template <typename T, int D, int C, int NT, bool EULER>
__global__ void __launch_bounds__(NT, 1) engine_kernel(const EngineArgs a) {
  using K = Cfg<T, D, C, NT>;
  constexpr int RS = K::RS, W = K::W, NW = K::NW, R = K::R, TPR = K::TPR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* coef = sm + K::OFF_COEF;
  T* b0row = sm + K::OFF_B0;
  T* scale_tab = sm + K::OFF_SCALE;
  T* slots = sm + K::OFF_SLOT;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cb = tid % TPR;                 // column block
  const int i0 = 4 * cb;                    // first grid column of this thread
  const int j0 = (tid / TPR) * R;           // first local v-row of this thread
  int rank = 0;
  if constexpr (C > 1) rank = (int)cg::this_cluster().block_rank();
  const int r0 = rank * RS;                 // first global v-row of this CTA
  const int64_t cid = blockIdx.x / C, ncl = gridDim.x / C;
  const bool hasL = cb > 0, hasR = cb < TPR - 1;
  const bool ldsL = (TPR > 32) && (lane == 0) && hasL;     // left neighbour in another warp
  const bool ldsR = (TPR > 32) && (lane == 31) && hasR;
  const bool edgeL = !hasL, edgeR = !hasR;                 // thread holds column 0 / column d-1
  const T mL = hasL ? T(1) : T(0), mR = hasR ? T(1) : T(0);
  const double inv2dx = 0.5 / a.dx, inv4dx2 = 0.25 / (a.dx * a.dx);
  const T tol = sizeof(T) == 4 ? (T)a.tol32 : (T)a.tol64;

  // element offset of (local row p in [-2, RS+1], column c in [-4, D+3])
  auto at = [](int p, int c) -> int { return (p + 2) * W + c + 4; };

  // zero padding columns of every row, and the halo rows on the grid boundary, in both buffers
  for (int e = tid; e < 2 * K::ROWS * 8; e += NT) {
    const int b = e / (K::ROWS * 8), rem = e % (K::ROWS * 8), row = rem / 8, cc = rem % 8;
    sm[b * K::BUF + (size_t)row * W + (cc < 4 ? cc : D + cc)] = T(0);
  }
  for (int e = tid; e < 2 * 4 * D; e += NT) {
    const int b = e / (4 * D), rem = e % (4 * D), hr = rem / D, c = rem % D;
    const int p = hr < 2 ? hr - 2 : RS + (hr - 2);
    const int jg = r0 + p;
    if (jg < 0 || jg >= D) sm[b * K::BUF + at(p, c)] = T(0);
  }
  sync_all<C>();

  // For row p with own columns v: the centred x differences d1 = u(i+1) - u(i-1)
  // and the distance-two sums s2 = u(i+2) + u(i-2) of the thread's four columns.
  // The neighbour columns come from the adjacent threads by shuffles; across a
  // row boundary they lie outside the grid and a 0/1 factor fused into the
  // multiply-adds removes them; across a warp boundary they are read from
  // shared memory.
  auto xterms = [&](const V4<T>& v, const T* buf, int p, V4<T>& d1, V4<T>& s2) {
    T lz = __shfl_up_sync(0xffffffffu, v.z, 1), lw = __shfl_up_sync(0xffffffffu, v.w, 1);
    T rx = __shfl_down_sync(0xffffffffu, v.x, 1), ry = __shfl_down_sync(0xffffffffu, v.y, 1);
    if (ldsL) {
      lz = buf[at(p, i0 - 2)];
      lw = buf[at(p, i0 - 1)];
    }
    if (ldsR) {
      rx = buf[at(p, i0 + 4)];
      ry = buf[at(p, i0 + 5)];
    }
    d1.x = fma(-mL, lw, v.y);
    d1.y = v.z - v.x;
    d1.z = v.w - v.y;
    d1.w = fma(mR, rx, -v.z);
    s2.x = fma(mL, lz, v.z);
    s2.y = fma(mL, lw, v.w);
    s2.z = fma(mR, rx, v.x);
    s2.w = fma(mR, ry, v.y);
  };

  // store the four own columns of local row p into buffer b, and into the facing
  // halo row of the neighbouring CTA
  auto store_row = [&](int b, int p, const V4<T>& v) {
    st4(sm + b * K::BUF + at(p, i0), v);
    if constexpr (C > 1) {
      if (p < 2 && rank > 0) {
        T* peer = cg::this_cluster().map_shared_rank(sm, rank - 1);
        st4(peer + b * K::BUF + at(RS + p, i0), v);
      }
      if (p >= RS - 2 && rank < C - 1) {
        T* peer = cg::this_cluster().map_shared_rank(sm, rank + 1);
        st4(peer + b * K::BUF + at(p - RS, i0), v);
      }
    }
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
  auto publish = [&](int par, T mn, T ma) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      mn = tmax(mn, __shfl_xor_sync(0xffffffffu, mn, off));
      ma = tmax(ma, __shfl_xor_sync(0xffffffffu, ma, off));
    }
    if (lane == 0) {
      slots[(par * NW + warp) * 2 + 0] = mn;
      slots[(par * NW + warp) * 2 + 1] = ma;
    }
  };

  for (int64_t path = cid; path < a.paths; path += ncl) {
    V4<T> acc[R];
    int cur = 0, par = 0;
    // ---- initial datum: own rows, plus the halo rows facing other CTAs ----------
    T m0 = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double* src = a.u0 + (size_t)(r0 + j0 + r) * D + i0;
      acc[r] = {(T)src[0], (T)src[1], (T)src[2], (T)src[3]};
      st4(sm + at(j0 + r, i0), acc[r]);
      m0 = tmax(m0, tmax(tmax(absnan(acc[r].x), absnan(acc[r].y)), tmax(absnan(acc[r].z), absnan(acc[r].w))));
    }
    if (j0 == 0 || j0 + R == RS) {
      for (int h = 0; h < 2; ++h) {
        const int p = j0 == 0 ? h - 2 : RS + h;
        const int jg = r0 + p;
        if (jg >= 0 && jg < D) {
          const double* src = a.u0 + (size_t)jg * D + i0;
          st4(sm + at(p, i0), V4<T>{(T)src[0], (T)src[1], (T)src[2], (T)src[3]});
        }
      }
    }
    publish(par, m0, m0);
    sync_all<C>();
    T unorm, u0max;
    gather(par, unorm, u0max);
    par ^= 1;
    bool scale_cap = false;
    unsigned long long nmv = 0;

    for (int n = 0; n < a.steps; ++n) {
      // ---- this step's operator: coefficient tables and Taylor parameters ---------
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
        m_terms = min((int)rec[MSK_WT_M], kMaxTerms);
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
      for (int k = tid; k <= kMaxTerms; k += NT)
        scale_tab[k] = EULER ? T(1) : (T)(k == 0 ? 1.0 : 1.0 / ((double)s_steps * k));
      for (int jl = tid; jl < RS; jl += NT) b0row[jl] = (T)fold_b0(a.band, D, r0 + jl, w, inv2dx);
      __syncthreads();
      const T te = (T)eta;

      for (int sub = 0; sub < s_steps; ++sub) {
        T c1 = unorm;   // norm of the previous Taylor term (term 0 = the state)
        for (int k = 1; k <= m_terms; ++k) {
          const T sc = scale_tab[k];
          auto make = [&](const T* q) -> RowCoef<T> {
            const T a1 = q[CF_A + 1] * sc, a3 = q[CF_A + 3] * sc;
            const T e1 = q[CF_AE + 0] * sc, e3 = q[CF_AE + 1] * sc;
            return {q[CF_A + 0] * sc, a1, q[CF_A + 2] * sc, a3, q[CF_A + 4] * sc,
                    q[CF_B + 0] * sc, q[CF_B + 1] * sc, q[CF_B + 2] * sc, q[CF_C + 0] * sc, q[CF_C + 1] * sc,
                    edgeL ? e1 : a1, edgeL ? e3 : a3, edgeR ? e1 : a1, edgeR ? e3 : a3};
          };
          const RowCoef<T> ci = make(coef + 4 * MSK_NCOEF);
          const int nxt = cur ^ 1;
          const T* src = sm + cur * K::BUF;
          T mn = T(0), ma = T(0);
          // sliding window: own columns of rows j-2..j+2, x terms of rows j-1..j+1
          V4<T> cw0 = ld4(src + at(j0 - 2, i0)), cw1 = ld4(src + at(j0 - 1, i0));
          V4<T> cw2 = ld4(src + at(j0, i0)), cw3 = ld4(src + at(j0 + 1, i0));
          V4<T> d10, s20, d11, s21, d12, s22;
          xterms(cw1, src, j0 - 1, d10, s20);
          xterms(cw2, src, j0, d11, s21);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int p = j0 + r;
            const int jg = r0 + p;
            const V4<T> cw4 = ld4(src + at(p + 2, i0));
            xterms(cw3, src, p + 1, d12, s22);
            RowCoef<T> c = ci;
            if (is_special_row(jg, D)) c = make(coef + special_index(jg, D) * MSK_NCOEF);
            else c.b1 = b0row[p] * sc;
            V4<T> out;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const T a1 = q == 0 ? c.a1q0 : (q == 3 ? c.a1q3 : c.a1);
              const T a3 = q == 0 ? c.a3q0 : (q == 3 ? c.a3q3 : c.a3);
              T v = c.a0 * get(cw0, q);
              v = fma(a1, get(cw1, q), v);
              v = fma(c.a2, get(cw2, q), v);
              v = fma(a3, get(cw3, q), v);
              v = fma(c.a4, get(cw4, q), v);
              v = fma(c.b0, get(d10, q), v);
              v = fma(c.b1, get(d11, q), v);
              v = fma(c.b2, get(d12, q), v);
              v = fma(c.c0, get(s20, q), v);
              v = fma(c.c1, get(s22, q), v);
              set(out, q, v);
            }
            store_row(nxt, p, out);
            if constexpr (EULER) {
              acc[r] = out;
            } else {
              acc[r].x += out.x;
              acc[r].y += out.y;
              acc[r].z += out.z;
              acc[r].w += out.w;
              mn = tmax(mn, amax4(out));
              ma = tmax(ma, amax4(acc[r]));
            }
            cw0 = cw1; cw1 = cw2; cw2 = cw3; cw3 = cw4;
            d10 = d11; s20 = s21; d11 = d12; s21 = s22;
          }
          ++nmv;
          if constexpr (EULER) {
            sync_all<C>();
            cur = nxt;
            break;
          } else {
            publish(par, mn, ma);
            sync_all<C>();
            T gn, ga;
            gather(par, gn, ga);
            par ^= 1;
            cur = nxt;
            unorm = ga;
            if (c1 + gn <= tol * ga) break;
            c1 = gn;
          }
        }
        if constexpr (!EULER) {
          // u <- e^{mu/s} (partial sum), into the buffer not holding the last term
#pragma unroll
          for (int r = 0; r < R; ++r) {
            acc[r].x *= te;
            acc[r].y *= te;
            acc[r].z *= te;
            acc[r].w *= te;
            store_row(cur ^ 1, j0 + r, acc[r]);
          }
          unorm = unorm * te;
          sync_all<C>();
          cur ^= 1;
        }
      }
    }

    // ---- solution, work counter and path status ----------------------------------
    T mfin = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      st4(reinterpret_cast<T*>(a.out) + (size_t)path * D * D + (size_t)(r0 + j0 + r) * D + i0, acc[r]);
      mfin = tmax(mfin, tmax(tmax(absnan(acc[r].x), absnan(acc[r].y)), tmax(absnan(acc[r].z), absnan(acc[r].w))));
    }
    if (a.work && rank == 0 && tid == 0) atomicAdd(a.work, nmv);
    publish(par, mfin, mfin);
    sync_all<C>();
    T gfin, gfin2;
    gather(par, gfin, gfin2);
    par ^= 1;
    if (a.status && rank == 0 && tid == 0) {
      uint32_t st = 0;
      if (!(gfin < T(INFINITY))) st |= MSK_PATH_NONFINITE;
      if (scale_cap) st |= MSK_PATH_SCALE_CAP;
      if (!((double)gfin <= 10.0 * (double)u0max)) st |= MSK_PATH_BLOWUP;
      a.status[path] = st;
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
  return msk_cuda(ctx, cudaLaunchKernelEx(&cfg, kern, a), "engine launch");
}

template <bool EULER>
msk_status dispatch(msk_ctx* ctx, int precision, const EngineArgs& a, cudaStream_t s) {
  const int d = ctx->d;
  if (precision == MSK_F32) {
    switch (d) {
      case 32: return launch_one<float, 32, 1, 32, EULER>(ctx, a, s);
      case 64: return launch_one<float, 64, 1, 128, EULER>(ctx, a, s);
      case 128: return launch_one<float, 128, 1, 512, EULER>(ctx, a, s);
      case 256: return launch_one<float, 256, 4, 512, EULER>(ctx, a, s);
      case 512: return launch_one<float, 512, 16, 512, EULER>(ctx, a, s);
    }
  } else {
    switch (d) {
      case 32: return launch_one<double, 32, 1, 32, EULER>(ctx, a, s);
      case 64: return launch_one<double, 64, 1, 128, EULER>(ctx, a, s);
      case 128: return launch_one<double, 128, 2, 256, EULER>(ctx, a, s);
      case 256: return launch_one<double, 256, 8, 256, EULER>(ctx, a, s);
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
  a.T = ctx->T;
  a.s_cap = kMskScaleCap;
  a.tol32 = 0x1p-24f;
  a.tol64 = 0x1p-53;
  a.c = coef_dev(ctx->coef);
  return euler ? dispatch<true>(ctx, precision, a, stream) : dispatch<false>(ctx, precision, a, stream);
}

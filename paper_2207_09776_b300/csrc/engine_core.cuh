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
#pragma once

#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "stencil.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kMaxTerms = 128;  // >= the largest Taylor degree of either theta table

struct EngineArgs {
  const double* band;
  const double* u0;
  const double* Wt;   // Magnus: [paths][steps][MSK_NWT]
  const double* dW;   // Euler:  [paths][steps]
  void* out;          // [paths][d][d] of T; null: the final state is not stored
  // Snapshots for output times: at the start of step n (n = steps: after the
  // last step) the state is stored into snap[path][q] (T, d x d) for
  // q = snap_first[n] .. snap_first[n] + snap_cnt[n] - 1 (tables of steps + 1
  // entries); snap null: none.
  void* snap;
  const int* snap_first;
  const int* snap_cnt;
  int n_out;
  int u0_self;        // 1: each path starts from its own out[path] (T) instead of u0
  // Euler: per step alpha(t_n) dt and sigma(t_n) ([steps][2], double and float copies)
  const double* em_d;
  const float* em_f;
  uint32_t* status;
  unsigned long long* work;
  // Optional dynamic path queue (single-CTA configurations): CTAs take queue
  // positions q = 0, 1, ... by an atomic counter and solve path order[q]; order
  // lists the paths by decreasing estimated cost, so the last paths handed out
  // are the cheapest (longest-processing-time-first).  Null: static striding.
  const long long* order;
  unsigned long long* queue;
  int64_t qlen;       // entries of order handed out by the queue (0: paths)
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
  // Clustered slabs of 512 threads (and double ones) keep the Taylor partial sum
  // in shared memory ([RS][D], each thread's own points) instead of registers:
  // their halo-exchange code needs the registers, and the register-resident sum
  // spills there.  With 256 threads (255 registers each) a float sum fits.
  static constexpr bool ACC_SMEM = C > 1 && (NT > 256 || sizeof(T) == 8);
  // 2 x C x 2 CTA-level norm slots; each pair is written by one vector store
  // through the cluster, so the region starts on a 16-byte boundary
  static constexpr size_t OFF_CSLOT = (OFF_SLOT + 4 * NW + 3) / 4 * 4;
  // unit-weight tables (built once per path): the twelve coefficients of the five
  // row classes for each basis operator alone, and the V1 centre of each of the six
  // D^x-class operators per local row; a step's tables are their weighted sums
  static constexpr int NDX = 6;
  static constexpr size_t OFF_EU = OFF_CSLOT + 4 * C;              // MSK_NOPS x 5 x 12
  static_assert(OFF_CSLOT * sizeof(T) % 16 == 0, "cluster norm slots must be 16-byte aligned");
  static constexpr size_t OFF_BU = OFF_EU + (size_t)MSK_NOPS * 5 * MSK_NCOEF;   // NDX x RS
  static constexpr size_t OFF_END = OFF_BU + (size_t)NDX * RS;
  static constexpr size_t OFF_ACC = (OFF_END + 3) / 4 * 4;
  // Single-CTA slabs also keep each step's interior-row coefficients pre-scaled by
  // 1/(s k) for every term k (16 slots: the twelve coefficients, padded for vector
  // loads), so a Taylor term loads them instead of scaling them.
  static constexpr size_t OFF_KC = (OFF_END + 3) / 4 * 4;                 // (kMaxTerms + 1) x 16
  static constexpr size_t END_KTAB = OFF_KC + (size_t)(kMaxTerms + 1) * 16;
  static constexpr bool KTAB = !ACC_SMEM && END_KTAB * sizeof(T) <= 232448;
  static constexpr size_t NELEM = ACC_SMEM ? OFF_ACC + (size_t)RS * D : (KTAB ? END_KTAB : OFF_END);
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

// max(m, |v.x|, |v.y|, |v.z|, |v.w|): two three-input maxima in float (max.f32 with three
// operands), four two-input ones in double; NaN is ignored as by fmax.
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float accmax4(float m, const V4<float>& v) {
  return max3f(fabsf(v.x), fabsf(v.y), max3f(fabsf(v.z), fabsf(v.w), m));
}
__device__ __forceinline__ double accmax4(double m, const V4<double>& v) { return fmax(m, amax4(v)); }

// Warp maximum of non-negative values: for float one redux.sync on the bit patterns
// (non-negative floats order like their bit patterns), for double a shuffle tree.
__device__ __forceinline__ float warp_max_nonneg(float x) {
  return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(x)));
}
__device__ __forceinline__ double warp_max_nonneg(double x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, off));
  return x;
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

// Barrier policies of the engine: all threads of one CTA, all CTAs of a
// thread-block cluster, or one named barrier over a subset of a CTA's warps.
// operator() spans every thread that shares the slab; local() the threads of
// the calling CTA (or of the named group) that share the per-step tables.
// The D^x-class operators (their V1 centre varies over the interior rows).
__constant__ int c_dx_ops[6] = {MSK_OP_BX, MSK_OP_BX_A0, MSK_OP_BX_BVV, MSK_OP_BXA0_A0, MSK_OP_BXA0_BVV,
                                MSK_OP_BVVA0_BX};

struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
  __device__ __forceinline__ void local() const { __syncthreads(); }
};
// Distributed shared memory through explicit shared::cluster addresses (mapa):
// the same offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t dsmem_addr(const void* p, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void dsmem_st4(uint32_t addr, const V4<float>& v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void dsmem_st4(uint32_t addr, const V4<double>& v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(v.x), "d"(v.y) : "memory");
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr + 16u), "d"(v.z), "d"(v.w) : "memory");
}
__device__ __forceinline__ float dsmem_ld(uint32_t addr, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double dsmem_ld(uint32_t addr, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void dsmem_st2(uint32_t addr, float a, float b) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void dsmem_st2(uint32_t addr, double a, double b) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(a), "d"(b) : "memory");
}
__device__ __forceinline__ long long dsmem_ld_s64(uint32_t addr) {
  long long v;
  asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}

struct ClusterSync {
  __device__ __forceinline__ void operator()() const { cg::this_cluster().sync(); }
  __device__ __forceinline__ void local() const { __syncthreads(); }
};
struct NamedSync {
  int id, count;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
  }
  __device__ __forceinline__ void local() const { (*this)(); }
};

// Zero the padding columns of every row and the halo rows on the grid boundary
// in both buffers of a slab (done once per kernel, or per work unit when the
// shared-memory layout changes between units).
template <typename T, int D, int C, int NT, class Sync>
__device__ __forceinline__ void slab_init(T* sm, const int tid, const int rank, const Sync& sync_all) {
  using K = Cfg<T, D, C, NT>;
  constexpr int RS = K::RS, W = K::W;
  const int r0 = rank * RS;
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
  sync_all();
}

// One path: initial datum, all Magnus (or Euler) steps, output and status.
// sm is the slab's shared memory (the same offset in every CTA of a cluster),
// tid the thread index within the threads that share `sync_all`, rank the
// CTA's index within the cluster (0 when C = 1).
template <typename T, int D, int C, int NT, bool EULER, class Sync>
__device__ __forceinline__ void solve_path(const EngineArgs& a, int64_t path, T* sm, const int tid,
                                           const int rank, const Sync& sync_all) {
  using K = Cfg<T, D, C, NT>;
  constexpr int RS = K::RS, W = K::W, NW = K::NW, R = K::R, TPR = K::TPR;
  T* coef = sm + K::OFF_COEF;
  T* b0row = sm + K::OFF_B0;
  T* scale_tab = sm + K::OFF_SCALE;
  T* slots = sm + K::OFF_SLOT;

  const int lane = tid & 31, warp = tid >> 5;
  const int cb = tid % TPR;                 // column block
  const int i0 = 4 * cb;                    // first grid column of this thread
  const int j0 = (tid / TPR) * R;           // first local v-row of this thread
  const int r0 = rank * RS;                 // first global v-row of this CTA
  const bool hasL = cb > 0, hasR = cb < TPR - 1;
  const bool ldsL = (TPR > 32) && (lane == 0) && hasL;     // left neighbour in another warp
  const bool ldsR = (TPR > 32) && (lane == 31) && hasR;
  const bool edgeL = !hasL, edgeR = !hasR;                 // thread holds column 0 / column d-1
  const bool top_strip = r0 + j0 == 0, bot_strip = r0 + j0 + R == D;   // strip holds grid rows 0, 1 / d-2, d-1
  const T mL = hasL ? T(1) : T(0), mR = hasR ? T(1) : T(0);
  const double inv2dx = 0.5 / a.dx, inv4dx2 = 0.25 / (a.dx * a.dx);
  const T tol = sizeof(T) == 4 ? (T)a.tol32 : (T)a.tol64;

  // element offset of (local row p in [-2, RS+1], column c in [-4, D+3])
  auto at = [](int p, int c) -> int { return (p + 2) * W + c + 4; };


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
  // halo row of the neighbouring CTA (shared::cluster stores)
  const uint32_t peer_lo = (C > 1 && rank > 0) ? dsmem_addr(sm, rank - 1) : 0u;
  const uint32_t peer_hi = (C > 1 && rank < C - 1) ? dsmem_addr(sm, rank + 1) : 0u;
  auto store_row = [&](int b, int p, const V4<T>& v) {
    st4(sm + b * K::BUF + at(p, i0), v);
    if constexpr (C > 1) {
      if (p < 2 && rank > 0) dsmem_st4(peer_lo + (uint32_t)((b * K::BUF + at(RS + p, i0)) * sizeof(T)), v);
      if (p >= RS - 2 && rank < C - 1)
        dsmem_st4(peer_hi + (uint32_t)((b * K::BUF + at(p - RS, i0)) * sizeof(T)), v);
    }
  };

  // Norms: every warp publishes its maxima; with clusters, warp 0 of each CTA
  // folds them into one CTA-level pair (after a CTA barrier) and pushes it into
  // slot `rank` of every CTA of the cluster (lane l stores to CTA l: remote
  // stores, off the critical path), so after the cluster barrier every warp reads
  // the C pairs from its own shared memory.  The result is identical in every
  // thread of the cluster.  Slots alternate by parity: a CTA already in the next
  // term writes the other parity, and cannot reach the one after before every CTA
  // has passed the barrier that follows these reads.
  T* cslot = sm + K::OFF_CSLOT;   // [2][C][2]
  auto gather = [&](int par, T& gn, T& ga) {
    gn = T(0);
    ga = T(0);
    if constexpr (C > 1) {
      if (lane < C) {
        gn = cslot[(par * C + lane) * 2 + 0];
        ga = cslot[(par * C + lane) * 2 + 1];
      }
    } else {
      for (int q = lane; q < NW; q += 32) {
        gn = tmax(gn, slots[(par * NW + q) * 2 + 0]);
        ga = tmax(ga, slots[(par * NW + q) * 2 + 1]);
      }
    }
    gn = warp_max_nonneg(gn);
    ga = warp_max_nonneg(ga);
  };
  auto publish = [&](int par, T mn, T ma) {
    mn = warp_max_nonneg(mn);
    ma = warp_max_nonneg(ma);
    if (lane == 0) {
      slots[(par * NW + warp) * 2 + 0] = mn;
      slots[(par * NW + warp) * 2 + 1] = ma;
    }
    if constexpr (C > 1) {
      sync_all.local();
      if (warp == 0) {
        T a = T(0), b = T(0);
        for (int q = lane; q < NW; q += 32) {
          a = tmax(a, slots[(par * NW + q) * 2 + 0]);
          b = tmax(b, slots[(par * NW + q) * 2 + 1]);
        }
        a = warp_max_nonneg(a);
        b = warp_max_nonneg(b);
        if (lane < C) dsmem_st2(dsmem_addr(cslot + (par * C + rank) * 2, lane), a, b);
      }
    }
  };

  {
    // partial sum of the Taylor series (and the state between steps): registers
    // or, for clustered slabs, shared memory at the thread's own points
    constexpr bool AS = K::ACC_SMEM;
    V4<T> accr[AS ? 1 : R];
    T* accS = sm + K::OFF_ACC;
    auto acc_get = [&](int r) -> V4<T> {
      if constexpr (AS) return ld4(accS + (size_t)(j0 + r) * D + i0);
      else return accr[r];
    };
    auto acc_put = [&](int r, const V4<T>& v) {
      if constexpr (AS) st4(accS + (size_t)(j0 + r) * D + i0, v);
      else accr[r] = v;
    };
    int cur = 0, par = 0;
    // ---- initial datum: own rows, plus the halo rows facing other CTAs ----------
    T m0 = T(0);
    // own points of the initial datum (u0, or the path's own output slot)
    const T* self0 = a.u0_self ? reinterpret_cast<const T*>(a.out) + (size_t)path * D * D : nullptr;
    auto load0 = [&](int jg) -> V4<T> {
      if (self0) return ld4(self0 + (size_t)jg * D + i0);
      const double* src = a.u0 + (size_t)jg * D + i0;
      return V4<T>{(T)src[0], (T)src[1], (T)src[2], (T)src[3]};
    };
    for (int r = 0; r < R; ++r) {
      const V4<T> v = load0(r0 + j0 + r);
      acc_put(r, v);
      st4(sm + at(j0 + r, i0), v);
      m0 = tmax(m0, tmax(tmax(absnan(v.x), absnan(v.y)), tmax(absnan(v.z), absnan(v.w))));
    }
    if (j0 == 0 || j0 + R == RS) {
      for (int h = 0; h < 2; ++h) {
        const int p = j0 == 0 ? h - 2 : RS + h;
        const int jg = r0 + p;
        if (jg >= 0 && jg < D) st4(sm + at(p, i0), load0(jg));
      }
    }
    publish(par, m0, m0);
    sync_all();
    T unorm, u0max;
    gather(par, unorm, u0max);
    par ^= 1;
    bool scale_cap = false;
    unsigned long long nmv = 0;
    const T dtT = (T)(a.T / a.steps);

    // ---- unit-weight tables of this context (see Cfg::OFF_EU) ---------------------
    {
      T* eu = sm + K::OFF_EU;
      T* bu = sm + K::OFF_BU;
      for (int e = tid; e < MSK_NOPS * 5; e += NT) {
        const int k = e / 5, r = e % 5;
        const int jr = r < 4 ? special_row(r, D) : 2;
        double wv[MSK_NOPS];
        for (int q = 0; q < MSK_NOPS; ++q) wv[q] = q == k ? 1.0 : 0.0;
        double cf[MSK_NCOEF];
        fold_row(a.band, D, jr, wv, 0.0, inv2dx, inv4dx2, cf);
        for (int q = 0; q < MSK_NCOEF; ++q) eu[(size_t)e * MSK_NCOEF + q] = (T)cf[q];
      }
      for (int e = tid; e < K::NDX * RS; e += NT) {
        const int c = e / RS, jl = e % RS;
        bu[e] = (T)(a.band[((size_t)c_dx_ops[c] * D + r0 + jl) * MSK_BAND + 2] * inv2dx);
      }
      sync_all.local();
    }

    // snapshots of the state at the start of step n (n = steps: the final state)
    auto snapshot = [&](int n) {
      if (!a.snap) return;
      const int q0 = a.snap_first[n], nq = a.snap_cnt[n];
      for (int q = q0; q < q0 + nq; ++q) {
        T* dst = reinterpret_cast<T*>(a.snap) + ((size_t)path * a.n_out + q) * D * D;
#pragma unroll
        for (int r = 0; r < R; ++r) st4(dst + (size_t)(r0 + j0 + r) * D + i0, acc_get(r));
      }
    };

    for (int n = 0; n < a.steps; ++n) {
      snapshot(n);
      // ---- this step's operator: coefficient tables and Taylor parameters ---------
      // The step's weights in the working precision: lane k (< 13) of every warp
      // converts weight k and lane 13 the diagonal shift (one conversion per warp);
      // shuffles broadcast them.  The tables are the weighted sums of the unit
      // tables (no double arithmetic per step on the slow double pipe).
      int s_steps = 1, m_terms = 1;
      double mu = 0.0;
      T wl = T(0);
      if constexpr (EULER) {
        const T* em = sizeof(T) == 4 ? reinterpret_cast<const T*>(a.em_f) : reinterpret_cast<const T*>(a.em_d);
        if (lane == MSK_OP_BX) wl = dtT;
        else if (lane == MSK_OP_BVV) wl = em[2 * n];                                   // alpha(t_n) dt
        else if (lane == MSK_OP_A0) wl = em[2 * n + 1] * (T)a.dW[path * a.steps + n];   // sigma(t_n) dW_n
        else if (lane == MSK_NOPS) wl = T(1);                                           // I + ...
      } else {
        // lanes 14, 15 carry s and m (exact in float: s <= 2^14, m <= 128)
        const double* rec = a.Wt + ((size_t)path * a.steps + n) * MSK_NWT;
        if (lane < MSK_NOPS) wl = (T)rec[lane];
        else if (lane == MSK_NOPS) wl = (T)(-rec[MSK_WT_MU]);
        else if (lane == MSK_NOPS + 1) wl = (T)rec[MSK_WT_S];
        else if (lane == MSK_NOPS + 2) wl = (T)rec[MSK_WT_M];
      }
      T wT[MSK_NOPS + 1];
#pragma unroll
      for (int k = 0; k <= MSK_NOPS; ++k) wT[k] = __shfl_sync(0xffffffffu, wl, k);
      if constexpr (!EULER) {
        const T sv = __shfl_sync(0xffffffffu, wl, MSK_NOPS + 1), mv = __shfl_sync(0xffffffffu, wl, MSK_NOPS + 2);
        s_steps = (int)sv;
        m_terms = min((int)mv, kMaxTerms);
        if (sv >= (T)a.s_cap) scale_cap = true;
        mu = -(double)wT[MSK_NOPS];
      }
      for (int q = tid; q < 5 * MSK_NCOEF; q += NT) {
        const T* e = sm + K::OFF_EU + q;
        T v = (q % MSK_NCOEF == CF_A + 2) ? wT[MSK_NOPS] : T(0);
#pragma unroll
        for (int k = 0; k < MSK_NOPS; ++k) v = fma(wT[k], e[k * 5 * MSK_NCOEF], v);
        coef[q] = v;
      }
      for (int k = tid; k <= kMaxTerms; k += NT)
        scale_tab[k] = (EULER || k == 0) ? T(1) : T(1) / ((T)s_steps * (T)k);
      {
        constexpr int dx[K::NDX] = {MSK_OP_BX, MSK_OP_BX_A0, MSK_OP_BX_BVV, MSK_OP_BXA0_A0, MSK_OP_BXA0_BVV,
                                    MSK_OP_BVVA0_BX};   // the D^x-class operators
        const T* bu = sm + K::OFF_BU;
        for (int jl = tid; jl < RS; jl += NT) {
          T v = T(0);
#pragma unroll
          for (int c = 0; c < K::NDX; ++c) v = fma(wT[dx[c]], bu[c * RS + jl], v);
          b0row[jl] = v;
        }
      }
      sync_all.local();
      if constexpr (K::KTAB && !EULER) {
        // the step's coefficients scaled for each term k = 1 .. m
        T* kc = sm + K::OFF_KC;
        for (int e = tid; e < (m_terms + 1) * 16; e += NT) {
          const int k = e >> 4, q = e & 15;
          kc[e] = q < MSK_NCOEF ? coef[4 * MSK_NCOEF + q] * scale_tab[k] : T(0);
        }
        sync_all.local();
      }
      T te = T(1);
      if constexpr (!EULER) {
        if constexpr (sizeof(T) == 4) te = (T)expf(-(float)wT[MSK_NOPS] / (float)s_steps);
        else te = (T)exp(mu / s_steps);
      }

      for (int sub = 0; sub < s_steps; ++sub) {
        T c1 = unorm;   // norm of the previous Taylor term (term 0 = the state)
        // the first four window rows of the next term are loaded right after the
        // barrier, before the termination test (wasted only when the series stops)
        V4<T> pw0, pw1, pw2, pw3;
        {
          const T* src = sm + cur * K::BUF;
          pw0 = ld4(src + at(j0 - 2, i0));
          pw1 = ld4(src + at(j0 - 1, i0));
          pw2 = ld4(src + at(j0, i0));
          pw3 = ld4(src + at(j0 + 1, i0));
        }
        for (int k = 1; k <= m_terms; ++k) {
          const T sc = scale_tab[k];
          auto make = [&](const T* q) -> RowCoef<T> {
            const T a1 = q[CF_A + 1] * sc, a3 = q[CF_A + 3] * sc;
            const T e1 = q[CF_AE + 0] * sc, e3 = q[CF_AE + 1] * sc;
            return {q[CF_A + 0] * sc, a1, q[CF_A + 2] * sc, a3, q[CF_A + 4] * sc,
                    q[CF_B + 0] * sc, q[CF_B + 1] * sc, q[CF_B + 2] * sc, q[CF_C + 0] * sc, q[CF_C + 1] * sc,
                    edgeL ? e1 : a1, edgeL ? e3 : a3, edgeR ? e1 : a1, edgeR ? e3 : a3};
          };
          RowCoef<T> ci;
          if constexpr (K::KTAB && !EULER) {
            const T* kc = sm + K::OFF_KC + k * 16;
            const V4<T> q0 = ld4(kc), q1 = ld4(kc + 4), q2 = ld4(kc + 8);
            ci = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y,
                  edgeL ? q2.z : q0.y, edgeL ? q2.w : q0.w, edgeR ? q2.z : q0.y, edgeR ? q2.w : q0.w};
          } else {
            ci = make(coef + 4 * MSK_NCOEF);
          }
          const int nxt = cur ^ 1;
          const T* src = sm + cur * K::BUF;
          T mn = T(0), ma = T(0);
          // sliding window: own columns of rows j-2..j+2, x terms of rows j-1..j+1
          V4<T> cw0 = pw0, cw1 = pw1, cw2 = pw2, cw3 = pw3;
          V4<T> d10, s20, d11, s21, d12, s22;
          xterms(cw1, src, j0 - 1, d10, s20);
          xterms(cw2, src, j0, d11, s21);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int p = j0 + r;
            const V4<T> cw4 = ld4(src + at(p + 2, i0));
            xterms(cw3, src, p + 1, d12, s22);
            auto stencil = [&](const RowCoef<T>& c) -> V4<T> {
              V4<T> o;
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
                set(o, q, v);
              }
              return o;
            };
            // The four boundary rows (rows of two warps at most, the branch is warp-uniform)
            // take their own coefficient set; every other row the interior set with its own
            // V1 centre.  Two separate evaluations keep the interior path free of selects.
            // With r a compile-time index, rows 2 .. R-3 of a strip never test anything: only
            // the first two rows of the top strip and the last two of the bottom strip are
            // boundary rows (precomputed per thread), and their class index is a constant.
            V4<T> out;
            const bool special = (r < 2 && top_strip) || (r >= R - 2 && bot_strip);
            if (__builtin_expect(special, 0)) {
              out = stencil(make(coef + (r < 2 && top_strip ? r : 4 - R + r) * MSK_NCOEF));
            } else {
              RowCoef<T> c = ci;
              c.b1 = b0row[p] * sc;
              out = stencil(c);
            }
            store_row(nxt, p, out);
            if constexpr (EULER) {
              acc_put(r, out);
            } else {
              V4<T> ac = acc_get(r);
              ac.x += out.x;
              ac.y += out.y;
              ac.z += out.z;
              ac.w += out.w;
              acc_put(r, ac);
              mn = accmax4(mn, out);
              ma = accmax4(ma, ac);
            }
            cw0 = cw1; cw1 = cw2; cw2 = cw3; cw3 = cw4;
            d10 = d11; s20 = s21; d11 = d12; s21 = s22;
          }
          ++nmv;
          if constexpr (EULER) {
            sync_all();
            cur = nxt;
            break;
          } else {
            publish(par, mn, ma);
            sync_all();
            {
              const T* srcn = sm + nxt * K::BUF;
              pw0 = ld4(srcn + at(j0 - 2, i0));
              pw1 = ld4(srcn + at(j0 - 1, i0));
              pw2 = ld4(srcn + at(j0, i0));
              pw3 = ld4(srcn + at(j0 + 1, i0));
            }
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
            V4<T> ac = acc_get(r);
            ac.x *= te;
            ac.y *= te;
            ac.z *= te;
            ac.w *= te;
            acc_put(r, ac);
            store_row(cur ^ 1, j0 + r, ac);
          }
          unorm = unorm * te;
          sync_all();
          cur ^= 1;
        }
      }
    }

    snapshot(a.steps);
    // ---- solution, work counter and path status ----------------------------------
    T mfin = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const V4<T> v = acc_get(r);
      if (a.out) st4(reinterpret_cast<T*>(a.out) + (size_t)path * D * D + (size_t)(r0 + j0 + r) * D + i0, v);
      mfin = tmax(mfin, tmax(tmax(absnan(v.x), absnan(v.y)), tmax(absnan(v.z), absnan(v.w))));
    }
    if (a.work && rank == 0 && tid == 0) atomicAdd(a.work, nmv);
    publish(par, mfin, mfin);
    sync_all();
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
    sync_all();   // nobody may still read this path's buffers or slots
  }
}


}  // namespace

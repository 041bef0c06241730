// S5b/S6 for grids whose state does not stay on chip: the streamed engine.
//
// Iterated Magnus (Section 2, "Iterated Magnus expansion") with the same scaled,
// truncated Taylor action as the resident engine (engine_core.cuh): on each
// step U <- e^{mu} (T_m((Omega - mu I)/s))^s U, the terms t_k = (Omega - mu I)
// t_{k-1} / (s k) folded-stencil matvecs (stencil.cuh), the series stopped when
// two consecutive terms fall below the tolerance relative to the partial sum.
//
// Data layout.  One CTA solves one path at a time.  The path's partial sum
// lives in its output slot out[path] ([v][x], HBM), the current Taylor term in
// one of two per-CTA scratch grids; nothing of the path stays on chip between
// passes.  A pass sweeps the grid once, top to bottom, in blocks of RT rows and
// evaluates LV consecutive Taylor terms on the way (temporal blocking): level 0
// is the term read from HBM, level L the term k + L, and level L works on block
// tau - L while level 0 reads block tau, so every level finds the rows of the
// level below it (its block and two halo rows on each side) in shared memory.
// Each level keeps a ring of 2 RT + 4 rows in shared memory (rows outside the
// grid are zero rows: Dirichlet, written into the ring with the last block).  Per pass and grid point the HBM traffic is
// one read of the term, one read and one write of the partial sum and one
// write of the last level's term: 16 bytes in float for LV terms.
//
// Thread mapping.  A thread owns four consecutive columns and RS consecutive
// rows of every block (RT = RS x the number of row strips).  Because the lag
// between levels is one whole block, a grid point is always evaluated by the
// same thread at every level of a pass, so the partial sum of the blocks in
// flight (LV of them) stays in that thread's registers: it is read from HBM
// once before level 1 and written once after the last level.  x-neighbours come
// from warp shuffles (shared memory across a warp boundary), as in the resident
// engine.
//
// Early termination is decided once per pass from the norms of each level's
// term and partial sum (reduced over the CTA at the pass end): terms past the
// stopping point that the pass already evaluated stay in the sum (each is
// below the tolerance), so the result differs from the resident engine's by
// less than the tolerance.
#include <utility>

#include "engine_core.cuh"

extern const double kMskScaleCap;

namespace {

template <typename T, int D, int NT, int LV, int RS>
struct SCfg {
  static constexpr int TPR = D / 4;          // threads per grid row
  static constexpr int NG = NT / TPR;        // row strips of a block
  static constexpr int RT = NG * RS;         // rows per block
  static constexpr int NB = D / RT;          // blocks per sweep
  static constexpr int W = D + 8;            // ring row: four zero columns each side
  static constexpr int RR = 2 * RT + 4;      // ring rows alive at once (with the two zero rows past the grid)
  static constexpr int NW = NT / 32;
  static constexpr int NRED = 2 * LV + 1;    // norms per pass: input, then (term, sum) per level
  static_assert(D % 32 == 0 && TPR >= 32 && TPR % 32 == 0, "rows must span whole warps");
  static_assert(NT % TPR == 0 && D % RT == 0, "blocks must tile the grid");
  static constexpr size_t RING = (size_t)RR * W;
  static constexpr size_t OFF_COEF = LV * RING;                    // 5 x 12 unscaled row classes
  static constexpr size_t OFF_KC = OFF_COEF + 5 * MSK_NCOEF;       // LV x 16: interior set per level
  static constexpr size_t OFF_B0 = OFF_KC + (size_t)LV * 16;       // D: V1 centre per row (unscaled)
  static constexpr size_t OFF_RED = OFF_B0 + D;                    // NW x NRED
  static constexpr size_t OFF_SC = OFF_RED + (size_t)NW * NRED;    // LV + 1: 1 / (s (k + L))
  static constexpr size_t NELEM = OFF_SC + LV + 1;
  static constexpr size_t OFF_PATH = (NELEM * sizeof(T) + 15) / 16 * 16;   // bytes: next path
  static constexpr size_t SMEM = OFF_PATH + 16;
  static_assert((OFF_KC * sizeof(T)) % 16 == 0 && (RING * sizeof(T)) % 16 == 0, "vector alignment");
  static_assert(SMEM <= 232448, "rings do not fit the 227 KB of shared memory");
};

struct StreamArgs {
  EngineArgs e;
  void* scratch;   // per CTA: two d x d grids of T (the current and the next Taylor term)
};

template <int... I, class F>
__device__ __forceinline__ void static_for_impl(std::integer_sequence<int, I...>, F&& f) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(std::make_integer_sequence<int, N>{}, f);
}

template <typename T, int D, int NT, int LV, int RS>
__global__ void __launch_bounds__(NT, 1) stream_engine_kernel(const StreamArgs sa) {
  using K = SCfg<T, D, NT, LV, RS>;
  constexpr int RT = K::RT, NB = K::NB, W = K::W, RR = K::RR, TPR = K::TPR, NW = K::NW, NRED = K::NRED;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* coef = sm + K::OFF_COEF;
  T* kc = sm + K::OFF_KC;
  T* b0row = sm + K::OFF_B0;
  T* red = sm + K::OFF_RED;
  T* sct = sm + K::OFF_SC;
  volatile long long* next_path = reinterpret_cast<long long*>(smem_raw + K::OFF_PATH);
  const EngineArgs& a = sa.e;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = tid / TPR, cb = tid % TPR, i0 = 4 * cb;
  const bool hasL = cb > 0, hasR = cb < TPR - 1;
  const bool ldsL = lane == 0 && hasL, ldsR = lane == 31 && hasR;   // neighbour column in another warp
  const bool edgeL = !hasL, edgeR = !hasR;
  const T mL = hasL ? T(1) : T(0), mR = hasR ? T(1) : T(0);
  const double inv2dx = 0.5 / a.dx, inv4dx2 = 0.25 / (a.dx * a.dx);
  const T tol = sizeof(T) == 4 ? (T)a.tol32 : (T)a.tol64;
  const size_t DD = (size_t)D * D;
  T* tbuf0 = reinterpret_cast<T*>(sa.scratch) + (size_t)blockIdx.x * 2 * DD;
  T* tbuf1 = tbuf0 + DD;

  auto ring = [&](int L) -> T* { return sm + (size_t)L * K::RING; };
  auto slot_of = [](int j) -> int { return (j + 2 * RR) % RR; };   // j >= -2
  auto rowp = [&](T* rg, int j) -> T* { return rg + (size_t)slot_of(j) * W + 4; };

  // x terms of a row (see engine_core.cuh): d1 = u(i+1) - u(i-1), s2 = u(i+2) + u(i-2)
  auto xterms = [&](const V4<T>& v, const T* row, V4<T>& d1, V4<T>& s2) {
    T lz = __shfl_up_sync(0xffffffffu, v.z, 1), lw = __shfl_up_sync(0xffffffffu, v.w, 1);
    T rx = __shfl_down_sync(0xffffffffu, v.x, 1), ry = __shfl_down_sync(0xffffffffu, v.y, 1);
    if (ldsL) {
      lz = row[i0 - 2];
      lw = row[i0 - 1];
    }
    if (ldsR) {
      rx = row[i0 + 4];
      ry = row[i0 + 5];
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
  auto make = [&](const T* q, T sc) -> RowCoef<T> {
    const T a1 = q[CF_A + 1] * sc, a3 = q[CF_A + 3] * sc;
    const T e1 = q[CF_AE + 0] * sc, e3 = q[CF_AE + 1] * sc;
    return {q[CF_A + 0] * sc, a1, q[CF_A + 2] * sc, a3, q[CF_A + 4] * sc,
            q[CF_B + 0] * sc, q[CF_B + 1] * sc, q[CF_B + 2] * sc, q[CF_C + 0] * sc, q[CF_C + 1] * sc,
            edgeL ? e1 : a1, edgeL ? e3 : a3, edgeR ? e1 : a1, edgeR ? e3 : a3};
  };
  // block-wide maxima of NRED non-negative values (every thread gets all of them)
  auto reduce_norms = [&](T (&v)[NRED]) {
#pragma unroll
    for (int q = 0; q < NRED; ++q) {
      const T m = warp_max_nonneg(v[q]);
      if (lane == 0) red[warp * NRED + q] = m;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NRED; ++q) {
      T m = T(0);
      for (int w = 0; w < NW; ++w) m = tmax(m, red[w * NRED + q]);
      v[q] = m;
    }
    __syncthreads();
  };

  // the zero columns of every ring row are written once
  for (int e = tid; e < LV * RR * 8; e += NT) {
    const int row = e / 8, c = e % 8;
    sm[(size_t)row * W + (c < 4 ? c : D + c)] = T(0);
  }

  long long spath = blockIdx.x;   // static striding when there is no queue
  for (;; spath += gridDim.x) {
    // ---- next path: cost-ordered queue (longest first), or static striding ---------
    long long path = spath;
    if (a.queue) {
      if (tid == 0) {
        const unsigned long long q = atomicAdd(a.queue, 1ull);
        *next_path = q < (unsigned long long)(a.qlen > 0 ? a.qlen : a.paths) ? a.order[q] : -1;
      }
      __syncthreads();
      path = *next_path;
      __syncthreads();   // nobody rewrites the slot before every thread has read it
    }
    if (path < 0 || path >= a.paths) break;

    T* acc_g = reinterpret_cast<T*>(a.out) + (size_t)path * DD;   // partial sum / state
    // ---- initial datum into the output slot; its maximum for the blow-up flag --------
    T u0max = T(0);
    for (size_t e = (size_t)tid * 4; e < DD; e += (size_t)NT * 4) {
      const double* src = a.u0 + e;
      const V4<T> v{(T)src[0], (T)src[1], (T)src[2], (T)src[3]};
      st4(acc_g + e, v);
      u0max = tmax(u0max, tmax(tmax(absnan(v.x), absnan(v.y)), tmax(absnan(v.z), absnan(v.w))));
    }
    {
      T v[NRED];
      v[0] = u0max;
#pragma unroll
      for (int q = 1; q < NRED; ++q) v[q] = T(0);
      reduce_norms(v);   // its barriers also order the stores above before the first pass
      u0max = v[0];
    }
    bool scale_cap = false;
    unsigned long long nmv = 0;
    T acc_scale = T(1);   // pending factor e^{mu/s} of the partial sum (applied when read)

    for (int n = 0; n < a.steps; ++n) {
      // ---- this step's operator: row-class coefficients and the V1 centres ----------
      const double* rec = a.Wt + ((size_t)path * a.steps + n) * MSK_NWT;
      const double mu = rec[MSK_WT_MU];
      const int s_steps = (int)rec[MSK_WT_S];
      const int m_terms = min((int)rec[MSK_WT_M], kMaxTerms);
      if (rec[MSK_WT_S] >= a.s_cap) scale_cap = true;
      if (tid < 5) {
        const int jr = tid < 4 ? special_row(tid, D) : 2;
        double cf[MSK_NCOEF];
        fold_row(a.band, D, jr, rec, -mu, inv2dx, inv4dx2, cf);
        for (int q = 0; q < MSK_NCOEF; ++q) coef[tid * MSK_NCOEF + q] = (T)cf[q];
      }
      for (int j = tid; j < D; j += NT) b0row[j] = (T)fold_b0(a.band, D, j, rec, inv2dx);
      T te;
      if constexpr (sizeof(T) == 4) te = expf((float)mu / (float)s_steps);
      else te = exp(mu / s_steps);
      __syncthreads();

      for (int sub = 0; sub < s_steps; ++sub) {
        int k = 0;          // terms of this sub-step evaluated so far
        T c1 = T(0);        // norm of the previous term (term 0: the state)
        bool done = false;
        bool first = true;  // the first pass reads the state (the partial sum) as term 0
        int in_buf = 0;     // later passes read the term from tbuf[in_buf]
        while (!done) {
          const int Lp = min(LV, m_terms - k);
          T* const in_g = first ? acc_g : (in_buf ? tbuf1 : tbuf0);
          T* const out_g = in_buf ? tbuf0 : tbuf1;     // the last level's term
          const T in_scale = first ? acc_scale : T(1);
          // pass set-up: per-level scales and interior coefficients, zero rows -2, -1
          if (tid <= LV) sct[tid] = (tid == 0 || tid > Lp) ? T(0) : T(1) / ((T)s_steps * (T)(k + tid));
          __syncthreads();
          for (int e = tid; e < LV * 16; e += NT) {
            const int L = e / 16, q = e % 16;
            kc[e] = q < MSK_NCOEF ? coef[4 * MSK_NCOEF + q] * sct[L + 1] : T(0);
          }
          for (int e = tid; e < LV * 2 * TPR; e += NT) {
            const int L = e / (2 * TPR), r = (e / TPR) % 2, c = e % TPR;
            st4(rowp(ring(L), r - 2) + 4 * c, V4<T>{T(0), T(0), T(0), T(0)});
          }
          T nin = T(0), nt[LV + 1], na[LV + 1];
#pragma unroll
          for (int L = 0; L <= LV; ++L) nt[L] = na[L] = T(0);
          V4<T> acc[LV][RS];
          V4<T> tpf[RS], apf[RS];
          // prefetch block 0 of the term
#pragma unroll
          for (int r = 0; r < RS; ++r) tpf[r] = ld4(in_g + (size_t)(g * RS + r) * D + i0);
          __syncthreads();

          // one time step: block tau of level 0, block tau - L of level L
          auto step = [&](int tau, auto Uc) {
            constexpr int U = decltype(Uc)::value;
            if (tau < NB) {
              T* r0 = ring(0);
#pragma unroll
              for (int r = 0; r < RS; ++r) {
                V4<T> v = tpf[r];
                v.x *= in_scale;
                v.y *= in_scale;
                v.z *= in_scale;
                v.w *= in_scale;
                st4(rowp(r0, tau * RT + g * RS + r) + i0, v);
                nin = accmax4(nin, v);
              }
              if (tau == NB - 1 && g == 0) {
                st4(rowp(r0, D) + i0, V4<T>{T(0), T(0), T(0), T(0)});
                st4(rowp(r0, D + 1) + i0, V4<T>{T(0), T(0), T(0), T(0)});
              }
            }
            // partial sum of block tau - 1 into its register slot (level 1 starts it now)
            if (tau >= 1 && tau - 1 < NB) {
              constexpr int S = (U + LV - 1) % LV;
#pragma unroll
              for (int r = 0; r < RS; ++r) {
                V4<T> v;
                if (first) v = ld4(rowp(ring(0), (tau - 1) * RT + g * RS + r) + i0);   // already scaled
                else {
                  v = apf[r];
                  v.x *= acc_scale;
                  v.y *= acc_scale;
                  v.z *= acc_scale;
                  v.w *= acc_scale;
                }
                acc[S][r] = v;
              }
            }
            // prefetch: term block tau + 1, partial-sum block tau
            if (tau + 1 < NB) {
#pragma unroll
              for (int r = 0; r < RS; ++r) tpf[r] = ld4(in_g + (size_t)((tau + 1) * RT + g * RS + r) * D + i0);
            }
            if (!first && tau < NB) {
#pragma unroll
              for (int r = 0; r < RS; ++r) apf[r] = ld4(acc_g + (size_t)(tau * RT + g * RS + r) * D + i0);
            }
            __syncthreads();
            static_for<LV>([&](auto Lc) {
              constexpr int L = decltype(Lc)::value + 1;
              if (L > Lp) return;
              const int b = tau - L;
              if (b >= 0 && b < NB) {
                constexpr int S = (U + LV - L % LV) % LV;
                T* src = ring(L - 1);
                T* dst = L < Lp ? ring(L < LV ? L : 0) : nullptr;
                const T sc = sct[L];
                RowCoef<T> ci;
                {
                  const T* q = kc + (L - 1) * 16;
                  const V4<T> q0 = ld4(q), q1 = ld4(q + 4), q2 = ld4(q + 8);
                  ci = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y,
                        edgeL ? q2.z : q0.y, edgeL ? q2.w : q0.w, edgeR ? q2.z : q0.y, edgeR ? q2.w : q0.w};
                }
                const int j0 = b * RT + g * RS;
                V4<T> cw0 = ld4(rowp(src, j0 - 2) + i0), cw1 = ld4(rowp(src, j0 - 1) + i0);
                V4<T> cw2 = ld4(rowp(src, j0) + i0), cw3 = ld4(rowp(src, j0 + 1) + i0);
                V4<T> d10, s20, d11, s21, d12, s22;
                xterms(cw1, rowp(src, j0 - 1), d10, s20);
                xterms(cw2, rowp(src, j0), d11, s21);
#pragma unroll
                for (int r = 0; r < RS; ++r) {
                  const int j = j0 + r;
                  const V4<T> cw4 = ld4(rowp(src, j + 2) + i0);
                  xterms(cw3, rowp(src, j + 1), d12, s22);
                  RowCoef<T> c;
                  if (__builtin_expect(j < 2 || j >= D - 2, 0)) {
                    c = make(coef + special_index(j, D) * MSK_NCOEF, sc);
                  } else {
                    c = ci;
                    c.b1 = b0row[j] * sc;
                  }
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
                  if (L < Lp) st4(rowp(dst, j) + i0, o);
                  else st4(out_g + (size_t)j * D + i0, o);
                  V4<T>& ac = acc[S][r];
                  ac.x += o.x;
                  ac.y += o.y;
                  ac.z += o.z;
                  ac.w += o.w;
                  nt[L] = accmax4(nt[L], o);
                  na[L] = accmax4(na[L], ac);
                  if (L == Lp) st4(acc_g + (size_t)j * D + i0, ac);
                  cw0 = cw1;
                  cw1 = cw2;
                  cw2 = cw3;
                  cw3 = cw4;
                  d10 = d11;
                  s20 = s21;
                  d11 = d12;
                  s21 = s22;
                }
                if (L < Lp && b == NB - 1 && g == 0) {
                  st4(rowp(dst, D) + i0, V4<T>{T(0), T(0), T(0), T(0)});
                  st4(rowp(dst, D + 1) + i0, V4<T>{T(0), T(0), T(0), T(0)});
                }
              }
              if (L < Lp) __syncthreads();
            });
            if (Lp == 1) __syncthreads();   // level 1 reads ring 0, which the next step rewrites
          };
          for (int t0 = 0; t0 < NB + Lp; t0 += LV) {
            static_for<LV>([&](auto Uc) {
              const int tau = t0 + decltype(Uc)::value;
              if (tau < NB + Lp) step(tau, Uc);
            });
          }
          // ---- norms of this pass, termination ------------------------------------
          T v[NRED];
          v[0] = nin;
#pragma unroll
          for (int L = 1; L <= LV; ++L) {
            v[2 * L - 1] = nt[L];
            v[2 * L] = na[L];
          }
          reduce_norms(v);   // also orders this pass's HBM stores before the next pass
          if (first) c1 = v[0];
          for (int L = 1; L <= Lp; ++L) {
            const T gn = v[2 * L - 1], ga = v[2 * L];
            if (c1 + gn <= tol * ga) {
              done = true;
              break;
            }
            c1 = gn;
          }
          nmv += (unsigned long long)Lp;
          k += Lp;
          if (k >= m_terms) done = true;
          first = false;
          in_buf ^= 1;
          acc_scale = T(1);
        }
        acc_scale = te;   // u = e^{mu/s} x (partial sum), applied when the sum is next read
      }
    }
    // ---- solution: apply the pending factor; maximum for the path status ----------
    T mfin = T(0);
    for (size_t e = (size_t)tid * 4; e < DD; e += (size_t)NT * 4) {
      V4<T> v = ld4(acc_g + e);
      v.x *= acc_scale;
      v.y *= acc_scale;
      v.z *= acc_scale;
      v.w *= acc_scale;
      st4(acc_g + e, v);
      mfin = tmax(mfin, tmax(tmax(absnan(v.x), absnan(v.y)), tmax(absnan(v.z), absnan(v.w))));
    }
    {
      T v[NRED];
      v[0] = mfin;
#pragma unroll
      for (int q = 1; q < NRED; ++q) v[q] = T(0);
      reduce_norms(v);
      mfin = v[0];
    }
    if (tid == 0) {
      if (a.work) atomicAdd(a.work, nmv);
      if (a.status) {
        uint32_t st = 0;
        if (!(mfin < T(INFINITY))) st |= MSK_PATH_NONFINITE;
        if (scale_cap) st |= MSK_PATH_SCALE_CAP;
        if (!((double)mfin <= 10.0 * (double)u0max)) st |= MSK_PATH_BLOWUP;
        a.status[path] = st;
      }
    }
    __syncthreads();
  }
  // Launched as the programmatic dependent of the resident clusters (split solve),
  // this grid ends only after that one has completed, so whatever follows on the
  // stream sees both grids' results; otherwise this returns at once.
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace

namespace {

// Two d x d term grids per CTA for `grid` CTAs, library-owned, grown on demand.
template <typename T, int D>
msk_status ensure_term_grids(msk_ctx* ctx, int64_t grid) {
  const size_t need = (size_t)grid * 2 * (size_t)D * D * sizeof(T);
  if (need <= ctx->stream_bytes) return MSK_OK;
  if (ctx->stream_scratch) cudaFree(ctx->stream_scratch);   // waits for work that may still use it
  ctx->stream_scratch = nullptr;
  ctx->stream_bytes = 0;
  msk_status st = msk_cuda(ctx, cudaMalloc(&ctx->stream_scratch, need), "streamed engine scratch");
  if (st != MSK_OK) return st;
  ctx->stream_bytes = need;
  return MSK_OK;
}

// grid_cap > 0: at most that many CTAs.  dependent: launched as the programmatic
// dependent of the kernel before it on the stream (it may start while that kernel
// still runs, on the SMs it leaves free; the two share no data but their inputs).
template <typename T, int D, int NT, int LV, int RS>
msk_status launch_stream_one(msk_ctx* ctx, const EngineArgs& e, cudaStream_t stream, int64_t grid_cap,
                             bool dependent) {
  using K = SCfg<T, D, NT, LV, RS>;
  auto kern = stream_engine_kernel<T, D, NT, LV, RS>;
  msk_status st = msk_cuda(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM),
                           "smem attribute (streamed engine)");
  if (st != MSK_OK) return st;
  int per_sm = 0;
  st = msk_cuda(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, K::SMEM), "occupancy");
  if (st != MSK_OK) return st;
  if (per_sm < 1) return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "streamed engine does not fit on an SM");
  int64_t grid = std::min<int64_t>((int64_t)per_sm * ctx->num_sms, e.order && e.qlen > 0 ? e.qlen : e.paths);
  if (grid_cap > 0) grid = std::min<int64_t>(grid, grid_cap);
  st = ensure_term_grids<T, D>(ctx, grid);
  if (st != MSK_OK) return st;
  StreamArgs sa{e, ctx->stream_scratch};
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = K::SMEM;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 1 : 0;
  return msk_cuda(ctx, cudaLaunchKernelEx(&cfg, kern, sa), "streamed engine launch");
}

}  // namespace

bool stream_engine_available(int d, int precision) {
  return d == 512 || d == 256 ? (precision == MSK_F32 || precision == MSK_F64) : false;
}

msk_status ensure_stream_scratch(msk_ctx* ctx, int precision, int64_t grid) {
  if (ctx->d == 512) return precision == MSK_F32 ? ensure_term_grids<float, 512>(ctx, grid)
                                                 : ensure_term_grids<double, 512>(ctx, grid);
  if (ctx->d == 256) return precision == MSK_F32 ? ensure_term_grids<float, 256>(ctx, grid)
                                                 : ensure_term_grids<double, 256>(ctx, grid);
  return MSK_OK;
}

msk_status launch_engine_stream(msk_ctx* ctx, int steps, int64_t paths, int precision, const double* Wt, void* out,
                                uint32_t* status, cudaStream_t stream, const long long* order,
                                unsigned long long* queue, int64_t qlen, int64_t grid_cap, bool dependent) {
  if (paths == 0) return MSK_OK;
  if (!out) return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "the streamed engine keeps the partial sum in the output");
  EngineArgs e{};
  e.band = ctx->band;
  e.u0 = ctx->u0;
  e.Wt = Wt;
  e.out = out;
  e.status = status;
  e.work = ctx->work;
  e.order = order;
  e.queue = queue;
  e.qlen = qlen;
  e.paths = paths;
  e.steps = steps;
  e.dx = ctx->dx;
  e.T = ctx->T;
  e.s_cap = kMskScaleCap;
  e.tol32 = 0x1p-20f;   // as the resident engine
  e.tol64 = 0x1p-53;
  e.c = coef_dev(ctx->coef);
  if (precision == MSK_F32) {
    switch (ctx->d) {
      case 512: return launch_stream_one<float, 512, 256, 4, 4>(ctx, e, stream, grid_cap, dependent);
      case 256: return launch_stream_one<float, 256, 256, 4, 4>(ctx, e, stream, grid_cap, dependent);
    }
  } else {
    switch (ctx->d) {
      case 512: return launch_stream_one<double, 512, 256, 1, 4>(ctx, e, stream, grid_cap, dependent);
      case 256: return launch_stream_one<double, 256, 256, 1, 4>(ctx, e, stream, grid_cap, dependent);
    }
  }
  return msk_fail(ctx, MSK_ERR_UNSUPPORTED, "grid size / precision combination not built (streamed engine)");
}

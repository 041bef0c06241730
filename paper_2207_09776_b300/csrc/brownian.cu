// S3: Brownian increments and per-step functionals, generated in-kernel.
//
// The paper evaluates the Lebesgue integrals of Eq. MagnusFormulas by simple
// Riemann sums on a fine grid of mesh Delta^Leb (Section 3, "Implementation"
// and "Error and notations").  The rule is read as the exact integral of the
// piecewise-linear interpolant of W through the fine nodes; on a fine cell of
// width delta with end values w0, w1 (step-local W~, restarted at the step):
//     int W~    += delta (w0 + w1) / 2
//     int W~^2  += delta (w0^2 + w0 w1 + w1^2) / 3
//     int s W~  += delta (s0 (2 w0 + w1) + s1 (w0 + 2 w1)) / 6
// and, for time-dependent sigma, alpha = a/2 (dW = dW_k/delta ds on the cell):
//     omega~    += sigma(t_mid) dW_k                     (omega = int sigma dW)
//     int omega~ += delta (omega0 + omega1) / 2
//     G1 = int omega~ ds - sum s_mid sigma(t_mid) dW_k
//     G2 = delta/2 sum (alpha0 omega0 + alpha1 omega1) - sum alpha_bar(s_mid) sigma(t_mid) dW_k.
//
// Parallel layout: one warp per (path, step), or per (path, interval of fine
// cells) for the solutions at output times inside a step.  The step's fine cells are
// processed in rounds of 32 x 64 cells; in a round each lane draws the normals
// of 64 consecutive cells (Philox4x32-10 + Box-Muller, double precision) into
// shared memory and sums its chunk's dW and sigma dW; an exclusive warp scan
// gives every lane the values of W~ and omega~ at its chunk start; a second
// pass over the staged increments accumulates the functionals, which are
// summed over the warp at the end.  The deterministic per-cell values
// (sigma at cell midpoints, alpha at the nodes, the antiderivative of alpha at
// the midpoints) come from a table built once per (T, n_fine, coefficients).
#include <type_traits>

#include "philox.cuh"
#include "msk_internal.cuh"

namespace {

constexpr int kChunk = 64;                 // cells per lane per round
constexpr int kWarps = 4;                  // warps (path-steps) per block
constexpr int kRound = 32 * kChunk;        // cells per round

struct BrownArgs {
  uint64_t seed, path_offset, path_stride;   // local path p is global path path_offset + p * path_stride
  int64_t n_fine, paths;
  int steps;
  double T;
  CoefDev c;
  // TRIG: [4][n_fine + 1] doubles sigma(mid), alpha(node), A(mid), A(node), then
  // [4][n_fine + 1] floats sigma(mid), alpha(node), A(node+1) - A(node), A(mid) - A(node);
  // null for CONST
  const double* tab;
  // Interval mode (steps = 1, paths = number of intervals): interval i covers the
  // fine cells jobs[3i+1] .. jobs[3i+1] + jobs[3i+2] - 1 of local path jobs[3i].
  const int64_t* jobs;
};

// antiderivative of alpha: A(t) = int_0^t alpha = (a0 t + a1 (1 - cos 2 pi t) / (2 pi)) / 2
__device__ __forceinline__ double alpha_anti(const CoefDev& c, double t) {
  return 0.5 * (c.a0 * t + c.a1 * (1.0 - cospi(2.0 * t)) / (2.0 * M_PI));
}

__global__ void cell_table_kernel(CoefDev c, int64_t n_fine, double T, double* tab) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n_fine) return;
  const double delta = T / (double)n_fine;
  const double tk = delta * (double)k, tm = delta * ((double)k + 0.5);
  const double sig = c.s0 * (1.0 + c.s1 * cospi(2.0 * tm)), alp = 0.5 * (c.a0 + c.a1 * sinpi(2.0 * tk));
  tab[k] = sig;                                                                    // sigma at cell midpoint
  tab[(n_fine + 1) + k] = alp;                                                     // alpha at node
  const double Am = alpha_anti(c, tm), An = alpha_anti(c, tk);
  tab[2 * (n_fine + 1) + k] = Am;                                                  // A at cell midpoint
  tab[3 * (n_fine + 1) + k] = An;                                                  // A at node
  // float copies, one float4 per cell: sigma(mid), alpha(node), the integral of alpha
  // over the cell and over its first half
  float4* tf = reinterpret_cast<float4*>(tab + 4 * (n_fine + 1));
  tf[k] = make_float4((float)sig, (float)alp, (float)(alpha_anti(c, tk + delta) - An), (float)(Am - An));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of eight per-lane values at once, by a transposed butterfly: in each of
// the first three rounds a lane keeps half of its values (chosen by one bit of its
// index) and adds its partner's copy of that half, then two plain rounds finish;
// 9 double additions instead of 40.  Every lane gets all eight totals back.
__device__ __forceinline__ void warp_sum8(double (&v)[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  double h[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double keep = b4 ? v[4 + j] : v[j], send = b4 ? v[j] : v[4 + j];
    h[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  double q[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double keep = b3 ? h[2 + j] : h[j], send = b3 ? h[j] : h[2 + j];
    q[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  double x = (b2 ? q[1] : q[0]) + __shfl_xor_sync(0xffffffffu, b2 ? q[0] : q[1], 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  // value k is now held by the lanes whose bits 4, 3, 2 spell k
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __shfl_sync(0xffffffffu, x, ((k & 4) << 2) | ((k & 2) << 2) | ((k & 1) << 2));
}

// exclusive prefix over the lanes and the warp total (the last lane's inclusive
// value, one shuffle instead of a second reduction)
__device__ __forceinline__ void warp_scan_total(double v, int lane, double& excl, double& total) {
  double x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  excl = x - v;
  total = __shfl_sync(0xffffffffu, x, 31);
}

template <bool FULL, bool TRIG, bool NF32>
__global__ void __launch_bounds__(32 * kWarps, 5) brownian_kernel(BrownArgs a, double* __restrict__ out) {
  // staged increments of one round (float in the float solves: half the shared
  // memory, so more warps fit on an SM)
  __shared__ typename std::conditional<NF32, float, double>::type stage[kWarps][32 * kChunk];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t wi = (int64_t)blockIdx.x * kWarps + wib;    // work item of this warp
  if (wi >= a.paths * a.steps) return;                      // whole warp leaves together
  // step-major order: the warps resident at one time work on the same step of
  // different paths, so the step's slice of the per-cell tables stays in L1
  const int64_t n_step = wi / a.paths;
  int64_t p = wi % a.paths;
  const int64_t idx = p * a.steps + n_step;                 // (path, step) record of this warp
  int64_t L = a.n_fine / a.steps;                           // cells of the step
  int64_t f0 = n_step * L;                                  // first fine cell of the step
  if (a.jobs) {
    p = a.jobs[3 * idx];
    f0 = a.jobs[3 * idx + 1];
    L = a.jobs[3 * idx + 2];
  }
  const double delta = a.T / (double)a.n_fine;
  const double sq = sqrt(delta);
  const uint64_t gpath = a.path_offset + (uint64_t)p * a.path_stride;
  const double* tsig = a.tab;
  const double* talp = a.tab + (a.n_fine + 1);
  const double* tA = a.tab + 2 * (a.n_fine + 1);
  double* st = reinterpret_cast<double*>(stage[wib]);   // double solves
  float* stf = reinterpret_cast<float*>(stage[wib]);    // float solves
  const double Astart = TRIG ? alpha_anti(a.c, delta * (double)f0) : 0.0;   // A at the step start
  const double sg0 = a.c.s0, al0 = 0.5 * a.c.a0;

  double W0 = 0.0, O0 = 0.0;                                // W~ and omega~ at the round start
  // Per-lane sums over the lane's cells (w0, w1 = W~ at a cell's ends, k = cell
  // index in the step, sdw = sigma dW of the cell); the functionals follow at
  // the end through the telescoping identities
  //   sum (w0 + w1) = 2 sum w0 + sum dw,   sum (w0 + 2 w1) = 3 sum w0 + 2 sum dw,
  //   sum (k + 1/2) sdw = sum k sdw + sum sdw / 2,   sum (om0 + om1) = 2 sum om0 + sum sdw.
  double Sw0 = 0.0, S2 = 0.0, Skw = 0.0, So0 = 0.0, Sks = 0.0, J3 = 0.0, J4 = 0.0;
  double swT = 0.0, soT = 0.0;                              // sum dw, sum sigma dW of the lane's cells
  // per cell k: {sigma(mid), alpha(node k), int of alpha over the cell, ... over its first half}
  const float4* tf4 = TRIG ? reinterpret_cast<const float4*>(a.tab + 4 * (a.n_fine + 1)) : nullptr;
  const double* tAn = TRIG ? a.tab + 3 * (a.n_fine + 1) : nullptr;     // A at the nodes
  for (int64_t rb = 0; rb < L; rb += kRound) {
    // ---- pass 1: normals of this lane's chunk, chunk sums -------------------------
    const int64_t c0 = rb + (int64_t)lane * kChunk;
    const int cnt = (int)max((int64_t)0, min((int64_t)kChunk, L - c0));
    double sw = 0.0, so = 0.0;
    if constexpr (NF32) {
      // float solves: float normals and float sums within the chunk (at most 64 cells,
      // values relative to the chunk start), folded into the double lane sums per chunk
      const float sqf = (float)sq;
      float swf = 0.0f, z0 = 0.0f, z1 = 0.0f;
      int q = 0;
      if (((f0 + c0) & 1) == 0) {
        // even start: cells 2i, 2i+1 of the chunk share a Philox call; two independent
        // calls per iteration (the same values and summation order as one cell at a time)
        for (; q + 4 <= cnt; q += 4) {
          const int64_t fi = f0 + c0 + q;
          float za0, za1, zb0, zb1;
          brownian_pair_f32f(a.seed, gpath, 0u, (uint64_t)(fi >> 1), za0, za1);
          brownian_pair_f32f(a.seed, gpath, 0u, (uint64_t)(fi >> 1) + 1, zb0, zb1);
          const float dw[4] = {sqf * za0, sqf * za1, sqf * zb0, sqf * zb1};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            stf[(q + e) * 32 + lane] = dw[e];
            swf += dw[e];
          }
        }
      }
      for (; q < cnt; ++q) {
        const int64_t fi = f0 + c0 + q;
        if (q == 0 || (fi & 1) == 0) brownian_pair_f32f(a.seed, gpath, 0u, (uint64_t)(fi >> 1), z0, z1);
        const float dw = sqf * ((fi & 1) ? z1 : z0);
        stf[q * 32 + lane] = dw;
        swf += dw;
      }
      sw = (double)swf;   // the chunk's sum of sigma dW comes out of pass 2
    } else {
      double z0 = 0.0, z1 = 0.0;
      for (int q = 0; q < cnt; ++q) {
        const int64_t fi = f0 + c0 + q;
        if (q == 0 || (fi & 1) == 0) brownian_pair(a.seed, gpath, 0u, (uint64_t)(fi >> 1), z0, z1);
        const double dw = sq * ((fi & 1) ? z1 : z0);
        st[q * 32 + lane] = dw;
        sw += dw;
        if (FULL) so += (TRIG ? tsig[fi] : sg0) * dw;
      }
    }
    double woff, wtot;
    warp_scan_total(sw, lane, woff, wtot);
    woff += W0;
    W0 += wtot;
    double ooff = 0.0;
    if constexpr (!NF32) {
      double otot;
      warp_scan_total(so, lane, ooff, otot);
      ooff += O0;
      O0 += otot;
    }
    if (!FULL) continue;
    swT += sw;
    if constexpr (!NF32) soT += so;
    // ---- pass 2: functionals over the staged increments -------------------------
    // Sums are kept without their constant factors (delta/2, delta/3, delta^2/6,
    // delta), applied once at the end; k is carried as a double counter.
    if constexpr (NF32) {
      // w = woff + x, om = ooff + y with x, y the float running sums inside the chunk;
      // k = c0 + kl.  Chunk sums A = sum x0, B = sum (x0^2 + x0 x1 + x1^2), Ck = sum kl (x0 + x1),
      // E = sum y0, Fk = sum kl sdw, H = sum (alpha0 + alpha1), I = sum (alpha0 y0 + alpha1 y1),
      // Jz = sum (z + ah) sdw with alpha_bar(s_mid) = zoff + z + ah: zoff = A(chunk start) -
      // A(step start) (double, once per chunk), z the float running integral of alpha.
      float x0 = 0.0f, y0 = 0.0f, kl = 0.0f, z = 0.0f;
      float A = 0.0f, Bq = 0.0f, Ck = 0.0f, E = 0.0f, Fk = 0.0f, H = 0.0f, I = 0.0f, Jz = 0.0f;
      // this cell's table entry; the next one (node k + 1 <= n_fine) supplies alpha(t_{k+1})
      float4 cur = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (TRIG && cnt > 0) cur = tf4[f0 + c0];
      for (int q = 0; q < cnt; ++q) {
        const int64_t fi = f0 + c0 + q;
        const float dw = stf[q * 32 + lane];
        const float x1 = x0 + dw, xs = x0 + x1;
        A += x0;
        Bq = fmaf(x0, xs, fmaf(x1, x1, Bq));
        Ck = fmaf(kl, xs, Ck);
        const float sdw = (TRIG ? cur.x : (float)sg0) * dw;
        const float y1 = y0 + sdw;
        E += y0;
        Fk = fmaf(kl, sdw, Fk);
        if (TRIG) {
          const float4 nxt = tf4[fi + 1];
          const float al0 = cur.y, al1 = nxt.y;
          H += al0 + al1;
          I = fmaf(al0, y0, fmaf(al1, y1, I));
          Jz = fmaf(z + cur.w, sdw, Jz);
          z += cur.z;
          cur = nxt;
        }
        x0 = x1;
        y0 = y1;
        kl += 1.0f;
      }
      // the chunk's sum of sigma dW (= omega~ at its end, relative to its start) gives the
      // omega~ offsets of the chunks
      so = (double)y0;
      double otot;
      warp_scan_total(so, lane, ooff, otot);
      ooff += O0;
      O0 += otot;
      soT += so;
      const double n = (double)cnt, kc = (double)c0, xe = (double)x0;
      const double sx = 2.0 * (double)A + xe;             // sum (x0 + x1)
      Sw0 += n * woff + (double)A;
      S2 += 3.0 * n * woff * woff + 3.0 * woff * sx + (double)Bq;
      Skw += kc * (2.0 * n * woff + sx) + 2.0 * woff * (0.5 * n * (n - 1.0)) + (double)Ck;
      So0 += n * ooff + (double)E;
      Sks += kc * (double)y0 + (double)Fk;
      if (TRIG) {
        J3 += ooff * (double)H + (double)I;
        if (cnt > 0) J4 += (tAn[f0 + c0] - Astart) * (double)y0 + (double)Jz;   // y0 = sum sdw of the chunk
      }
    } else {
      double w0 = woff, om0 = ooff;
      double kd = (double)c0;
      for (int q = 0; q < cnt; ++q) {
        const int64_t fi = f0 + c0 + q;
        const double dw = st[q * 32 + lane];
        const double w1 = w0 + dw;
        const double ws = w0 + w1;
        Sw0 += w0;
        S2 = fma(w0, ws, fma(w1, w1, S2));                     // delta/3 sum (w0^2 + w0 w1 + w1^2)
        Skw = fma(kd, ws, Skw);                                // sum k (w0 + w1)
        const double sig = TRIG ? tsig[fi] : sg0;
        const double sdw = sig * dw;
        const double om1 = om0 + sdw;
        So0 += om0;
        Sks = fma(kd, sdw, Sks);                               // sum k sigma dW
        if (TRIG) {
          J3 = fma(talp[fi], om0, fma(talp[fi + 1], om1, J3)); // delta/2 sum (alpha0 om0 + alpha1 om1)
          J4 = fma(tA[fi] - Astart, sdw, J4);                  // sum alpha_bar(s_mid) sigma dW
        }
        w0 = w1;
        om0 = om1;
        kd += 1.0;
      }
    }
    __syncwarp();   // the stage buffer is rewritten by the next round
  }
  if (FULL) {
    const double S1 = 2.0 * Sw0 + swT;                       // sum (w0 + w1)
    const double S3 = 3.0 * (Skw + Sw0) + 2.0 * swT;          // sum (3k (w0 + w1) + w0 + 2 w1)
    const double J1 = 2.0 * So0 + soT;                       // sum (om0 + om1)
    const double J2 = Sks + 0.5 * soT;                       // sum (k + 1/2) sigma dW
    double t[8] = {S1, S2, S3, J1, J2, TRIG ? J3 : 0.0, TRIG ? J4 : 0.0, 0.0};
    warp_sum8(t, lane);
    const double I1 = 0.5 * delta * t[0];
    const double I2 = delta / 3.0 * t[1];
    const double I3 = delta * delta / 6.0 * t[2];
    const double jom = 0.5 * delta * t[3];
    const double ssdw = delta * t[4];
    // constant coefficients: alpha_bar(s) = alpha s and alpha0 = alpha1 = alpha
    const double jaom = TRIG ? 0.5 * delta * t[5] : al0 * jom;
    const double abdw = TRIG ? t[6] : al0 * ssdw;
    if (lane == 0) {
      double* o = out + idx * MSK_NF;
      o[MSK_F_DW] = W0;
      o[MSK_F_I1] = I1;
      o[MSK_F_I2] = I2;
      o[MSK_F_I3] = I3;
      o[MSK_F_OM] = O0;
      o[MSK_F_JOM] = jom;
      o[MSK_F_G1] = jom - ssdw;
      o[MSK_F_G2] = jaom - abdw;
    }
  } else if (lane == 0) {
    out[idx] = W0;
  }
}

}  // namespace

// Per-cell table of the deterministic coefficient values, rebuilt when T,
// n_fine or the coefficient profile changed since the last build.
static msk_status ensure_cell_table(msk_ctx* ctx, cudaStream_t stream) {
  const msk_coeffs& c = ctx->coef;
  if (ctx->tab && ctx->tab_n == ctx->n_fine && ctx->tab_T == ctx->T && ctx->tab_coef.a0 == c.a0 &&
      ctx->tab_coef.a1 == c.a1 && ctx->tab_coef.s0 == c.s0 && ctx->tab_coef.s1 == c.s1 &&
      ctx->tab_coef.kind == c.kind)
    return MSK_OK;
  if (ctx->tab && ctx->tab_n != ctx->n_fine) {
    cudaFree(ctx->tab);   // waits for work that may still read it
    ctx->tab = nullptr;
  }
  if (!ctx->tab) {
    msk_status st = msk_cuda(ctx, cudaMalloc(&ctx->tab, 6 * (size_t)(ctx->n_fine + 1) * sizeof(double)),
                             "cell table allocation");
    if (st != MSK_OK) return st;
  }
  const int64_t n = ctx->n_fine + 1;
  cell_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(coef_dev(c), ctx->n_fine, ctx->T, ctx->tab);
  msk_status st = msk_cuda(ctx, cudaGetLastError(), "cell table");
  if (st != MSK_OK) return st;
  ctx->tab_n = ctx->n_fine;
  ctx->tab_T = ctx->T;
  ctx->tab_coef = c;
  return MSK_OK;
}

// One launch of the kernel variant for (functionals or increments, coefficient kind, normal precision).
static void dispatch_brownian(const BrownArgs& a, bool full, bool trig, bool nf32, double* out, cudaStream_t stream) {
  const int64_t n = a.paths * a.steps;
  const unsigned blocks = (unsigned)((n + kWarps - 1) / kWarps);
  const unsigned t = 32 * kWarps;
  if (!full) {
    if (nf32) brownian_kernel<false, false, true><<<blocks, t, 0, stream>>>(a, out);
    else brownian_kernel<false, false, false><<<blocks, t, 0, stream>>>(a, out);
  } else if (trig) {
    if (nf32) brownian_kernel<true, true, true><<<blocks, t, 0, stream>>>(a, out);
    else brownian_kernel<true, true, false><<<blocks, t, 0, stream>>>(a, out);
  } else {
    if (nf32) brownian_kernel<true, false, true><<<blocks, t, 0, stream>>>(a, out);
    else brownian_kernel<true, false, false><<<blocks, t, 0, stream>>>(a, out);
  }
}

msk_status launch_brownian(msk_ctx* ctx, int steps, int64_t paths, double* out, bool increments_only,
                           cudaStream_t stream, bool nf32) {
  const int64_t n = paths * steps;
  if (n == 0) return MSK_OK;
  const bool trig = ctx->coef.kind == MSK_COEF_TRIG;
  if (trig && !increments_only) {
    msk_status st = ensure_cell_table(ctx, stream);
    if (st != MSK_OK) return st;
  }
  BrownArgs a{ctx->seed, ctx->path_offset, 1, ctx->n_fine, paths, steps, ctx->T, coef_dev(ctx->coef),
              trig ? ctx->tab : nullptr, nullptr};
  dispatch_brownian(a, !increments_only, trig, nf32, out, stream);
  return msk_cuda(ctx, cudaGetLastError(), "brownian kernel");
}

// Functionals of arbitrary fine-cell intervals: jobs_dev[3 i .. 3 i + 2] = (local
// path, first cell, number of cells) of interval i (device, njobs entries).
msk_status launch_brownian_jobs(msk_ctx* ctx, const int64_t* jobs_dev, int64_t njobs, double* out,
                                cudaStream_t stream, bool nf32) {
  if (njobs == 0) return MSK_OK;
  const bool trig = ctx->coef.kind == MSK_COEF_TRIG;
  if (trig) {
    msk_status st = ensure_cell_table(ctx, stream);
    if (st != MSK_OK) return st;
  }
  BrownArgs a{ctx->seed, ctx->path_offset, 1, ctx->n_fine, njobs, 1, ctx->T, coef_dev(ctx->coef),
              trig ? ctx->tab : nullptr, jobs_dev};
  dispatch_brownian(a, true, trig, nf32, out, stream);
  return msk_cuda(ctx, cudaGetLastError(), "brownian kernel (intervals)");
}

// Functionals of the global paths first, first + stride, ... (paths of them).
msk_status launch_brownian_strided(msk_ctx* ctx, int steps, int64_t paths, double* out, uint64_t first,
                                   uint64_t stride, cudaStream_t stream, bool nf32) {
  const int64_t n = paths * steps;
  if (n == 0) return MSK_OK;
  const bool trig = ctx->coef.kind == MSK_COEF_TRIG;
  if (trig) {
    msk_status st = ensure_cell_table(ctx, stream);
    if (st != MSK_OK) return st;
  }
  BrownArgs a{ctx->seed, first, stride, ctx->n_fine, paths, steps, ctx->T, coef_dev(ctx->coef),
              trig ? ctx->tab : nullptr, nullptr};
  dispatch_brownian(a, true, trig, nf32, out, stream);
  return msk_cuda(ctx, cudaGetLastError(), "brownian kernel");
}

// Variants for callers that supply the per-cell table buffer themselves
// (6 * (n_fine + 1) doubles); used by the entry point that allocates nothing.
msk_status launch_cell_table_into(msk_ctx* ctx, double* tab, cudaStream_t stream) {
  const int64_t n = ctx->n_fine + 1;
  cell_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(coef_dev(ctx->coef), ctx->n_fine, ctx->T, tab);
  return msk_cuda(ctx, cudaGetLastError(), "cell table");
}

msk_status launch_brownian_with_table(msk_ctx* ctx, int steps, int64_t paths, double* out, const double* tab,
                                      cudaStream_t stream, bool nf32) {
  const int64_t n = paths * steps;
  if (n == 0) return MSK_OK;
  const bool trig = ctx->coef.kind == MSK_COEF_TRIG;
  BrownArgs a{ctx->seed, ctx->path_offset, 1, ctx->n_fine, paths, steps, ctx->T, coef_dev(ctx->coef),
              trig ? tab : nullptr, nullptr};
  dispatch_brownian(a, true, trig, nf32, out, stream);
  return msk_cuda(ctx, cudaGetLastError(), "brownian kernel");
}

// Allocate/refresh the per-cell coefficient table now (so that a later
// launch_brownian performs no allocation, e.g. inside a stream capture).
msk_status msk_prepare_brownian(msk_ctx* ctx, cudaStream_t stream) {
  if (ctx->coef.kind != MSK_COEF_TRIG) return MSK_OK;
  return ensure_cell_table(ctx, stream);
}

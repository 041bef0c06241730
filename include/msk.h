/*
 * msk.h — C ABI of the B300 stochastic Magnus solver for the kinetic Langevin SPDE
 *
 *   du = ( a(t)/2 d_vv u + kappa v d_x u ) dt + sigma(t) d_v u dW          (Eq. spde)
 *
 * discretised in space by central finite differences with zero Dirichlet
 * boundary (Section 2, "Computation of A and B") into the linear matrix SDE
 * dU = B U dt + A U dW (Eq. SPDEvec), and integrated over many Brownian paths
 * at once by the iterated Ito-stochastic Magnus scheme of orders 1..3
 * (Eq. MagnusFormulas; Section 2, "Iterated Magnus expansion"), with the
 * Euler-Maruyama scheme (Eq. EulerMaruyama) as comparator.
 *
 * Conventions for every entry point
 *  - Every call returns msk_status and never throws, exits or prints.
 *  - The library owns the context, its operator tables and its scratch
 *    buffers.  The caller owns every buffer passed in ("_dev" = device
 *    memory of the context's device, "_host" = host memory) and the CUDA
 *    stream; work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 *    default stream) and the call returns without synchronising unless
 *    stated.  The library never frees caller memory.
 *  - Solution arrays are [path][v][x] with x fastest (the paper's vec
 *    ordering, vec index i + n_x j), element type double for MSK_F64 and
 *    float for MSK_F32.
 *  - A failed call returns non-MSK_OK and leaves a message for
 *    msk_last_error(ctx); per-path numerical trouble (non-finite values,
 *    Taylor scaling cap, blow-up) is reported in the optional per-path
 *    status words and does not fail the call.
 *  - Sizes: 32 <= n_x = n_v <= 512, n_x a multiple of 32 and one of
 *    32, 64, 128, 256, 512; paths >= 0 (0 is a no-op); steps >= 1 dividing
 *    n_fine.  Violations return MSK_ERR_ARG before any device work.
 */
#ifndef MSK_H
#define MSK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msk_ctx msk_ctx;

typedef enum {
  MSK_OK = 0,
  MSK_ERR_ARG = 1,          /* invalid argument (checked before any device work) */
  MSK_ERR_CUDA = 2,         /* a CUDA runtime call failed (message in msk_last_error) */
  MSK_ERR_OOM = 3,          /* device allocation failed */
  MSK_ERR_TIMEOUT = 4,      /* reserved: a bounded device wait ran out */
  MSK_ERR_NONFINITE = 5,    /* non-finite scalar argument */
  MSK_ERR_UNSUPPORTED = 6   /* valid request this build does not implement */
} msk_status;

enum { MSK_COEF_CONST = 0, MSK_COEF_TRIG = 1 };
enum { MSK_XPROF_NONE = 0, MSK_XPROF_RATIONAL = 1, MSK_XPROF_VALUES = 2 };
enum { MSK_F64 = 0, MSK_F32 = 1 };
enum { MSK_REF_EXPLICIT = 0, MSK_REF_BUFFER = 1 };

/* per-path status bits */
#define MSK_PATH_NONFINITE 1u   /* a non-finite value reached the solution */
#define MSK_PATH_SCALE_CAP 2u   /* Taylor scaling count hit its cap (result inaccurate) */
#define MSK_PATH_BLOWUP 4u      /* max|u_T| > 10 max|u_0| (Magnus explosion, Section 3.1) */

/* Brownian functionals per (path, step), see msk_brownian_functionals */
#define MSK_NF 8
enum { MSK_F_DW = 0, MSK_F_I1, MSK_F_I2, MSK_F_I3, MSK_F_OM, MSK_F_JOM, MSK_F_G1, MSK_F_G2 };

/* Basis operators of the Magnus logarithm (Kronecker factors: v-matrix (x) x-matrix),
 * with Bx = kappa diag(v) (x) D^x, Bvv = D^vv (x) I, A0 = D^v (x) I. */
#define MSK_NOPS 13
enum {
  MSK_OP_BX = 0, MSK_OP_BVV, MSK_OP_A0, MSK_OP_A0A0, MSK_OP_BX_A0, MSK_OP_BVV_A0,
  MSK_OP_BX_BVV, MSK_OP_BXA0_A0, MSK_OP_BVVA0_A0, MSK_OP_BXA0_BX, MSK_OP_BXA0_BVV,
  MSK_OP_BVVA0_BX, MSK_OP_BVVA0_BVV
};

/* Per (path, step) record written by msk_omega_weights (doubles):
 * [0, MSK_NOPS) operator weights, then
 *   MSK_WT_ALPHA  the bound alpha that chose (s, m): an upper bound of the minimum of
 *                 Al-Mohy & Higham's alpha_p(Omega - mu I) over the p with
 *                 p (p - 1) <= m + 1 (<= MSK_WT_NORM); alpha / s <= theta_m
 *   MSK_WT_WORK   expected stencil applications of the step (path ordering), 0 if unused
 *   MSK_WT_EPS    ||E||_inf (a bound with an x profile or general coefficients) of the
 *                 Brownian part E of Omega - mu I (the terms whose weights vanish with the
 *                 functionals); s >= ||E|| / theta_E, theta_E = 14 (float), 24 (double)
 *   MSK_WT_MU     shift mu = trace(Omega) / n
 *   MSK_WT_NORM   ||Omega - mu I||_inf (exact for the Langevin operators; a bound
 *                 over the operators with an x profile or general coefficients)
 *   MSK_WT_S, MSK_WT_M  Taylor scaling count s and degree cap m (alpha / s <= theta_m). */
#define MSK_NWT 20
enum { MSK_WT_ALPHA = 13, MSK_WT_WORK = 14, MSK_WT_EPS = 15, MSK_WT_MU = 16, MSK_WT_NORM = 17, MSK_WT_S = 18,
       MSK_WT_M = 19 };

/* Interior grid n_x x n_v on [ax,bx] x [av,bv]; Delta = (b - a)/(n + 1)
 * (Eq. xGrid, vGrid).  This build requires nx == nv. */
typedef struct {
  int32_t nx, nv;
  double ax, bx, av, bv;
} msk_grid;

/* Langevin coefficients: f^x = drift_sign * v, g^vv = a(t), sigma^v = sigma(t)
 * (Eq. coeffsLangevinConst has drift_sign = -1 and constant a, sigma).
 * MSK_COEF_CONST: a = a0, sigma = s0.
 * MSK_COEF_TRIG:  a(t) = a0 + a1 sin(2 pi t), sigma(t) = s0 (1 + s1 cos(2 pi t)). */
typedef struct {
  int32_t drift_sign;
  int32_t kind;
  double a0, a1, s0, s1;
} msk_coeffs;

/* Gaussian initial datum u0(z) = scale * N(z; mean, cov) (Eq. initialdatum is
 * mean 0, cov I, scale 2 pi). */
typedef struct {
  double mean_x, mean_v, cov_xx, cov_xv, cov_vv, scale;
} msk_gaussian;

/* Create a context on CUDA device `device`: builds the grid, the finite
 * difference operators and the thirteen basis-operator band tables on the
 * device (Section 2, "Computation of A and B"; commutators of
 * Eq. MagnusFormulas).  Defaults: drift +1, a = 1, sigma = 0.5, standard
 * Gaussian density, seed 0, n_fine 10000, T 1, no x profile.  *out is NULL
 * on failure.  nx = nv = d with 8 <= d <= 512 (else MSK_ERR_ARG); the
 * constant-coefficient engine is built for d = 32, 64, 128, 256, 512 (float)
 * and 32 .. 256 (double), the variable-coefficient engine (msk_set_x_profile)
 * for any d whose five-field slab fits a cluster of at most 16 CTAs; other
 * combinations fail at solve time with MSK_ERR_UNSUPPORTED. */
msk_status msk_create(msk_ctx** out, const msk_grid* grid, int device);

/* Release the context and every library-owned device buffer.  NULL is a no-op.
 * Must not be called while work using the context is in flight.
 * A context's scratch (functionals, weights, path order) is shared by its
 * solves: calls on one context are ordered on one stream, or the caller
 * synchronises between calls issued on different streams or host threads.
 * Growing the scratch frees the old buffer (cudaFree, which waits for the
 * device) and is not possible while a stream of the device is being captured
 * into a graph: size it with one uncaptured call first. */
void msk_destroy(msk_ctx* ctx);

/* Multiply-add throughput of the CUDA cores of `device` in TFLOP/s (2 flop per
 * fused multiply-add), MSK_F32 or MSK_F64, measured on `stream` by a kernel of
 * independent FMA chains over every SM (a few milliseconds; synchronises the
 * stream).  No counterpart in the paper: the denominator of the roofline
 * fraction of the engines, whose state stays on chip.  Bad precision or null
 * output -> MSK_ERR_ARG. */
msk_status msk_fma_throughput(int device, int precision, double* tflops_out, void* stream);

/* Engine of the Magnus solves of the Langevin operators (constant or
 * time-dependent coefficients):
 *   MSK_ENGINE_AUTO      the resident engine wherever it holds the grid, the streamed
 *                        engine where only it does (double at d = 512); in float at
 *                        d = 256 and 512 the split below (default)
 *   MSK_ENGINE_RESIDENT  each path's state in shared memory (a cluster of up to 16
 *                        CTAs; d = 32 .. 512 in float, 32 .. 256 in double)
 *   MSK_ENGINE_STREAMED  each path's state in HBM, swept by one CTA per path with
 *                        several Taylor terms per sweep (d = 256, 512; float and
 *                        double); needs two d x d grids of library scratch per CTA,
 *                        so msk_solve_magnus_noalloc refuses it
 *   MSK_ENGINE_SPLIT     where both engines exist (d = 256 in float and double,
 *                        d = 512 in float): the resident clusters take the paths of
 *                        the lower indices on the SMs they fill, the streamed engine
 *                        the last n_s paths on the SMs the clusters leave free, both
 *                        at once; n_s = a whole number of paths per free SM, from
 *                        the two engines' measured rates.  Only msk_solve_magnus and
 *                        msk_magnus_from_weights with more than two paths per SM and
 *                        an output in device memory split (not msk_solve_magnus_host,
 *                        nor any output in mapped host memory: the streamed engine
 *                        would sweep it over the bus); elsewhere this mode acts as
 *                        MSK_ENGINE_AUTO.  Every
 *                        path's result equals, bit for bit, the one of the engine that
 *                        took it, and which engine takes a path depends only on the
 *                        path count and the device's SM count.
 * Euler-Maruyama, output times, x profiles and general coefficients always use the
 * resident engines.  Both engines give the same solution within the Taylor
 * tolerance.  Bad mode -> MSK_ERR_ARG. */
#define MSK_ENGINE_AUTO 0
#define MSK_ENGINE_RESIDENT 1
#define MSK_ENGINE_STREAMED 2
#define MSK_ENGINE_SPLIT 3
msk_status msk_set_engine(msk_ctx* ctx, int mode);

/* Last error message of the context ("" if none).  For ctx NULL: the message
 * of the last msk_create that failed after validating its arguments on this
 * thread, or "null context". */
const char* msk_last_error(const msk_ctx* ctx);

/* Set the coefficient profile (see msk_coeffs).  Non-finite values -> MSK_ERR_NONFINITE. */
msk_status msk_set_coefficients(msk_ctx* ctx, const msk_coeffs* coeffs);

/* Variable coefficients in x (Section 3.2, Eq. coeffsLangevinVar):
 *   g^vv(x, v) = a(t) psi(x),   sigma^v(x, v) = sigma(t) sqrt(psi(x)),
 * so that Bvv = D^vv (x) Psi and A0 = D^v (x) Psi^(1/2) with Psi = diag(psi(x_i)).
 *   kind MSK_XPROF_NONE      psi = 1 (the constant-coefficient operators; default)
 *   kind MSK_XPROF_RATIONAL  psi(x) = 1 + c / (1 + x^2), evaluated on the x nodes on
 *                            the device (c = 1 is the paper's choice); c >= 0
 *   kind MSK_XPROF_VALUES    psi_host[i] = psi(x_i), i = 0 .. d-1 (host, copied), all > 0
 * With a profile, msk_solve_magnus / msk_solve_magnus_noalloc /
 * msk_magnus_from_weights / msk_solve_euler / msk_select_steps run the
 * variable-coefficient engine, which applies Omega by composing the two base
 * operators B and A0 (exact truncated products) instead of folded stencils.
 * With constant coefficients the engine composes the six operators of
 * Eq. MagnusFormulas (B = Bx + a/2 Bvv) and msk_magnus_from_weights reads only the
 * weights of BX, A0, A0A0, BX_A0, BXA0_A0 and BXA0_BX, the others being implied;
 * with time-dependent ones (MSK_COEF_TRIG) it composes all thirteen MSK_OP_*
 * operators over Bx, Bvv and A0 and reads all thirteen weights.  msk_apply_omega, msk_explicit_solution,
 * msk_error with MSK_REF_EXPLICIT and batches -> MSK_ERR_UNSUPPORTED (no closed
 * form exists).  Invalid kind, c < 0, non-positive or non-finite values ->
 * MSK_ERR_ARG / MSK_ERR_NONFINITE before any device work. */
msk_status msk_set_x_profile(msk_ctx* ctx, int kind, double c, const double* psi_host);

/* General coefficients (Eq. generalSPDE, Section 2 "Computation of A and B"):
 * coef_host (host, copied) holds 9 grids [9][v][x] of the time-independent
 * coefficient functions at the interior nodes, in the order
 *   h, f^x, f^v, g^xx, g^xv, g^vv, sigma, sigma^x, sigma^v,
 * of du = (h u + f^x u_x + f^v u_v + g^xx/2 u_xx + g^xv u_xv + g^vv/2 u_vv) dt
 *        + (sigma u + sigma^x u_x + sigma^v u_v) dW.
 * B becomes the nine-point and A the five-point central-difference stencil with
 * these per-point coefficients (zero Dirichlet boundary), and msk_solve_magnus /
 * _noalloc / _times, msk_magnus_from_weights, msk_solve_euler and msk_select_steps
 * run the general-coefficient engine (Omega by composing B and A; the coefficient
 * set of msk_set_coefficients and any x profile are ignored while this is set).
 * NULL returns to the Langevin operators.  msk_apply_omega, msk_explicit_solution,
 * msk_error with MSK_REF_EXPLICIT and batches -> MSK_ERR_UNSUPPORTED.  Non-finite
 * values -> MSK_ERR_NONFINITE before any device work.  Synchronises the device. */
msk_status msk_set_general_coefficients(msk_ctx* ctx, const double* coef_host);

/* Set a Gaussian initial datum; evaluated on the interior grid on the device. */
msk_status msk_set_initial_gaussian(msk_ctx* ctx, const msk_gaussian* g);

/* Copy a caller-owned initial datum u0_dev ([v][x], double, device) into the context. */
msk_status msk_set_initial(msk_ctx* ctx, const double* u0_dev, void* stream);

/* Brownian stream: Philox4x32-10 key = seed, path p of a call uses global index
 * path_offset + p; n_fine increments of variance T/n_fine on [0, T] (the
 * fine "Lebesgue" grid of Section 3, "Error and notations"). */
msk_status msk_set_seed(msk_ctx* ctx, uint64_t seed, uint64_t path_offset, int64_t n_fine,
                        double T);

/* Raw Philox4x32-10 words of the Brownian stream: out_dev[4 q + r] = word r of
 * counter (first_pair + q, path lo, path hi, tag), key (seed lo, seed hi),
 * q = 0..npairs-1.  Integer work; used to check bit-exactness. */
msk_status msk_philox_words(uint64_t seed, uint64_t path, uint32_t tag, int64_t first_pair,
                            int64_t npairs, uint32_t* out_dev, void* stream);

/* S3: per-step Brownian functionals on the fine grid (Section 3,
 * "Implementation": Lebesgue integrals by Riemann sums), read as exact
 * integrals of the piecewise-linear interpolant of W:
 *   F_dev[(p * steps + n) * MSK_NF + f], f = DW, I1 = int W~, I2 = int W~^2,
 *   I3 = int s W~, OM = int sigma dW, JOM = int omega~, G1, G2 (time-dependent
 *   weights, see msk_omega_weights), with W~ the Brownian motion restarted at
 *   the step start.  F_dev: caller-owned double[paths * steps * MSK_NF]. */
msk_status msk_brownian_functionals(msk_ctx* ctx, int steps, int64_t paths, double* F_dev,
                                    void* stream);

/* As msk_brownian_functionals, with the standard normals of each Philox pair
 * formed in double (normals = MSK_F64: identical to msk_brownian_functionals)
 * or in single precision (MSK_F32: uniforms (hi + 1/2) 2^-32 from the high
 * words, float Box-Muller; every functional still accumulated in double).
 * The float solves (msk_solve_magnus / msk_solve_euler / msk_solve_magnus_noalloc
 * with MSK_F32, batches, surrogate reference solutions) use MSK_F32 normals:
 * they differ from the double ones by about 1e-7 relative. */
msk_status msk_brownian_functionals_ex(msk_ctx* ctx, int steps, int64_t paths, int normals, double* F_dev,
                                       void* stream);

/* Brownian increments over `steps` equal steps: dW_dev[p * steps + n] (double). */
msk_status msk_brownian_increments(msk_ctx* ctx, int steps, int64_t paths, double* dW_dev,
                                   void* stream);

/* S4 + S5a: Magnus weights of the order-`order` logarithm (Eq. MagnusFormulas;
 * for MSK_COEF_TRIG the time-dependent order-2 extension of the Appendix's
 * Picard step), the trace shift mu = trace(Omega)/n, an infinity-norm bound of
 * Omega - mu I and the Taylor scaling/degree pair (s, m) chosen by the
 * backward-error bound of Al-Mohy & Higham (2011) at unit roundoff of
 * `precision`.  F_dev from msk_brownian_functionals; Wt_dev: caller-owned
 * double[paths * steps * MSK_NWT]. */
msk_status msk_omega_weights(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                             const double* F_dev, double* Wt_dev, void* stream);

/* S5a: infinity norms of the powers of the deterministic part of Omega, the
 * input of the (s, m) selection of msk_omega_weights (Section 2, `expmvtay2`,
 * after Al-Mohy & Higham (2011), who bound the scaling by
 * alpha_p = max(||A^p||^(1/p), ||A^(p+1)||^(1/(p+1))) instead of ||A||).
 * X_n = Omega_n - mu_n I with every Brownian functional set to zero (the terms
 * h Bx + alpha_bar Bvv - (int sigma^2)/2 A0^2 - G3/2 [Bx,Bvv] of step n, shared by
 * all paths): out_dev[r * 9 + q - 1] = ||X_r^q||_inf, q = 1 .. 9, computed in
 * float by propagating unit rows.  *rows_out = 1 for MSK_COEF_CONST (X is the
 * same every step), steps for MSK_COEF_TRIG, 0 with an x profile or general
 * coefficients (those engines bound the norm over their operators; nothing is
 * written).  out_dev: caller-owned float[*rows_out * 9], or NULL to query
 * *rows_out only. */
msk_status msk_power_norms(msk_ctx* ctx, int order, int steps, float* out_dev, int* rows_out, void* stream);

/* One application out = Omega u of Omega = sum_k w_k Op_k, weights_dev
 * [paths][MSK_NOPS] (double), u_dev/out_dev [paths][v][x] double.  Exposes the
 * widened-stencil operator tables for parity checks. */
msk_status msk_apply_omega(msk_ctx* ctx, const double* weights_dev, int64_t paths,
                           const double* u_dev, double* out_dev, void* stream);

/* S5b + S6: iterated Magnus solve (Section 2, "Iterated Magnus expansion"):
 * `steps` equal sub-intervals of [0, T], on each U <- exp(Omega_n) U by the
 * scaled truncated Taylor action with early termination.  precision MSK_F64:
 * all arithmetic in double; MSK_F32: stencil/Taylor arithmetic in float with
 * the Brownian functionals, weights, norm bound and (s, m) in double.
 * u_out_dev: [paths][v][x] of double (MSK_F64) or float (MSK_F32).
 * path_status_dev: optional uint32[paths] of MSK_PATH_* bits (may be NULL).
 * Scratch (functionals, weights, the engine's path order) is library-owned
 * and grows on demand. */
msk_status msk_solve_magnus(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                            void* u_out_dev, uint32_t* path_status_dev, void* stream);

/* msk_solve_magnus with the initial datum and the results in host memory
 * (Section 3, "Implementation": the solutions of all paths are produced on the
 * GPU; this call returns them to the host without a separate copy step).
 * u0_host: optional double[nv][nx] initial datum (NULL keeps the context's);
 * it is copied to the device on `stream` before the solve (any host memory;
 * page-locked memory makes the copy asynchronous).  u_out_host: [paths][v][x]
 * of double (MSK_F64) or float (MSK_F32); path_status_host: optional
 * uint32[paths].  Both must be page-locked and mapped into the device's address
 * space (cudaHostAlloc, a pinned torch tensor, or cudaHostRegister with
 * cudaHostRegisterMapped); otherwise the call returns MSK_ERR_ARG before any
 * work is enqueued.  The solver's kernels store each finished path directly
 * into u_out_host, so the device-to-host transfer overlaps the solve of the
 * remaining paths.  Caller-owned buffers; the results are complete once
 * `stream` has reached the end of the call (synchronise it before reading). */
msk_status msk_solve_magnus_host(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                                 const double* u0_host, void* u_out_host, uint32_t* path_status_host,
                                 void* stream);

/* S5b + S6 only: the iterated Magnus solve from precomputed per-(path, step)
 * records Wt_dev (layout of msk_omega_weights, double[paths * steps * MSK_NWT],
 * caller-owned).  msk_solve_magnus = msk_brownian_functionals +
 * msk_omega_weights + this call, with library-owned scratch.  With more than
 * two paths per SM the paths are solved in order of decreasing estimated cost
 * sum_n s_n m_n (a path order and a counter in the library's scratch, which
 * grows on demand); each path's result is independent of that order. */
msk_status msk_magnus_from_weights(msk_ctx* ctx, int steps, int64_t paths, int precision,
                                   const double* Wt_dev, void* u_out_dev,
                                   uint32_t* path_status_dev, void* stream);

/* Solutions at several output times inside the Magnus sub-intervals (Section 3,
 * "Implementation": the expansion of a sub-interval is evaluated at every requested
 * time, all times and trajectories in parallel).  times_cells (host, n_times
 * entries, strictly increasing, each in 1 .. n_fine) are output times in fine cells,
 * t_q = T times_cells[q] / n_fine.  With `steps` sub-intervals of L = n_fine/steps
 * cells and n = times_cells[q] / L (t_n <= t_q < t_{n+1}),
 *   u(t_q) = exp(Y(t_n, t_q)) u(t_n),
 * Y(t_n, t_q) the order-`order` logarithm of Eq. MagnusFormulas over [t_n, t_q] (its
 * functionals from the same Brownian path) and u(t_n) the iterated solution after n
 * steps; an output at a sub-interval end is the iterated solution there.
 * u_out_dev: [paths][n_times][v][x] of double (MSK_F64) or float (MSK_F32),
 * caller-owned; path_status_dev (nullable): uint32[paths * n_times], the MSK_PATH_*
 * bits of the partial step OR those of the path's whole iterated solve.  Scratch is
 * library-owned (as msk_solve_magnus, plus 14 doubles per (path, output)).  Also with
 * an x profile (msk_set_x_profile).  Bad times -> MSK_ERR_ARG before device work. */
msk_status msk_solve_magnus_times(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                                  const int64_t* times_cells, int n_times, void* u_out_dev,
                                  uint32_t* path_status_dev, void* stream);

/* msk_solve_magnus for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is a property of the library, not of the method.
 * Callers whose device memory belongs to another allocator (a framework's
 * caching allocator, a fixed budget) or who must not hit cudaMalloc/cudaFree
 * (which synchronise the device) inside a latency-bound loop get the same
 * solve with its scratch (functionals, weights, per-cell table) taken from one
 * file-scope __device__ array of 2^21 doubles (16 MiB) that every GPU loading
 * the library holds until exit.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  Requests needing more than the array
 * (paths * steps * (MSK_NF + MSK_NWT) doubles, plus 6 (n_fine + 1) for
 * MSK_COEF_TRIG, plus ceil(9 r / 2) for the power norms of the Taylor
 * selection, r = steps for MSK_COEF_TRIG and 1 otherwise, 0 with an x profile
 * or general coefficients) fail with MSK_ERR_ARG before any device work.  The
 * power norms are recomputed by every call (no cache).  The first call
 * on a device looks up the array's address (once per device); make it before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents (nothing in it needs to start at zero); calls whose work overlaps
 * on the GPU race on it and must be serialised by the caller.  With an x
 * profile or general coefficients the operator table those engines read is
 * allocated by msk_set_x_profile / msk_set_general_coefficients, never by a
 * solve, so this call stays allocation-free there too.  Arguments and
 * outputs as for msk_solve_magnus. */
msk_status msk_solve_magnus_noalloc(msk_ctx* ctx, int order, int steps, int64_t paths,
                                    int precision, void* u_out_dev,
                                    uint32_t* path_status_dev, void* stream);

/* Work counter: number of whole-grid stencil applications (Taylor terms and
 * Euler steps, summed over paths) performed by the engine since the last
 * reset, read after synchronising `stream`.  reset != 0 zeroes it afterwards. */
msk_status msk_work_counter(msk_ctx* ctx, uint64_t* matvecs_host, int reset, void* stream);

/* S10: uneven batches in one persistent launch.  An item is one context (grid
 * 64, 128 or 256; its coefficients, initial datum and seed as set at
 * msk_batch_create, which snapshots them) with its own order, step count and
 * path count; the outputs are float [paths][d][d] (float stencil/Taylor
 * arithmetic, double functionals, weights and Taylor parameters).  All items
 * must live on one device. */
typedef struct {
  msk_ctx* ctx;
  int32_t order;
  int32_t steps;
  int64_t paths;
  float* u_out_dev;        /* caller-owned [paths][d][d] */
  uint32_t* status_dev;    /* optional [paths] of MSK_PATH_* bits */
} msk_batch_item;

typedef struct msk_batch msk_batch;

/* Build a batch: library-owned scratch for every item, the work lists of the
 * persistent kernels (units of a 4-CTA cluster: one 256^2 path, four 128^2
 * paths, or four/eight 64^2 paths; tasks of one CTA: one 128^2 path, or one or
 * two 64^2 paths), and the variant cached under `tune_cache` for this device
 * and batch shape (NULL or "": default variant 0). */
msk_status msk_batch_create(msk_batch** out, const msk_batch_item* items, int n_items,
                            const char* tune_cache);

/* Run the batch on `stream`: per-item Brownian functionals, weights and path
 * cost order, then the persistent kernels over all items' paths (variants 0 and
 * 2: the cluster megakernel over the 256^2 paths and, as its programmatic
 * dependent, the task kernel over the smaller grids' paths; 1 and 3: the
 * megakernel over every path; 4: each item's own engine launch).  The first
 * run captures these launches into a CUDA graph (on a private stream of the
 * batch); every run launches that graph on `stream`.  One batch holds one set
 * of queue counters and scratch: runs of the same batch must not overlap
 * (successive runs on one stream are fine). */
msk_status msk_batch_run(msk_batch* b, void* stream);

/* Autotune: time every variant (queue order x 64^2 packing of the megakernel,
 * and per-item engine launches) on this batch, keep the fastest, append it to
 * `tune_cache` (if given), report the chosen variant and the five times in
 * milliseconds (ms_out[5], nullable). */
msk_status msk_batch_tune(msk_batch* b, void* stream, const char* tune_cache, int* variant_out,
                          float* ms_out);

/* Current variant of the batch (0..3 persistent kernels: bit 0 every path in
 * cluster units with the items interleaved, else 256^2 units plus one-CTA
 * tasks largest grid first; bit 1 one 64^2 path per CTA instead of two; 4: each
 * item's own engine launch), and setting it explicitly (0..4; the next run
 * re-captures the graph). */
int msk_batch_variant(const msk_batch* b);
msk_status msk_batch_set_variant(msk_batch* b, int variant);

const char* msk_batch_last_error(const msk_batch* b);
void msk_batch_destroy(msk_batch* b);

/* S11: learned surrogate of the Magnus solver (not part of the paper).
 *
 * For each path, features x = [dW_k / sqrt(h), int W ds_k / s3,
 * int s dW_k / s3]_{k < K} (h = T/K, s3 = h^1.5/sqrt 3; the Ito integrals of
 * the path's fine increments over each of K equal substeps, piecewise-linear
 * W in each fine cell, single-precision normals from the same Philox words as
 * the solver) are mapped by an MLP of `layers` GELU layers of width `hidden`
 * (bf16 operands, fp32 accumulation) to r scaled POD coefficients c, and
 * u_T = mean + coef_scale * c Phi.  The network is trained by the library's
 * forward/backward kernels and Adam on Magnus solutions (order ref_order,
 * ref_steps steps, float arithmetic) of the same paths.  Serving audits every
 * audit_every-th path against the Magnus solver and falls back to it.
 *
 * Layouts: features uint16 (bfloat16 bits) [paths][3K]; coefficients float
 * [paths][r]; solutions float [paths][v][x]; the flat parameter vector is
 * float, per layer l = 0..layers: W_l [out][in] at offset W_l, then b_l [out]
 * at offset b_l (msk_surrogate_param_layout; every block starts at a multiple
 * of 8 elements).  A surrogate keeps a pointer to its context (which must
 * outlive it) and reads the context's seed, path offset and n_fine at each
 * call; one host thread at a time may use a surrogate. */
typedef struct msk_surrogate msk_surrogate;

typedef struct {
  int32_t steps;         /* K feature substeps (divides n_fine); input width 3K <= 4096 */
  int32_t rank;          /* r POD modes, 1..64 */
  int32_t hidden;        /* hidden width, a multiple of 64 in 64..4096 */
  int32_t layers;        /* hidden layers, 1..8 */
  int32_t train_batch;   /* largest training minibatch (activation buffers) */
  int32_t infer_batch;   /* paths per inference chunk */
  int32_t ref_order;     /* Magnus order of the reference solutions, 1..3 */
  int32_t ref_steps;     /* Magnus steps of the reference solutions (divides n_fine) */
  uint64_t init_seed;    /* Philox key of the He-normal weight init (tag 4) and the POD sketch (tag 3) */
} msk_surrogate_config;

/* Create (weights He-normal N(0, 2/fan_in), biases and Adam state zero); on
 * failure the message is in msk_last_error(ctx). */
msk_status msk_surrogate_create(msk_surrogate** out, msk_ctx* ctx, const msk_surrogate_config* cfg);
void msk_surrogate_destroy(msk_surrogate* s);
const char* msk_surrogate_last_error(const msk_surrogate* s);

/* Number of floats in the flat parameter vector (-1 for NULL), and the offsets
 * of W_l and b_l: offsets_host[2 l], offsets_host[2 l + 1], l = 0..layers. */
int64_t msk_surrogate_num_params(const msk_surrogate* s);
msk_status msk_surrogate_param_layout(const msk_surrogate* s, int64_t* offsets_host);

/* Copy the parameters out / in (set also refreshes the bf16 copy and resets Adam). */
msk_status msk_surrogate_get_params(msk_surrogate* s, float* params_dev, void* stream);
msk_status msk_surrogate_set_params(msk_surrogate* s, const float* params_dev, void* stream);

/* Features of the context's paths path0 .. path0 + paths - 1 into X_dev. */
msk_status msk_surrogate_features(msk_surrogate* s, int64_t path0, int64_t paths, uint16_t* X_dev,
                                  void* stream);

/* Reference solutions (Magnus, ref_order, ref_steps, float) of the same paths
 * into U_dev [paths][d][d]. */
msk_status msk_surrogate_reference(msk_surrogate* s, int64_t path0, int64_t paths, float* U_dev,
                                   void* stream);

/* POD of N snapshots S_dev [N][d][d]: mean and the leading r right singular
 * vectors of S - mean by a randomized range finder (Gaussian sketch of
 * min(r + 16, 80) columns, one power iteration, eigen-orthonormalisation,
 * Rayleigh-Ritz), each mode signed so that its entry of largest magnitude is
 * positive.  Directions with sigma <= 1e-6 sigma_1 (below the resolution of
 * float snapshots) are not resolved: if fewer than r modes remain, the
 * remaining rows of Phi are zero.  coef_scale = sqrt(sum_j sigma_j^2 / (N r))
 * over the resolved modes.  sv_host (nullable) receives the min(r + 16, 80)
 * singular-value estimates.  Synchronises `stream`.  MSK_ERR_ARG if the
 * snapshots do not vary about their mean. */
msk_status msk_surrogate_fit_pod(msk_surrogate* s, const float* S_dev, int64_t N, double* sv_host,
                                 void* stream);

/* Read / set the POD basis: mean [d*d], Phi [r][d*d] (orthonormal rows, or zero), coef_scale.
 * Both synchronise `stream`.  get: any output may be NULL. */
msk_status msk_surrogate_get_pod(msk_surrogate* s, float* mean_dev, float* phi_dev, double* scale_host,
                                 void* stream);
msk_status msk_surrogate_set_pod(msk_surrogate* s, const float* mean_dev, const float* phi_dev,
                                 double coef_scale, void* stream);

/* Scaled coefficients C = (S - mean) Phi^T / coef_scale [N][r] (synchronises),
 * and the decode U = mean + coef_scale C Phi [N][d][d] (U_dev 16-byte aligned). */
msk_status msk_surrogate_project(msk_surrogate* s, const float* S_dev, int64_t N, float* C_dev,
                                 void* stream);
msk_status msk_surrogate_decode(msk_surrogate* s, const float* C_dev, int64_t N, float* U_dev,
                                void* stream);

/* Network output for B feature rows (any B; chunks of infer_batch). */
msk_status msk_surrogate_forward(msk_surrogate* s, const uint16_t* X_dev, int64_t B, float* C_dev,
                                 void* stream);

/* Loss L = (1/B) sum_b sum_j (out_bj - C_bj)^2 of B <= train_batch rows and
 * its gradient (flat, like the parameters) into the surrogate's gradient
 * buffer; loss_dev (float[1]) and grads_dev (float[num_params]) nullable copies. */
msk_status msk_surrogate_loss_grads(msk_surrogate* s, const uint16_t* X_dev, const float* C_dev, int64_t B,
                                    float* loss_dev, float* grads_dev, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the
 * gradient of the last msk_surrogate_loss_grads. */
msk_status msk_surrogate_adam_step(msk_surrogate* s, float lr, void* stream);

/* `epochs` passes over N rows in minibatches of train_batch (in order, the last
 * one ragged), one Adam step each; loss_hist_dev (nullable) float[epochs * nb],
 * nb = ceil(N / train_batch), receives each step's loss. */
msk_status msk_surrogate_train(msk_surrogate* s, const uint16_t* X_dev, const float* C_dev, int64_t N,
                               int epochs, float lr, float* loss_hist_dev, void* stream);

/* Serve paths path0 .. path0 + paths - 1: features, network, decode into U_dev
 * (16-byte aligned).  audit_every > 0: paths j * audit_every of each
 * infer_batch chunk are re-solved by the reference Magnus solver; a path whose
 * relative L2 distance exceeds tol (or is not finite) is replaced by the Magnus
 * solution; if more than max_fail_frac of the audited paths fail, every path
 * is re-solved by Magnus.  flags_dev (nullable) uint32[paths]: bit 0 audited,
 * bit 1 replaced, bit 2 whole-batch fallback.  report_host (nullable)
 * double[5] = {audited, max error, mean error, failed, whole-batch fallback}.
 * With audit_every > 0 the call synchronises `stream`. */
msk_status msk_surrogate_infer(msk_surrogate* s, int64_t path0, int64_t paths, float* U_dev,
                               uint32_t* flags_dev, int64_t audit_every, double tol,
                               double max_fail_frac, double* report_host, void* stream);

/* Test hook of the failure path (no counterpart in the paper): with on != 0 every
 * tensor-core GEMM of this surrogate makes its epilogue warps first wait on an
 * mbarrier that no thread ever arrives at, for a bounded number of polls.  The
 * wait runs out on a healthy pipeline: the warps skip their tiles (still
 * releasing each accumulator), the producer waits for its issued TMA loads and the
 * MMA issuer for its issued MMAs, TMEM is freed, and the next
 * msk_surrogate_sync_status returns MSK_ERR_TIMEOUT (the error word stays set for
 * this surrogate).  The outputs of those calls are undefined.  The GPU context
 * stays usable.  on = 0 restores normal operation (the word is not cleared). */
msk_status msk_surrogate_set_wait_test(msk_surrogate* s, int on);

/* Synchronise `stream` and report the surrogate's device status: MSK_ERR_TIMEOUT
 * if a tensor-core pipeline wait of any earlier call ran out (the affected
 * outputs are invalid), else MSK_OK. */
msk_status msk_surrogate_sync_status(msk_surrogate* s, void* stream);

/* Step-size control (Remark stepSizeControl): for K = k_min, 2 k_min, 4 k_min, ...
 * <= k_max that divide n_fine (at most 16 of them), solve the context's paths
 * 0 .. paths-1 (a subset of trajectories chosen through the seed's path
 * offset) with orders 2 and 3 from the same Brownian functionals, and accept
 * the first K whose largest per-path relative L2 distance between the two
 * solutions (whole grid) is <= tol; a non-finite distance (blow-up) rejects K.
 * *K_out = the accepted K, or the last candidate if none is accepted;
 * dist_host (nullable, double[16]) the distance of every K tried; n_tried
 * (nullable) their number.  Allocates its own scratch and synchronises `stream`. */
msk_status msk_select_steps(msk_ctx* ctx, double tol, int k_min, int k_max, int64_t paths, int precision,
                            int* K_out, double* dist_host, int* n_tried, void* stream);

/* S7: Euler-Maruyama (Eq. EulerMaruyama) with `steps` equal steps, a(t),
 * sigma(t) at the left end of each step, dW the sum of the fine increments. */
msk_status msk_solve_euler(msk_ctx* ctx, int steps, int64_t paths, int precision,
                           void* u_out_dev, uint32_t* path_status_dev, void* stream);

/* S9: closed-form solution for the Gaussian initial datum, per path,
 * u_T = c0 N(M_T m0 + c_T, M_T S0 M_T^T + C_T) (Section 3.1's fundamental
 * solution integrated against the Gaussian datum), u_out_dev [paths][v][x] double. */
msk_status msk_explicit_solution(msk_ctx* ctx, int64_t paths, double* u_out_dev, void* stream);

/* S8: per-path relative Frobenius error over the central 2^-kappa part
 * (Eq. meanErr: Err; index range [lo, lo + floor(d/2^kappa)),
 * lo = floor(d/2 - d/2^(kappa+1))).  ref_kind MSK_REF_EXPLICIT evaluates the
 * closed form on the fly (ref_dev ignored); MSK_REF_BUFFER reads ref_dev
 * ([paths][v][x], element type ref_precision).  err_per_path_dev: double[paths];
 * err_mean_dev: optional double[1] = mean over paths (Err). */
msk_status msk_error(msk_ctx* ctx, const void* u_dev, int u_precision, int64_t paths,
                     int ref_kind, const void* ref_dev, int ref_precision, int kappa,
                     double* err_per_path_dev, double* err_mean_dev, void* stream);

/* Per-path moments of a solution: mom_dev[6 p + r] = mass, mean x, mean v,
 * cov xx, cov xv, cov vv (double). */
msk_status msk_moments(msk_ctx* ctx, const void* u_dev, int precision, int64_t paths,
                       double* mom_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MSK_H */

// Internal declarations shared by the CUDA translation units of libmsk.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/msk.h"

// x-factor class of a basis operator V (x) X: X = I, D^x or (D^x)^2.
enum { XC_I = 0, XC_DX = 1, XC_DXX = 2 };

// Band half-width of the v-factor tables: offsets -2..2 are stored.
#define MSK_BAND 5

struct msk_ctx {
  int device = 0;
  int d = 0;                 // n_x = n_v
  double ax = 0, bx = 0, av = 0, bv = 0, dx = 0, dv = 0;
  msk_coeffs coef{};
  msk_gaussian u0g{};
  uint64_t seed = 0, path_offset = 0;
  int64_t n_fine = 10000;
  double T = 1.0;
  double* u0 = nullptr;       // [d][d] (v-major, x fastest), device
  double* band = nullptr;     // [MSK_NOPS][d][MSK_BAND], device
  double* aux = nullptr;      // [MSK_NOPS] operator traces, then C_T (3), then check flags
  unsigned long long* work = nullptr;   // engine work counter (stencil applications)
  double host_trace[MSK_NOPS] = {0};
  double cT[3] = {0, 0, 0};   // deterministic covariance of the closed form
  double* tab = nullptr;      // per fine cell: sigma(mid), alpha(node), A(mid) (time-dependent coefficients)
  int64_t tab_n = 0;
  double tab_T = 0;
  msk_coeffs tab_coef{};
  void* scratch = nullptr;    // library-owned scratch (functionals + weights)
  size_t scratch_bytes = 0;
  int num_sms = 0;
  // x profile of the variable coefficients (msk_set_x_profile)
  int xprof = 0;              // MSK_XPROF_*; 0: constant-coefficient operators
  double* psi = nullptr;      // [d] psi(x_i), device
  double* var_tab = nullptr;  // 6 traces, 6 shifted norms of the variable-coefficient operators; partials
  bool var_dirty = true;      // var_tab must be rebuilt (profile, a0, drift or general coefficients changed)
  int var_ops_built = 0;      // operators var_tab holds: 6 (constant coefficients) or 13 (time-dependent)
  // general coefficients of Eq. generalSPDE (msk_set_general_coefficients)
  int gen = 0;
  // bumped by every call that changes the operators, coefficients or time grid
  unsigned long long setup_gen = 1;
  // cached infinity norms of the powers of each step's deterministic Omega part
  // (launch_power_norms), for the (steps, order >= 2) of the last solve
  float* pow_tab = nullptr;
  // engine choice (msk_set_engine) and the streamed engine's per-CTA term grids
  int engine_mode = MSK_ENGINE_AUTO;
  void* stream_scratch = nullptr;
  size_t stream_bytes = 0;
  int64_t pow_cap = 0;        // floats allocated
  int pow_steps = 0, pow_o2 = -1;
  unsigned long long pow_gen = 0;
  double* gen64 = nullptr;    // [14][d][d] stencil fields: B (9), A (5)
  float* gen32 = nullptr;
  std::string err;
};

// x-class of each basis operator (same order as the MSK_OP_* enum).
static const int kOpXClass[MSK_NOPS] = {
    XC_DX,  // Bx        = kappa diag(v) (x) D^x
    XC_I,   // Bvv       = D^vv (x) I
    XC_I,   // A0        = D^v (x) I
    XC_I,   // A0^2
    XC_DX,  // [Bx,A0]
    XC_I,   // [Bvv,A0]
    XC_DX,  // [Bx,Bvv]
    XC_DX,  // [[Bx,A0],A0]
    XC_I,   // [[Bvv,A0],A0]
    XC_DXX, // [[Bx,A0],Bx]
    XC_DX,  // [[Bx,A0],Bvv]
    XC_DX,  // [[Bvv,A0],Bx]
    XC_I,   // [[Bvv,A0],Bvv]
};

// Status helpers (host).
msk_status msk_fail(msk_ctx* ctx, msk_status st, const std::string& msg);
msk_status msk_cuda(msk_ctx* ctx, cudaError_t e, const char* what);
msk_status msk_ensure_scratch(msk_ctx* ctx, size_t bytes);
bool msk_supported_d(int d);

// Launchers implemented in the .cu files (all asynchronous on `stream`).
msk_status launch_band_tables(msk_ctx* ctx, cudaStream_t stream);
msk_status launch_gaussian_u0(msk_ctx* ctx, cudaStream_t stream);
// nf32: normals of each Philox pair formed in single precision (the float
// solves); the functionals are accumulated in double either way.
msk_status launch_brownian(msk_ctx* ctx, int steps, int64_t paths, double* out, bool increments_only,
                           cudaStream_t stream, bool nf32 = false);
msk_status launch_brownian_strided(msk_ctx* ctx, int steps, int64_t paths, double* out, uint64_t first,
                                   uint64_t stride, cudaStream_t stream, bool nf32 = false);
msk_status launch_omega(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                        const double* F, double* Wt, cudaStream_t stream);
// Powers of the deterministic part of Omega (Langevin operators with constant or
// time-dependent coefficients): pow_tab[n * MSK_POW_J + q - 1] >= ||X_n^q||_inf for
// q = 1 .. MSK_POW_J, X_n = Omega_n - mu_n I with every Brownian functional set to
// zero (one row when X_n does not depend on n).  The (s, m) selection bounds
// ||(Omega - mu I)^p||^(1/p) with them (Al-Mohy & Higham's alpha_p).
#define MSK_POW_J 9
int power_norm_rows(const msk_ctx* ctx, int steps);   // rows of the table (0: not used for this context)
msk_status launch_power_norms(msk_ctx* ctx, int order, int steps, float* pow_tab, cudaStream_t stream);
// launch_omega with an explicit power-norm table (null: the plain norm bound);
// launch_omega itself uses the context's cached table (allocated on demand).
msk_status launch_omega_tab(msk_ctx* ctx, int order, int steps, int64_t paths, int precision,
                            const double* F, double* Wt, const float* pow_tab, cudaStream_t stream);
msk_status launch_engine(msk_ctx* ctx, bool euler, int steps, int64_t paths, int precision,
                         const double* Wt, const double* dW, void* out, uint32_t* status,
                         cudaStream_t stream);
// Optional engine behaviour for the solutions at output times inside the steps:
// snapshots of the state at step starts into snap[path][q] (q = snap_first[n] ..
// + snap_cnt[n] - 1 at the start of step n, n = 0 .. steps, n = steps meaning after
// the last step; n_out slots per path), and/or starting every path from its own
// output slot (u0_self).  out may be null (final state not stored).
struct EngineSnap {
  void* snap = nullptr;
  const int* snap_first = nullptr;
  const int* snap_cnt = nullptr;
  int n_out = 0;
  int u0_self = 0;
  // Euler-Maruyama: alpha(t_n) dt and sigma(t_n) per step ([steps][2], double and float)
  const double* em_d = nullptr;
  const float* em_f = nullptr;
  // Magnus solves on one CTA per path: the path order and queue counter written by
  // launch_path_order (null: static assignment of paths to CTAs)
  const long long* order = nullptr;
  unsigned long long* queue = nullptr;
  int64_t qlen = 0;   // entries of order the queue hands out (0: paths)
};
// Order the paths by decreasing estimated Taylor cost sum_n s_n m_n (from the
// records Wt) into order[paths] and reset *queue to 0, for the engine's dynamic queue.
// With first > 0: paths first .. first + paths - 1 (order holds their global indices).
msk_status launch_path_order(msk_ctx* ctx, const double* Wt, int steps, int64_t paths, long long* order,
                             unsigned long long* queue, cudaStream_t stream, int64_t first = 0);
// The Magnus engine from the records Wt, with the paths ordered by decreasing
// estimated cost and handed out by a queue when that pays off (order_buf:
// paths entries, queue: one counter; both scratch; null: static assignment).
// queue2 (a second counter, may be null) allows the split solve (engine_split).
msk_status launch_magnus_queued(msk_ctx* ctx, int steps, int64_t paths, int precision, const double* Wt, void* out,
                                uint32_t* status, cudaStream_t stream, long long* order_buf,
                                unsigned long long* queue, unsigned long long* queue2 = nullptr);
// Split solve (engine.cu): the resident engine's clusters fill what they can of the
// device and the streamed engine runs, as their programmatic dependent, on the SMs
// they leave free.  engine_split gives the number n_s of paths of a `paths`-path
// solve that go to the streamed engine (the last n_s indices; 0: no split) and the
// free SMs; launch_engine_split runs it with two path orders and queue counters.
msk_status engine_split(msk_ctx* ctx, int precision, int64_t paths, int64_t* n_s, int64_t* free_sms);
msk_status launch_engine_split(msk_ctx* ctx, int steps, int64_t paths, int64_t n_s, int64_t free_sms, int precision,
                               const double* Wt, void* out, uint32_t* status, cudaStream_t stream,
                               long long* order_buf, unsigned long long* queue, unsigned long long* queue2);
// Fill the Euler table of `steps` steps: em_d[2n] = alpha(t_n) dt, em_d[2n+1] = sigma(t_n), em_f the same in float.
msk_status launch_em_table(msk_ctx* ctx, int steps, double* em_d, float* em_f, cudaStream_t stream);
msk_status launch_engine_ex(msk_ctx* ctx, bool euler, int steps, int64_t paths, int precision,
                            const double* Wt, const double* dW, void* out, uint32_t* status,
                            cudaStream_t stream, const EngineSnap& x);
// Interval mode of the Brownian and weight kernels (times.cu).
msk_status launch_brownian_jobs(msk_ctx* ctx, const int64_t* jobs_dev, int64_t njobs, double* out,
                                cudaStream_t stream, bool nf32);
msk_status launch_omega_jobs(msk_ctx* ctx, int order, int64_t njobs, int precision, const double* F,
                             const double* job_th_dev, double* Wt, cudaStream_t stream);
// Streamed engine (engine_stream.cu): the Magnus solve with every path's state in
// HBM (its output slot and two per-CTA term grids of library scratch), for grids
// whose state does not stay on chip.
bool stream_engine_available(int d, int precision);
// qlen: entries of order the queue hands out (0: paths); grid_cap > 0: at most that
// many CTAs; dependent: launched as the programmatic dependent of the kernel before
// it on the stream (the split solve).
msk_status launch_engine_stream(msk_ctx* ctx, int steps, int64_t paths, int precision, const double* Wt, void* out,
                                uint32_t* status, cudaStream_t stream, const long long* order,
                                unsigned long long* queue, int64_t qlen = 0, int64_t grid_cap = 0,
                                bool dependent = false);
// The streamed engine's term grids for `grid` CTAs (allocated before a split solve's launches).
msk_status ensure_stream_scratch(msk_ctx* ctx, int precision, int64_t grid);
bool resident_engine_available(int d, int precision);
// whether the Magnus solves of this context run the streamed engine (msk_set_engine)
bool engine_is_streamed(const msk_ctx* ctx, int precision);
// Variable-coefficient path (engine_var.cu): the engine, and the traces and
// norms of its six operators for the (s, m) selection (rebuilt when dirty).
msk_status launch_engine_var(msk_ctx* ctx, bool euler, int steps, int64_t paths, int precision,
                             const double* Wt, const double* dW, void* out, uint32_t* status,
                             cudaStream_t stream, const EngineSnap& x);
msk_status ensure_var_tables(msk_ctx* ctx, cudaStream_t stream);
int var_table_ops(const msk_ctx* ctx);
msk_status launch_psi_rational(msk_ctx* ctx, double c, cudaStream_t stream);

// Device-side coefficient profiles.
struct CoefDev {
  int kind;
  double a0, a1, s0, s1;
};

__host__ __device__ inline CoefDev coef_dev(const msk_coeffs& c) {
  CoefDev r;
  r.kind = c.kind;
  r.a0 = c.a0;
  r.s0 = c.s0;
  r.a1 = c.kind == MSK_COEF_TRIG ? c.a1 : 0.0;
  r.s1 = c.kind == MSK_COEF_TRIG ? c.s1 : 0.0;
  return r;
}

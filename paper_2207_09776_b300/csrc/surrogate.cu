// Learned surrogate of the Magnus solver: per-path Brownian features ->
// BF16 MLP -> POD coefficients -> u_T, trained on Magnus solutions by the
// library's own forward/backward kernels, served with a Magnus audit and
// fallback.  C ABI in include/msk.h (msk_surrogate_*).
#include <math.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "surrogate_kernels.cuh"

using namespace sgk;

struct msk_surrogate {
  msk_ctx* ctx = nullptr;
  msk_surrogate_config cfg{};
  int n = 0;                        // grid points d^2
  int in_dim = 0;                   // 3K
  int L = 0;                        // weight layers (hidden layers + output)
  std::vector<int> dims;            // in, H, ..., H, r
  std::vector<int64_t> offW, offB;  // offsets in the flat parameter vector
  int64_t nparam = 0;
  // POD
  float* mean = nullptr;            // [n]
  float* phi = nullptr;             // [r][n]
  double coef_scale = 0;            // network coefficients are (u - mean) Phi^T / coef_scale
  bool pod_ready = false;
  // parameters and Adam state (flat, fp32 master + bf16 copy)
  float* w = nullptr;
  bf16* w16 = nullptr;
  float* grad = nullptr;
  float* am = nullptr;
  float* av = nullptr;
  int64_t t = 0;
  // training activations [train_batch][.]
  std::vector<float*> z;
  std::vector<bf16*> h;
  float* out = nullptr;
  float* g = nullptr;
  bf16* g16 = nullptr;
  float* dz[2] = {nullptr, nullptr};
  bf16* dz16[2] = {nullptr, nullptr};
  float* ws = nullptr;              // split-K workspace
  int64_t ws_elems = 0;
  double* partial = nullptr;        // loss partial sums
  float* loss = nullptr;
  // inference [infer_batch][.]
  bf16* iX = nullptr;
  bf16* ih[2] = {nullptr, nullptr};
  float* iout = nullptr;
  // reference solves and audit (grown on demand)
  void* rs = nullptr;
  size_t rs_bytes = 0;
  float* uref = nullptr;
  size_t uref_bytes = 0;
  double* aerr = nullptr;
  size_t aerr_bytes = 0;
  std::string err;
};

namespace {

constexpr int kLossBlocks = 296;
// POD: directions whose squared singular value is below kRelKeep times the
// largest are below the resolution of float snapshots (sigma < 1e-6 sigma_max)
// and are dropped.
constexpr double kRelKeep = 1e-12;
constexpr int kRefChunk = 32768;   // paths per reference-solve launch group

msk_status sfail(msk_surrogate* s, msk_status st, const std::string& msg) {
  if (s) s->err = msg;
  return st;
}

msk_status scuda(msk_surrogate* s, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MSK_OK;
  cudaGetLastError();
  return sfail(s, e == cudaErrorMemoryAllocation ? MSK_ERR_OOM : MSK_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

// Propagate a failure of a context-level launcher into the surrogate's message.
msk_status from_ctx(msk_surrogate* s, msk_status st) {
  if (st != MSK_OK) s->err = s->ctx->err;
  return st;
}

template <typename T>
msk_status salloc(msk_surrogate* s, T** p, size_t elems, const char* what) {
  return scuda(s, cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(elems, 1) * sizeof(T)), what);
}

template <typename T>
msk_status sgrow(msk_surrogate* s, T** p, size_t* bytes, size_t want, const char* what) {
  if (want <= *bytes) return MSK_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *bytes = 0;
  msk_status st = scuda(s, cudaMalloc(reinterpret_cast<void**>(p), want), what);
  if (st == MSK_OK) *bytes = want;
  return st;
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// One BF16 GEMM launch (see gemm_bf16_kernel); EPI_F32 with splits > 1 writes
// the split-K partials to the workspace and reduces them into C in fixed order.
template <bool A_KC, bool B_KC, int EPI>
msk_status gemm(msk_surrogate* s, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, float* C,
                int ldc, bf16* C16, int ldc16, const float* bias, const float* aux, int ldaux, bool split,
                cudaStream_t stream) {
  if (M == 0 || N == 0) return MSK_OK;
  GemmArgs g{};
  g.A = A;
  g.B = B;
  g.M = M;
  g.N = N;
  g.K = K;
  g.lda = lda;
  g.ldb = ldb;
  g.vecA = aligned16(A) && lda % 8 == 0;
  g.vecB = aligned16(B) && ldb % 8 == 0;
  g.C = C;
  g.ldc = ldc;
  g.C16 = C16;
  g.ldc16 = ldc16;
  g.bias = bias;
  g.aux = aux;
  g.ldaux = ldaux;
  const int bm = (M + GBM - 1) / GBM, bn = (N + GBN - 1) / GBN;
  int splits = 1, kchunk = ((K + GBK - 1) / GBK) * GBK;
  if (split && EPI == EPI_F32) {
    const int want = std::max(1, (2 * s->ctx->num_sms + bm * bn - 1) / (bm * bn));
    splits = std::min(want, std::max(1, K / 64));
    kchunk = ((K + splits - 1) / splits + GBK - 1) / GBK * GBK;
    splits = (K + kchunk - 1) / kchunk;
    if (splits > 1 && (int64_t)splits * M * N > s->ws_elems) {   // workspace too small: no split
      splits = 1;
      kchunk = ((K + GBK - 1) / GBK) * GBK;
    }
  }
  g.kchunk = std::max(kchunk, GBK);
  if (splits > 1) {
    g.C = s->ws;
    g.ldc = N;
    g.split_stride = (int64_t)M * N;
  }
  gemm_bf16_kernel<A_KC, B_KC, EPI><<<dim3(bn, bm, splits), 256, 0, stream>>>(g);
  msk_status st = scuda(s, cudaGetLastError(), "gemm kernel");
  if (st != MSK_OK || splits == 1) return st;
  // C is contiguous [M][N] (weight gradients)
  reduce_splits_kernel<<<blocks_for((int64_t)M * N), 256, 0, stream>>>(s->ws, splits, (int64_t)M * N, C);
  return scuda(s, cudaGetLastError(), "split-K reduction");
}

// Forward pass of B rows of X.  train: keeps z_l and h_l of every hidden layer;
// otherwise ping-pongs the inference buffers.  Output: out [B][r] (fp32).
msk_status forward_chain(msk_surrogate* s, const bf16* X, int64_t B, bool train, float* out, cudaStream_t stream) {
  const bf16* hin = X;
  int in = s->in_dim;
  const int H = s->cfg.hidden;
  for (int l = 0; l < s->L - 1; ++l) {
    float* zl = train ? s->z[l] : nullptr;
    bf16* hl = train ? s->h[l] : s->ih[l & 1];
    msk_status st = gemm<true, true, EPI_BIAS_GELU>(s, hin, in, s->w16 + s->offW[l], in, (int)B, H, in, zl, H, hl, H,
                                                    s->w + s->offB[l], nullptr, 0, false, stream);
    if (st != MSK_OK) return st;
    hin = hl;
    in = H;
  }
  const int l = s->L - 1, r = s->cfg.rank;
  return gemm<true, true, EPI_BIAS_F32>(s, hin, in, s->w16 + s->offW[l], in, (int)B, r, in, out, r, nullptr, 0,
                                        s->w + s->offB[l], nullptr, 0, false, stream);
}

// Loss and gradients of one minibatch (B <= train_batch) into s->grad and s->loss.
msk_status loss_grads(msk_surrogate* s, const bf16* X, const float* C, int64_t B, cudaStream_t stream) {
  msk_status st = forward_chain(s, X, B, true, s->out, stream);
  if (st != MSK_OK) return st;
  const int r = s->cfg.rank, H = s->cfg.hidden, L = s->L;
  loss_grad_kernel<<<kLossBlocks, 256, 0, stream>>>(s->out, C, B * r, 1.0f / (float)B, s->g, s->g16, s->partial);
  loss_final_kernel<<<1, 256, 0, stream>>>(s->partial, kLossBlocks, 1.0 / (double)B, s->loss);
  st = scuda(s, cudaGetLastError(), "loss kernels");
  if (st != MSK_OK) return st;
  const bf16* cur16 = s->g16;
  const float* cur = s->g;
  int cur_dim = r;
  for (int l = L - 1; l >= 0; --l) {
    const int in = s->dims[l];
    const bf16* hprev = l > 0 ? s->h[l - 1] : X;
    // dW_l = dz_l^T h_{l-1}  ([out][in], split-K over the batch)
    st = gemm<false, false, EPI_F32>(s, cur16, cur_dim, hprev, in, cur_dim, in, (int)B, s->grad + s->offW[l], in,
                                     nullptr, 0, nullptr, nullptr, 0, true, stream);
    if (st != MSK_OK) return st;
    colsum_kernel<<<blocks_for(cur_dim, 32), dim3(32, 8), 0, stream>>>(cur, (int)B, cur_dim, s->grad + s->offB[l]);
    st = scuda(s, cudaGetLastError(), "bias gradient");
    if (st != MSK_OK) return st;
    if (l == 0) break;
    // dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1})
    float* nd = s->dz[l & 1];
    bf16* nd16 = s->dz16[l & 1];
    st = gemm<true, false, EPI_GELU_BWD>(s, cur16, cur_dim, s->w16 + s->offW[l], in, (int)B, H, cur_dim, nd, H, nd16,
                                         H, nullptr, s->z[l - 1], H, false, stream);
    if (st != MSK_OK) return st;
    cur = nd;
    cur16 = nd16;
    cur_dim = H;
  }
  return MSK_OK;
}

msk_status adam(msk_surrogate* s, float lr, cudaStream_t stream) {
  s->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - pow(b1, (double)s->t)), c2 = (float)(1.0 - pow(b2, (double)s->t));
  adam_kernel<<<blocks_for(s->nparam), 256, 0, stream>>>(s->w, s->w16, s->grad, s->am, s->av, s->nparam, lr,
                                                         (float)b1, (float)b2, 1e-8f, c1, c2);
  return scuda(s, cudaGetLastError(), "adam kernel");
}

// Magnus FP32 solutions (reference order/steps) of the global paths
// first + i * stride, i < paths, into U [paths][n].
msk_status reference_solve(msk_surrogate* s, uint64_t first, uint64_t stride, int64_t paths, float* U,
                           cudaStream_t stream) {
  msk_ctx* ctx = s->ctx;
  const int steps = s->cfg.ref_steps, order = s->cfg.ref_order;
  for (int64_t o = 0; o < paths; o += kRefChunk) {
    const int64_t P = std::min<int64_t>(kRefChunk, paths - o);
    const size_t nF = (size_t)P * steps * MSK_NF, nW = (size_t)P * steps * MSK_NWT;
    msk_status st = sgrow(s, &s->rs, &s->rs_bytes, (nF + nW) * sizeof(double), "reference scratch");
    if (st != MSK_OK) return st;
    double* F = reinterpret_cast<double*>(s->rs);
    double* Wt = F + nF;
    st = from_ctx(s, launch_brownian_strided(ctx, steps, P, F, first + (uint64_t)o * stride, stride, stream));
    if (st == MSK_OK) st = from_ctx(s, launch_omega(ctx, order, steps, P, MSK_F32, F, Wt, stream));
    if (st == MSK_OK)
      st = from_ctx(s, launch_engine(ctx, false, steps, P, MSK_F32, Wt, nullptr, U + (size_t)o * s->n, nullptr, stream));
    if (st != MSK_OK) return st;
  }
  return MSK_OK;
}

msk_status features(msk_surrogate* s, uint64_t first, int64_t paths, bf16* X, cudaStream_t stream) {
  if (paths == 0) return MSK_OK;
  const int K = s->cfg.steps;
  features_kernel<<<blocks_for(paths * K * 32), 256, 0, stream>>>(s->ctx->seed, first, 1, paths, K, s->ctx->n_fine, X);
  return scuda(s, cudaGetLastError(), "features kernel");
}

msk_status decode(msk_surrogate* s, const float* C, int64_t P, float* U, cudaStream_t stream) {
  if (P == 0) return MSK_OK;
  const dim3 grid(blocks_for(s->n / 4), (unsigned)((P + 7) / 8));
  // coefficients are scaled: u = mean + coef_scale * C Phi.  The scale is folded
  // into Phi at fit/set time (phi holds coef_scale * Phi).
  decode_kernel<<<grid, 256, 0, stream>>>(C, P, s->cfg.rank, s->phi, s->mean, s->n, U);
  return scuda(s, cudaGetLastError(), "decode kernel");
}

void free_all(msk_surrogate* s) {
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  F(s->mean);
  F(s->phi);
  F(s->w);
  F(s->w16);
  F(s->grad);
  F(s->am);
  F(s->av);
  for (float* p : s->z) F(p);
  for (bf16* p : s->h) F(p);
  F(s->out);
  F(s->g);
  F(s->g16);
  for (int i = 0; i < 2; ++i) {
    F(s->dz[i]);
    F(s->dz16[i]);
    F(s->ih[i]);
  }
  F(s->ws);
  F(s->partial);
  F(s->loss);
  F(s->iX);
  F(s->iout);
  F(s->rs);
  F(s->uref);
  F(s->aerr);
}

// The context's n_fine may change after creation (msk_set_seed).
msk_status check_fine(msk_surrogate* s) {
  const int64_t nf = s->ctx->n_fine;
  if (nf % s->cfg.steps != 0 || nf % s->cfg.ref_steps != 0)
    return sfail(s, MSK_ERR_ARG, "steps and ref_steps must divide the context's n_fine");
  return MSK_OK;
}

msk_status check_pod(msk_surrogate* s) {
  return s->pod_ready ? MSK_OK : sfail(s, MSK_ERR_ARG, "POD basis not set (msk_surrogate_fit_pod / set_pod)");
}

}  // namespace

// ============================================================================ C ABI

extern "C" const char* msk_surrogate_last_error(const msk_surrogate* s) {
  return s ? s->err.c_str() : "null surrogate";
}

extern "C" void msk_surrogate_destroy(msk_surrogate* s) {
  if (!s) return;
  cudaSetDevice(s->ctx->device);
  free_all(s);
  delete s;
}

extern "C" int64_t msk_surrogate_num_params(const msk_surrogate* s) { return s ? s->nparam : -1; }

extern "C" msk_status msk_surrogate_create(msk_surrogate** out, msk_ctx* ctx, const msk_surrogate_config* cfg) {
  if (!out) return MSK_ERR_ARG;
  *out = nullptr;
  if (!ctx || !cfg) return MSK_ERR_ARG;
  const msk_surrogate_config& c = *cfg;
  if (c.steps < 1 || ctx->n_fine % c.steps != 0) return msk_fail(ctx, MSK_ERR_ARG, "steps must divide n_fine");
  if (c.rank < 1 || c.rank > 64) return msk_fail(ctx, MSK_ERR_ARG, "rank must be in 1..64");
  if (c.hidden < 64 || c.hidden > 4096 || c.hidden % 64 != 0)
    return msk_fail(ctx, MSK_ERR_ARG, "hidden must be a multiple of 64 in 64..4096");
  if (c.layers < 1 || c.layers > 8) return msk_fail(ctx, MSK_ERR_ARG, "layers must be in 1..8");
  if (c.train_batch < 1 || c.infer_batch < 1) return msk_fail(ctx, MSK_ERR_ARG, "batch sizes must be >= 1");
  if (c.ref_order < 1 || c.ref_order > 3) return msk_fail(ctx, MSK_ERR_ARG, "ref_order must be 1, 2 or 3");
  if (c.ref_steps < 1 || ctx->n_fine % c.ref_steps != 0) return msk_fail(ctx, MSK_ERR_ARG, "ref_steps must divide n_fine");
  if (3 * c.steps > 4096) return msk_fail(ctx, MSK_ERR_ARG, "3 * steps must be <= 4096");
  msk_surrogate* s = new (std::nothrow) msk_surrogate();
  if (!s) return msk_fail(ctx, MSK_ERR_OOM, "host allocation");
  s->ctx = ctx;
  s->cfg = c;
  s->n = ctx->d * ctx->d;
  s->in_dim = 3 * c.steps;
  s->L = c.layers + 1;
  s->dims.push_back(s->in_dim);
  for (int l = 0; l < c.layers; ++l) s->dims.push_back(c.hidden);
  s->dims.push_back(c.rank);
  int64_t off = 0;
  for (int l = 0; l < s->L; ++l) {
    const int64_t fin = s->dims[l], fout = s->dims[l + 1];
    s->offW.push_back(off);
    off += fout * fin;
    off = (off + 7) / 8 * 8;   // keep every block 16-byte aligned in the bf16 copy
    s->offB.push_back(off);
    off += fout;
    off = (off + 7) / 8 * 8;
  }
  s->nparam = off;
  const int64_t TB = c.train_batch, IB = c.infer_batch, H = c.hidden, r = c.rank;
  msk_status st = scuda(s, cudaSetDevice(ctx->device), "set device");
  if (st == MSK_OK) st = salloc(s, &s->mean, s->n, "POD mean");
  if (st == MSK_OK) st = salloc(s, &s->phi, (size_t)r * s->n, "POD basis");
  if (st == MSK_OK) st = salloc(s, &s->w, s->nparam, "parameters");
  if (st == MSK_OK) st = salloc(s, &s->w16, s->nparam, "bf16 parameters");
  if (st == MSK_OK) st = salloc(s, &s->grad, s->nparam, "gradients");
  if (st == MSK_OK) st = salloc(s, &s->am, s->nparam, "Adam m");
  if (st == MSK_OK) st = salloc(s, &s->av, s->nparam, "Adam v");
  s->z.assign(c.layers, nullptr);
  s->h.assign(c.layers, nullptr);
  for (int l = 0; l < c.layers && st == MSK_OK; ++l) {
    st = salloc(s, &s->z[l], (size_t)TB * H, "activations");
    if (st == MSK_OK) st = salloc(s, &s->h[l], (size_t)TB * H, "activations");
  }
  if (st == MSK_OK) st = salloc(s, &s->out, (size_t)TB * r, "outputs");
  if (st == MSK_OK) st = salloc(s, &s->g, (size_t)TB * r, "output gradient");
  if (st == MSK_OK) st = salloc(s, &s->g16, (size_t)TB * r, "output gradient");
  for (int i = 0; i < 2 && st == MSK_OK; ++i) {
    st = salloc(s, &s->dz[i], (size_t)TB * H, "backward buffers");
    if (st == MSK_OK) st = salloc(s, &s->dz16[i], (size_t)TB * H, "backward buffers");
    if (st == MSK_OK) st = salloc(s, &s->ih[i], (size_t)IB * H, "inference buffers");
  }
  // split-K workspace: up to 2 * SMs splits of the largest weight gradient
  s->ws_elems = (int64_t)2 * std::max(ctx->num_sms, 1) * std::max<int64_t>(H * H, H * std::max<int64_t>(r, s->in_dim));
  s->ws_elems = std::min<int64_t>(s->ws_elems, (int64_t)16 * H * H + 1);
  if (st == MSK_OK) st = salloc(s, &s->ws, s->ws_elems, "split-K workspace");
  if (st == MSK_OK) st = salloc(s, &s->partial, kLossBlocks, "loss partials");
  if (st == MSK_OK) st = salloc(s, &s->loss, 1, "loss");
  if (st == MSK_OK) st = salloc(s, &s->iX, (size_t)IB * s->in_dim, "inference features");
  if (st == MSK_OK) st = salloc(s, &s->iout, (size_t)IB * r, "inference outputs");
  if (st == MSK_OK)
    st = scuda(s, cudaFuncSetAttribute(sym_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * SK_Q * SK_Q * (int)sizeof(double) + SK_Q * (int)sizeof(int)),
               "eigen kernel attribute");
  // parameters: He-normal weights (Philox tag 4, counter blocks per layer), zero biases, zero Adam state
  if (st == MSK_OK) st = scuda(s, cudaMemset(s->w, 0, s->nparam * sizeof(float)), "parameter init");
  for (int l = 0; l < s->L && st == MSK_OK; ++l) {
    const int64_t cnt = (int64_t)s->dims[l + 1] * s->dims[l];
    init_weights_kernel<<<blocks_for(cnt), 256>>>(s->w + s->offW[l], cnt, s->dims[l], c.init_seed,
                                                  (uint64_t)l << 40);
    st = scuda(s, cudaGetLastError(), "weight init");
  }
  if (st == MSK_OK) {
    to_bf16_kernel<<<blocks_for(s->nparam), 256>>>(s->w, s->w16, s->nparam);
    st = scuda(s, cudaGetLastError(), "bf16 copy");
  }
  if (st == MSK_OK) st = scuda(s, cudaMemset(s->am, 0, s->nparam * sizeof(float)), "Adam init");
  if (st == MSK_OK) st = scuda(s, cudaMemset(s->av, 0, s->nparam * sizeof(float)), "Adam init");
  if (st == MSK_OK) st = scuda(s, cudaMemset(s->grad, 0, s->nparam * sizeof(float)), "gradient init");
  if (st == MSK_OK) st = scuda(s, cudaDeviceSynchronize(), "surrogate init");
  if (st != MSK_OK) {
    msk_fail(ctx, st, s->err);
    free_all(s);
    delete s;
    return st;
  }
  *out = s;
  return MSK_OK;
}

extern "C" msk_status msk_surrogate_get_params(msk_surrogate* s, float* params_dev, void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (!params_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  return scuda(s, cudaMemcpyAsync(params_dev, s->w, s->nparam * sizeof(float), cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream), "copy parameters");
}

extern "C" msk_status msk_surrogate_set_params(msk_surrogate* s, const float* params_dev, void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (!params_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  cudaStream_t st_ = (cudaStream_t)stream;
  msk_status st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st == MSK_OK)
    st = scuda(s, cudaMemcpyAsync(s->w, params_dev, s->nparam * sizeof(float), cudaMemcpyDeviceToDevice, st_),
               "copy parameters");
  if (st != MSK_OK) return st;
  to_bf16_kernel<<<blocks_for(s->nparam), 256, 0, st_>>>(s->w, s->w16, s->nparam);
  st = scuda(s, cudaGetLastError(), "bf16 copy");
  if (st == MSK_OK) st = scuda(s, cudaMemsetAsync(s->am, 0, s->nparam * sizeof(float), st_), "Adam reset");
  if (st == MSK_OK) st = scuda(s, cudaMemsetAsync(s->av, 0, s->nparam * sizeof(float), st_), "Adam reset");
  s->t = 0;
  return st;
}

extern "C" msk_status msk_surrogate_param_layout(const msk_surrogate* s, int64_t* offsets_host) {
  if (!s || !offsets_host) return MSK_ERR_ARG;
  for (int l = 0; l < s->L; ++l) {
    offsets_host[2 * l] = s->offW[l];
    offsets_host[2 * l + 1] = s->offB[l];
  }
  return MSK_OK;
}

extern "C" msk_status msk_surrogate_features(msk_surrogate* s, int64_t path0, int64_t paths, uint16_t* X_dev,
                                             void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (path0 < 0 || paths < 0) return sfail(s, MSK_ERR_ARG, "negative path range");
  if (paths == 0) return MSK_OK;
  if (!X_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  msk_status st = check_fine(s);
  if (st != MSK_OK) return st;
  st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st != MSK_OK) return st;
  return features(s, s->ctx->path_offset + (uint64_t)path0, paths, reinterpret_cast<bf16*>(X_dev),
                  (cudaStream_t)stream);
}

extern "C" msk_status msk_surrogate_reference(msk_surrogate* s, int64_t path0, int64_t paths, float* U_dev,
                                              void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (path0 < 0 || paths < 0) return sfail(s, MSK_ERR_ARG, "negative path range");
  if (paths == 0) return MSK_OK;
  if (!U_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  msk_status st = check_fine(s);
  if (st != MSK_OK) return st;
  st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st != MSK_OK) return st;
  return reference_solve(s, s->ctx->path_offset + (uint64_t)path0, 1, paths, U_dev, (cudaStream_t)stream);
}

extern "C" msk_status msk_surrogate_fit_pod(msk_surrogate* s, const float* S_dev, int64_t N, double* sv_host,
                                            void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (N < 1) return sfail(s, MSK_ERR_ARG, "need at least one snapshot");
  if (!S_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  cudaStream_t stm = (cudaStream_t)stream;
  msk_status st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st != MSK_OK) return st;
  const int n = s->n, r = s->cfg.rank, Q = std::min(r + 16, SK_Q);
  // scratch
  const int chunks = (int)std::min<int64_t>(256, (N + 255) / 256);
  const int64_t rows_chunk = (N + chunks - 1) / chunks;
  const int ysplit = (int)std::min<int64_t>(8, std::max<int64_t>(1, N / 1024));
  const int64_t yrows = (N + ysplit - 1) / ysplit;
  const int64_t gc_rows = std::max<int64_t>(1024, (N + 511) / 512);
  const int gc_blocks = (int)((N + gc_rows - 1) / gc_rows);
  double *part = nullptr, *Gm = nullptr, *M = nullptr, *sv = nullptr, *gpart = nullptr;
  float *G = nullptr, *Ypart = nullptr, *Y = nullptr, *Qa = nullptr, *Qb = nullptr;
  int* kept_d = nullptr;
  auto cleanup = [&]() {
    for (void* p : {(void*)part, (void*)Gm, (void*)M, (void*)sv, (void*)gpart, (void*)G, (void*)Ypart, (void*)Y,
                    (void*)Qa, (void*)Qb, (void*)kept_d})
      if (p) cudaFree(p);
  };
  st = salloc(s, &part, (size_t)chunks * n, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &G, (size_t)N * Q, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &Ypart, (size_t)ysplit * Q * n, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &Y, (size_t)Q * n, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &Qa, (size_t)Q * n, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &Qb, (size_t)Q * n, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &Gm, (size_t)Q * Q, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &M, (size_t)Q * Q, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &sv, (size_t)Q, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &gpart, (size_t)gc_blocks * Q * Q, "POD scratch");
  if (st == MSK_OK) st = salloc(s, &kept_d, 1, "POD scratch");
  if (st != MSK_OK) {
    cleanup();
    return st;
  }
  const size_t eig_smem = 2 * (size_t)Q * Q * sizeof(double) + Q * sizeof(int);
  int kept = 0;
  // sketch of the row space: Y = W^T (S - mean), W [N][q] (Gaussian or the previous Z)
  auto sketch = [&](const float* W, int q) -> msk_status {
    sketch_kernel<<<dim3(blocks_for(n, SK_F), ysplit), 256, 0, stm>>>(S_dev, s->mean, W, N, n, q, yrows, Ypart);
    reduce_splits_kernel<<<blocks_for((int64_t)q * n), 256, 0, stm>>>(Ypart, ysplit, (int64_t)q * n, Y);
    return scuda(s, cudaGetLastError(), "POD sketch");
  };
  // orthonormal rows spanning the rows of In (q x n): eigen-decomposition of In In^T
  auto orth = [&](const float* In, int q, float* Out) -> msk_status {
    gram_rows_kernel<<<dim3(q, q), 256, 0, stm>>>(In, q, n, Gm);
    sym_eig_kernel<<<1, 128, eig_smem, stm>>>(Gm, q, 0, kRelKeep, 0, M, kept_d, nullptr);
    msk_status e = scuda(s, cudaGetLastError(), "POD orthonormalisation");
    if (e == MSK_OK) e = scuda(s, cudaMemcpyAsync(&kept, kept_d, sizeof(int), cudaMemcpyDeviceToHost, stm), "copy");
    if (e == MSK_OK) e = scuda(s, cudaStreamSynchronize(stm), "POD sync");
    if (e != MSK_OK) return e;
    if (kept < 1) return sfail(s, MSK_ERR_ARG, "snapshots have no variation about their mean");
    small_left_mul_kernel<<<dim3(blocks_for(n), kept), 256, 0, stm>>>(M, kept, q, In, n, Out);
    return scuda(s, cudaGetLastError(), "POD basis update");
  };
  // 1. mean
  colsum_partial_kernel<<<dim3(blocks_for(n), chunks), 256, 0, stm>>>(S_dev, N, n, rows_chunk, part);
  colmean_final_kernel<<<blocks_for(n), 256, 0, stm>>>(part, chunks, n, N, s->mean);
  // 2. Gaussian sketch and two orthonormalisation passes
  gaussian_kernel<<<blocks_for(N * Q), 256, 0, stm>>>(G, N * Q, s->cfg.init_seed);
  st = scuda(s, cudaGetLastError(), "POD mean / test matrix");
  if (st == MSK_OK) st = sketch(G, Q);
  if (st == MSK_OK) st = orth(Y, Q, Qa);
  int q = kept;
  if (st == MSK_OK) st = orth(Qa, q, Qb);
  q = kept;
  // 3. one power iteration: Z = (S - mean) Qb^T, Y = Z^T (S - mean)
  if (st == MSK_OK) {
    rows_dot_kernel<<<(unsigned)((N + PR_R - 1) / PR_R), 256, 0, stm>>>(S_dev, s->mean, N, n, Qb, q, G);
    st = scuda(s, cudaGetLastError(), "POD projection");
  }
  if (st == MSK_OK) st = sketch(G, q);
  if (st == MSK_OK) st = orth(Y, q, Qa);
  q = kept;
  if (st == MSK_OK) st = orth(Qa, q, Qb);
  q = kept;
  // 4. Rayleigh-Ritz: Z = (S - mean) Qb^T, Z^T Z = V Lambda V^T, Phi = V^T Qb
  if (st == MSK_OK) {
    rows_dot_kernel<<<(unsigned)((N + PR_R - 1) / PR_R), 256, 0, stm>>>(S_dev, s->mean, N, n, Qb, q, G);
    gram_cols_partial_kernel<<<gc_blocks, 256, 0, stm>>>(G, N, q, gc_rows, gpart);
    sum_partials_d_kernel<<<blocks_for((int64_t)q * q), 256, 0, stm>>>(gpart, gc_blocks, (int64_t)q * q, Gm);
    sym_eig_kernel<<<1, 128, eig_smem, stm>>>(Gm, q, 1, kRelKeep, r, M, kept_d, sv);
    st = scuda(s, cudaGetLastError(), "POD Rayleigh-Ritz");
  }
  double svh[SK_Q] = {0};
  if (st == MSK_OK) st = scuda(s, cudaMemcpyAsync(&kept, kept_d, sizeof(int), cudaMemcpyDeviceToHost, stm), "copy");
  if (st == MSK_OK) st = scuda(s, cudaMemcpyAsync(svh, sv, q * sizeof(double), cudaMemcpyDeviceToHost, stm), "copy");
  if (st == MSK_OK) st = scuda(s, cudaStreamSynchronize(stm), "POD sync");
  const int modes = kept;   // resolved modes; rows modes..r-1 of the basis are zero
  if (st == MSK_OK) {
    double e2 = 0;
    for (int j = 0; j < modes; ++j) e2 += svh[j] * svh[j];
    s->coef_scale = sqrt(e2 / ((double)N * r));
    if (!(s->coef_scale > 0)) st = sfail(s, MSK_ERR_ARG, "zero POD energy");
  }
  if (st == MSK_OK) st = scuda(s, cudaMemsetAsync(Qa, 0, (size_t)r * n * sizeof(float), stm), "POD basis");
  if (st == MSK_OK && modes > 0) {
    small_left_mul_kernel<<<dim3(blocks_for(n), modes), 256, 0, stm>>>(M, modes, q, Qb, n, Qa);
    fix_sign_kernel<<<modes, 256, 0, stm>>>(Qa, n);
    st = scuda(s, cudaGetLastError(), "POD basis");
  }
  // stored basis holds coef_scale * Phi (decode multiplies coefficients back)
  if (st == MSK_OK) {
    const double sc = s->coef_scale;
    std::vector<double> scale_m((size_t)r * r, 0.0);
    for (int j = 0; j < r; ++j) scale_m[(size_t)j * r + j] = sc;
    st = scuda(s, cudaMemcpyAsync(M, scale_m.data(), scale_m.size() * sizeof(double), cudaMemcpyHostToDevice, stm),
               "copy");
    if (st == MSK_OK) {
      small_left_mul_kernel<<<dim3(blocks_for(n), r), 256, 0, stm>>>(M, r, r, Qa, n, s->phi);
      st = scuda(s, cudaGetLastError(), "POD basis scaling");
    }
    if (st == MSK_OK) st = scuda(s, cudaStreamSynchronize(stm), "POD sync");
  }
  if (st == MSK_OK && sv_host)
    for (int j = 0; j < Q; ++j) sv_host[j] = j < q ? svh[j] : 0.0;
  if (st == MSK_OK) s->pod_ready = true;
  cleanup();
  return st;
}

extern "C" msk_status msk_surrogate_get_pod(msk_surrogate* s, float* mean_dev, float* phi_dev, double* scale_host,
                                            void* stream) {
  if (!s) return MSK_ERR_ARG;
  msk_status st = check_pod(s);
  if (st != MSK_OK) return st;
  cudaStream_t stm = (cudaStream_t)stream;
  if (mean_dev)
    st = scuda(s, cudaMemcpyAsync(mean_dev, s->mean, s->n * sizeof(float), cudaMemcpyDeviceToDevice, stm), "copy");
  if (st == MSK_OK && phi_dev) {
    // return the orthonormal basis: phi / coef_scale
    const int r = s->cfg.rank;
    std::vector<double> m((size_t)r * r, 0.0);
    for (int j = 0; j < r; ++j) m[(size_t)j * r + j] = 1.0 / s->coef_scale;
    double* Md = nullptr;
    st = salloc(s, &Md, m.size(), "scratch");
    if (st == MSK_OK) st = scuda(s, cudaMemcpy(Md, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice), "copy");
    if (st == MSK_OK) {
      small_left_mul_kernel<<<dim3(blocks_for(s->n), r), 256, 0, stm>>>(Md, r, r, s->phi, s->n, phi_dev);
      st = scuda(s, cudaGetLastError(), "POD basis copy");
    }
    if (st == MSK_OK) st = scuda(s, cudaStreamSynchronize(stm), "sync");
    if (Md) cudaFree(Md);
  }
  if (st == MSK_OK && scale_host) *scale_host = s->coef_scale;
  return st;
}

extern "C" msk_status msk_surrogate_set_pod(msk_surrogate* s, const float* mean_dev, const float* phi_dev,
                                            double coef_scale, void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (!mean_dev || !phi_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  if (!(coef_scale > 0) || !isfinite(coef_scale)) return sfail(s, MSK_ERR_ARG, "coef_scale must be positive");
  cudaStream_t stm = (cudaStream_t)stream;
  msk_status st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st == MSK_OK)
    st = scuda(s, cudaMemcpyAsync(s->mean, mean_dev, s->n * sizeof(float), cudaMemcpyDeviceToDevice, stm), "copy");
  const int r = s->cfg.rank;
  std::vector<double> m((size_t)r * r, 0.0);
  for (int j = 0; j < r; ++j) m[(size_t)j * r + j] = coef_scale;
  double* Md = nullptr;
  if (st == MSK_OK) st = salloc(s, &Md, m.size(), "scratch");
  if (st == MSK_OK) st = scuda(s, cudaMemcpy(Md, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice), "copy");
  if (st == MSK_OK) {
    small_left_mul_kernel<<<dim3(blocks_for(s->n), r), 256, 0, stm>>>(Md, r, r, phi_dev, s->n, s->phi);
    st = scuda(s, cudaGetLastError(), "POD basis copy");
  }
  if (st == MSK_OK) st = scuda(s, cudaStreamSynchronize(stm), "sync");
  if (Md) cudaFree(Md);
  if (st == MSK_OK) {
    s->coef_scale = coef_scale;
    s->pod_ready = true;
  }
  return st;
}

extern "C" msk_status msk_surrogate_project(msk_surrogate* s, const float* S_dev, int64_t N, float* C_dev,
                                            void* stream) {
  if (!s) return MSK_ERR_ARG;
  msk_status st = check_pod(s);
  if (st != MSK_OK) return st;
  if (N < 0) return sfail(s, MSK_ERR_ARG, "N < 0");
  if (N == 0) return MSK_OK;
  if (!S_dev || !C_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  // phi holds coef_scale * Phi, so (S - mean) phi^T / coef_scale^2 = (S - mean) Phi^T / coef_scale
  // is computed as (S - mean) (phi / coef_scale^2)^T.
  const int r = s->cfg.rank;
  cudaStream_t stm = (cudaStream_t)stream;
  float* B = nullptr;
  double* Md = nullptr;
  st = salloc(s, &B, (size_t)r * s->n, "scratch");
  std::vector<double> m((size_t)r * r, 0.0);
  for (int j = 0; j < r; ++j) m[(size_t)j * r + j] = 1.0 / (s->coef_scale * s->coef_scale);
  if (st == MSK_OK) st = salloc(s, &Md, m.size(), "scratch");
  if (st == MSK_OK) st = scuda(s, cudaMemcpy(Md, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice), "copy");
  if (st == MSK_OK) {
    small_left_mul_kernel<<<dim3(blocks_for(s->n), r), 256, 0, stm>>>(Md, r, r, s->phi, s->n, B);
    rows_dot_kernel<<<(unsigned)((N + PR_R - 1) / PR_R), 256, 0, stm>>>(S_dev, s->mean, N, s->n, B, r, C_dev);
    st = scuda(s, cudaGetLastError(), "projection");
  }
  if (st == MSK_OK) st = scuda(s, cudaStreamSynchronize(stm), "sync");
  if (B) cudaFree(B);
  if (Md) cudaFree(Md);
  return st;
}

extern "C" msk_status msk_surrogate_decode(msk_surrogate* s, const float* C_dev, int64_t N, float* U_dev,
                                           void* stream) {
  if (!s) return MSK_ERR_ARG;
  msk_status st = check_pod(s);
  if (st != MSK_OK) return st;
  if (N < 0) return sfail(s, MSK_ERR_ARG, "N < 0");
  if (N == 0) return MSK_OK;
  if (!C_dev || !U_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  if (!aligned16(U_dev)) return sfail(s, MSK_ERR_ARG, "U_dev must be 16-byte aligned");
  st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st != MSK_OK) return st;
  return decode(s, C_dev, N, U_dev, (cudaStream_t)stream);
}

extern "C" msk_status msk_surrogate_forward(msk_surrogate* s, const uint16_t* X_dev, int64_t B, float* C_dev,
                                            void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (B < 0) return sfail(s, MSK_ERR_ARG, "B < 0");
  if (B == 0) return MSK_OK;
  if (!X_dev || !C_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  msk_status st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  const bf16* X = reinterpret_cast<const bf16*>(X_dev);
  for (int64_t o = 0; o < B && st == MSK_OK; o += s->cfg.infer_batch) {
    const int64_t P = std::min<int64_t>(s->cfg.infer_batch, B - o);
    st = forward_chain(s, X + o * s->in_dim, P, false, C_dev + o * s->cfg.rank, (cudaStream_t)stream);
  }
  return st;
}

extern "C" msk_status msk_surrogate_loss_grads(msk_surrogate* s, const uint16_t* X_dev, const float* C_dev, int64_t B,
                                               float* loss_dev, float* grads_dev, void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (B < 1 || B > s->cfg.train_batch) return sfail(s, MSK_ERR_ARG, "B must be in 1..train_batch");
  if (!X_dev || !C_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  cudaStream_t stm = (cudaStream_t)stream;
  msk_status st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st == MSK_OK) st = loss_grads(s, reinterpret_cast<const bf16*>(X_dev), C_dev, B, stm);
  if (st == MSK_OK && loss_dev)
    st = scuda(s, cudaMemcpyAsync(loss_dev, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, stm), "copy");
  if (st == MSK_OK && grads_dev)
    st = scuda(s, cudaMemcpyAsync(grads_dev, s->grad, s->nparam * sizeof(float), cudaMemcpyDeviceToDevice, stm),
               "copy");
  return st;
}

extern "C" msk_status msk_surrogate_adam_step(msk_surrogate* s, float lr, void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (!(lr > 0) || !isfinite(lr)) return sfail(s, MSK_ERR_ARG, "lr must be positive");
  msk_status st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st != MSK_OK) return st;
  return adam(s, lr, (cudaStream_t)stream);
}

extern "C" msk_status msk_surrogate_train(msk_surrogate* s, const uint16_t* X_dev, const float* C_dev, int64_t N,
                                          int epochs, float lr, float* loss_hist_dev, void* stream) {
  if (!s) return MSK_ERR_ARG;
  if (N < 1 || epochs < 0) return sfail(s, MSK_ERR_ARG, "N must be >= 1 and epochs >= 0");
  if (!X_dev || !C_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  if (!(lr > 0) || !isfinite(lr)) return sfail(s, MSK_ERR_ARG, "lr must be positive");
  cudaStream_t stm = (cudaStream_t)stream;
  msk_status st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  const bf16* X = reinterpret_cast<const bf16*>(X_dev);
  const int64_t TB = s->cfg.train_batch, nb = (N + TB - 1) / TB;
  for (int e = 0; e < epochs && st == MSK_OK; ++e)
    for (int64_t b = 0; b < nb && st == MSK_OK; ++b) {
      const int64_t o = b * TB, B = std::min(TB, N - o);
      st = loss_grads(s, X + o * s->in_dim, C_dev + o * s->cfg.rank, B, stm);
      if (st == MSK_OK) st = adam(s, lr, stm);
      if (st == MSK_OK && loss_hist_dev)
        st = scuda(s, cudaMemcpyAsync(loss_hist_dev + e * nb + b, s->loss, sizeof(float), cudaMemcpyDeviceToDevice,
                                      stm), "copy");
    }
  return st;
}

extern "C" msk_status msk_surrogate_infer(msk_surrogate* s, int64_t path0, int64_t paths, float* U_dev,
                                          uint32_t* flags_dev, int64_t audit_every, double tol,
                                          double max_fail_frac, double* report_host, void* stream) {
  if (!s) return MSK_ERR_ARG;
  msk_status st = check_pod(s);
  if (st != MSK_OK) return st;
  if (path0 < 0 || paths < 0 || audit_every < 0) return sfail(s, MSK_ERR_ARG, "negative argument");
  if (audit_every > 0 && (!(tol >= 0) || !(max_fail_frac >= 0)))
    return sfail(s, MSK_ERR_ARG, "tol and max_fail_frac must be >= 0");
  if (report_host)
    for (int i = 0; i < 5; ++i) report_host[i] = 0.0;
  if (paths == 0) return MSK_OK;
  if (!U_dev) return sfail(s, MSK_ERR_ARG, "null buffer");
  if (!aligned16(U_dev)) return sfail(s, MSK_ERR_ARG, "U_dev must be 16-byte aligned");
  st = check_fine(s);
  if (st != MSK_OK) return st;
  cudaStream_t stm = (cudaStream_t)stream;
  st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st == MSK_OK && flags_dev)
    st = scuda(s, cudaMemsetAsync(flags_dev, 0, paths * sizeof(uint32_t), stm), "flags reset");
  const uint64_t first = s->ctx->path_offset + (uint64_t)path0;
  const int64_t IB = s->cfg.infer_batch;
  int64_t na_total = 0;
  if (audit_every > 0)
    for (int64_t o = 0; o < paths; o += IB) na_total += (std::min(IB, paths - o) + audit_every - 1) / audit_every;
  if (st == MSK_OK && na_total > 0) st = sgrow(s, &s->aerr, &s->aerr_bytes, na_total * sizeof(double), "audit errors");
  int64_t na_done = 0;
  for (int64_t o = 0; o < paths && st == MSK_OK; o += IB) {
    const int64_t P = std::min(IB, paths - o);
    float* U = U_dev + (size_t)o * s->n;
    st = features(s, first + (uint64_t)o, P, s->iX, stm);
    if (st == MSK_OK) st = forward_chain(s, s->iX, P, false, s->iout, stm);
    if (st == MSK_OK) st = decode(s, s->iout, P, U, stm);
    if (st != MSK_OK || audit_every == 0) continue;
    const int64_t na = (P + audit_every - 1) / audit_every;
    st = sgrow(s, &s->uref, &s->uref_bytes, (size_t)na * s->n * sizeof(float), "audit solutions");
    if (st == MSK_OK) st = reference_solve(s, first + (uint64_t)o, (uint64_t)audit_every, na, s->uref, stm);
    if (st == MSK_OK) {
      audit_kernel<<<(unsigned)na, 256, 0, stm>>>(U, s->uref, na, audit_every, s->n, tol, s->aerr + na_done,
                                                  flags_dev ? flags_dev + o : nullptr);
      st = scuda(s, cudaGetLastError(), "audit kernel");
    }
    na_done += na;
  }
  if (st != MSK_OK || audit_every == 0) return st;
  std::vector<double> e(na_total);
  st = scuda(s, cudaMemcpyAsync(e.data(), s->aerr, na_total * sizeof(double), cudaMemcpyDeviceToHost, stm), "copy");
  if (st == MSK_OK) st = scuda(s, cudaStreamSynchronize(stm), "audit sync");
  if (st != MSK_OK) return st;
  double mx = 0, sum = 0;
  int64_t fails = 0;
  for (double v : e) {
    mx = std::max(mx, v);
    sum += v;
    if (!(v <= tol)) ++fails;
  }
  const bool whole = (double)fails > max_fail_frac * (double)na_total;
  if (whole) {
    st = reference_solve(s, first, 1, paths, U_dev, stm);
    if (st == MSK_OK && flags_dev) {
      or_flags_kernel<<<blocks_for(paths), 256, 0, stm>>>(flags_dev, paths, 4u);
      st = scuda(s, cudaGetLastError(), "flags");
    }
  }
  if (report_host) {
    report_host[0] = (double)na_total;
    report_host[1] = mx;
    report_host[2] = sum / (double)na_total;
    report_host[3] = (double)fails;
    report_host[4] = whole ? 1.0 : 0.0;
  }
  return st;
}

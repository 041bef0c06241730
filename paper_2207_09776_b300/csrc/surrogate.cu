// Learned surrogate of the Magnus solver: per-path Brownian features ->
// BF16 MLP -> POD coefficients -> u_T, trained on Magnus solutions by the
// library's own forward/backward kernels, served with a Magnus audit and
// fallback.  C ABI in include/msk.h (msk_surrogate_*).
#include <math.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <tuple>
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
  int ldk = 0;                      // 3r rounded up to a multiple of 8
  bf16* basis = nullptr;            // split decode basis [n][ldk] = [phi_hi | phi_lo | phi_hi]
  // parameters and Adam state (flat, fp32 master + bf16 copy)
  float* w = nullptr;
  bf16* w16 = nullptr;
  float* grad = nullptr;
  float* am = nullptr;
  float* av = nullptr;
  int64_t t = 0;
  bf16* w16T = nullptr;              // per layer W_l^T [in][out] (bf16), same offsets as w
  // training activations [train_batch][.] and their transposes [.][ldT]
  int ldT = 0;                        // train_batch rounded up to a multiple of 8
  std::vector<float*> z;
  std::vector<bf16*> h;
  std::vector<bf16*> hT;
  bf16* XT = nullptr;
  float* out = nullptr;
  float* g = nullptr;
  bf16* g16 = nullptr;
  bf16* g16T = nullptr;
  float* dz[2] = {nullptr, nullptr};
  bf16* dz16[2] = {nullptr, nullptr};
  bf16* dz16T[2] = {nullptr, nullptr};
  float* ws = nullptr;              // split-K workspace
  int64_t ws_elems = 0;
  double* partial = nullptr;        // loss partial sums
  float* loss = nullptr;
  // inference [infer_batch][.]
  bf16* iX = nullptr;
  bf16* ih[2] = {nullptr, nullptr};
  bf16* iA = nullptr;               // split coefficients [infer_batch][ldk] = [c_hi | c_hi | c_lo]
  // reference solves and audit (grown on demand)
  void* rs = nullptr;
  size_t rs_bytes = 0;
  float* uref = nullptr;
  size_t uref_bytes = 0;
  double* aerr = nullptr;
  size_t aerr_bytes = 0;
  uint32_t* dev_err = nullptr;        // set by kernels whose bounded waits ran out
  int wait_test = 0;                  // msk_surrogate_set_wait_test
  cudaStream_t aud = nullptr;         // audit stream (higher priority), overlaps the serve kernels
  cudaEvent_t ev_in = nullptr, ev_aud = nullptr;
  std::map<std::tuple<uintptr_t, int, int, int, int>, CUtensorMap> maps;   // TMA descriptors
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// TMA descriptor of a row-major matrix [rows][cols] (row stride ld elements of
// esize bytes), box of box_rows x box_cols (box_cols * esize = 128 bytes) with
// the 128-byte swizzle; cached per shape.  bf16 operands use 64-column boxes;
// the decode's float output uses 32 x 32 boxes.
msk_status tensor_map_any(msk_surrogate* s, const void* ptr, int esize, int rows, int cols, int ld, int box_cols,
                          int box_rows, CUtensorMap* out) {
  const auto key = std::make_tuple(reinterpret_cast<uintptr_t>(ptr), rows, cols, ld * esize, box_rows);
  const auto it = s->maps.find(key);
  if (it != s->maps.end()) {
    *out = it->second;
    return MSK_OK;
  }
  if (!aligned16(ptr) || ((int64_t)ld * esize) % 16 != 0 || ld < cols)
    return sfail(s, MSK_ERR_UNSUPPORTED, "GEMM operand must be 16-byte aligned with a 16-byte multiple row stride");
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return sfail(s, MSK_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUtensorMap m;
  const CUresult r = fn(&m, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return sfail(s, MSK_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  if (s->maps.size() > 4096) s->maps.clear();
  s->maps.emplace(key, m);
  *out = m;
  return MSK_OK;
}

msk_status tensor_map(msk_surrogate* s, const bf16* ptr, int rows, int cols, int ld, int box_rows, CUtensorMap* out) {
  return tensor_map_any(s, ptr, (int)sizeof(bf16), rows, cols, ld, TC_BK, box_rows, out);
}

struct TcOut {
  float* C = nullptr;
  int ldc = 0;
  bf16* C16 = nullptr;
  int ldc16 = 0;
  bf16* CT = nullptr;
  int ldct = 0;
  const float* bias = nullptr;
  const float* aux = nullptr;
  int ldaux = 0;
};

constexpr int kStages = 4;        // pipeline depth of the MLP GEMMs
constexpr int kDecodeStages = 3;  // decode: K = 3r <= 192 is three k-blocks per tile

// Persistent launch: as many CTAs as fit (at most one per tile).
template <int BN, int EPI, int ST>
cudaError_t launch_tc(msk_surrogate* s, const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc,
                      const TcArgs& g, int tiles_m, int tiles_n, int splits, cudaStream_t stream) {
  auto kern = gemm_tc_kernel<BN, EPI, ST>;
  const size_t smem = tc_smem_bytes(BN, ST, EPI);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TC_THREADS, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (int64_t)tiles_m * tiles_n * splits;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)std::max(per_sm, 1) * s->ctx->num_sms));
  kern<<<grid, TC_THREADS, smem, stream>>>(ta, tb, tc, g, tiles_m, tiles_n, splits);
  return cudaGetLastError();
}

template <int BN, int EPI, int ST>
cudaError_t tc_attribute() {
  return cudaFuncSetAttribute(gemm_tc_kernel<BN, EPI, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes(BN, ST, EPI));
}

template <int BN>
cudaError_t tc_attributes() {
  cudaError_t e = tc_attribute<BN, EPI_F32, kStages>();
  if (e == cudaSuccess) e = tc_attribute<BN, EPI_BIAS_F32, kStages>();
  if (e == cudaSuccess) e = tc_attribute<BN, EPI_BIAS_GELU, kStages>();
  if (e == cudaSuccess) e = tc_attribute<BN, EPI_GELU_BWD, kStages>();
  if (e == cudaSuccess) e = tc_attribute<BN, EPI_BIAS_SPLIT, kStages>();
  if (e == cudaSuccess) e = tc_attribute<BN, EPI_ADD_MEAN, kDecodeStages>();
  return e;
}

// C = A B^T with A [M][K] (row stride lda) and B [N][K] (row stride ldb), both
// bf16 K-major, on the tcgen05 kernel.  The tile width is the widest of 256,
// 128, 64 whose grid still covers the SMs; split (EPI_F32 only) spreads K over
// blockIdx.z into the workspace and reduces in a fixed order into C [M][N].
template <int EPI>
msk_status gemm(msk_surrogate* s, const bf16* A, int lda, int M, const bf16* B, int ldb, int N, int K, const TcOut& o,
                bool split, cudaStream_t stream) {
  if (M == 0 || N == 0) return MSK_OK;
  if (K < 1) return sfail(s, MSK_ERR_ARG, "GEMM with K = 0");
  const int sms = std::max(1, s->ctx->num_sms);
  const int bm = (M + TC_BM - 1) / TC_BM;
  int BN = N > 128 ? 256 : (N > 64 ? 128 : 64);
  while (BN > 64 && (int64_t)bm * ((N + BN - 1) / BN) < sms) BN /= 2;
  const int bn = (N + BN - 1) / BN;
  const auto rup = [](int64_t x, int64_t m) { return (x + m - 1) / m * m; };
  int splits = 1, kchunk = (int)rup(K, TC_BK);
  if (split && EPI == EPI_F32) {
    const int64_t tiles = (int64_t)bm * bn;
    splits = (int)std::min<int64_t>(std::max<int64_t>(1, (sms + tiles - 1) / tiles), std::max(1, K / 256));
    kchunk = (int)rup((K + splits - 1) / splits, TC_BK);
    splits = (K + kchunk - 1) / kchunk;
    if (splits > 1 && (int64_t)splits * M * N > s->ws_elems) {   // workspace too small: no split
      splits = 1;
      kchunk = (int)rup(K, TC_BK);
    }
  }
  CUtensorMap ta, tb, tc;
  msk_status st = tensor_map(s, A, M, K, lda, TC_BM, &ta);
  if (st == MSK_OK) st = tensor_map(s, B, N, K, ldb, BN, &tb);
  if (st == MSK_OK) {
    if (EPI == EPI_ADD_MEAN) {   // float output written by 32 x 32 TMA stores
      if (N % 32 != 0) return sfail(s, MSK_ERR_UNSUPPORTED, "decode width must be a multiple of 32");
      st = tensor_map_any(s, o.C, (int)sizeof(float), M, N, o.ldc, 32, 32, &tc);
    } else {
      tc = ta;   // unused
    }
  }
  if (st != MSK_OK) return st;
  TcArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.kchunk = kchunk;
  g.C = o.C;
  g.ldc = o.ldc;
  g.C16 = o.C16;
  g.ldc16 = o.ldc16;
  g.CT = o.CT;
  g.ldct = o.ldct;
  g.bias = o.bias;
  g.aux = o.aux;
  g.ldaux = o.ldaux;
  g.err = s->dev_err;
  g.wait_test = s->wait_test;
  if (splits > 1) {
    g.C = s->ws;
    g.ldc = N;
    g.split_stride = (int64_t)M * N;
  }
  constexpr int ST = EPI == EPI_ADD_MEAN ? kDecodeStages : kStages;
  cudaError_t e;
  if (BN == 256) e = launch_tc<256, EPI, ST>(s, ta, tb, tc, g, bm, bn, splits, stream);
  else if (BN == 128) e = launch_tc<128, EPI, ST>(s, ta, tb, tc, g, bm, bn, splits, stream);
  else e = launch_tc<64, EPI, ST>(s, ta, tb, tc, g, bm, bn, splits, stream);
  st = scuda(s, e, "tensor-core GEMM");
  if (st != MSK_OK || splits == 1) return st;
  reduce_splits_kernel<<<blocks_for((int64_t)M * N), 256, 0, stream>>>(s->ws, splits, (int64_t)M * N, o.C);
  return scuda(s, cudaGetLastError(), "split-K reduction");
}

// W_l^T [in][out] (bf16) of every layer, the B operand of the data gradients.
msk_status refresh_transposed_weights(msk_surrogate* s, cudaStream_t stream) {
  for (int l = 0; l < s->L; ++l) {
    const int out = s->dims[l + 1], in = s->dims[l];
    transpose_bf16_kernel<<<dim3(blocks_for(in, 32), blocks_for(out, 32)), dim3(32, 8), 0, stream>>>(
        s->w16 + s->offW[l], out, in, in, s->w16T + s->offW[l], out);
  }
  return scuda(s, cudaGetLastError(), "weight transpose");
}

// Forward pass of B rows of X.  train: keeps z_l, h_l and h_l^T of every
// hidden layer; otherwise ping-pongs the inference buffers.  Output: out [B][r] (fp32).
msk_status forward_chain(msk_surrogate* s, const bf16* X, int64_t B, bool train, float* out, cudaStream_t stream,
                         bf16* split_out = nullptr) {
  const bf16* hin = X;
  int in = s->in_dim;
  const int H = s->cfg.hidden;
  for (int l = 0; l < s->L - 1; ++l) {
    TcOut o;
    o.bias = s->w + s->offB[l];
    if (train) {
      o.C = s->z[l];
      o.ldc = H;
      o.C16 = s->h[l];
      o.ldc16 = H;
      o.CT = s->hT[l];
      o.ldct = s->ldT;
    } else {
      o.C16 = s->ih[l & 1];
      o.ldc16 = H;
    }
    msk_status st = gemm<EPI_BIAS_GELU>(s, hin, in, (int)B, s->w16 + s->offW[l], in, H, in, o, false, stream);
    if (st != MSK_OK) return st;
    hin = o.C16;
    in = H;
  }
  const int l = s->L - 1, r = s->cfg.rank;
  TcOut o;
  o.C = out;
  o.ldc = r;
  o.bias = s->w + s->offB[l];
  if (split_out) {   // also write the split coefficients for the tensor-core decode
    o.C16 = split_out;
    o.ldc16 = s->ldk;
    return gemm<EPI_BIAS_SPLIT>(s, hin, in, (int)B, s->w16 + s->offW[l], in, r, in, o, false, stream);
  }
  return gemm<EPI_BIAS_F32>(s, hin, in, (int)B, s->w16 + s->offW[l], in, r, in, o, false, stream);
}

// Loss and gradients of one minibatch (B <= train_batch) into s->grad and s->loss.
// Every GEMM is K-major x K-major: weight gradients contract over the batch
// with the transposed copies dz^T and h^T written by the producing epilogues,
// data gradients use the transposed weights W^T.
msk_status loss_grads(msk_surrogate* s, const bf16* X, const float* C, int64_t B, cudaStream_t stream) {
  msk_status st = forward_chain(s, X, B, true, s->out, stream);
  if (st != MSK_OK) return st;
  const int r = s->cfg.rank, H = s->cfg.hidden, L = s->L, ldT = s->ldT;
  transpose_bf16_kernel<<<dim3(blocks_for(s->in_dim, 32), blocks_for(B, 32)), dim3(32, 8), 0, stream>>>(
      X, (int)B, s->in_dim, s->in_dim, s->XT, ldT);
  loss_grad_kernel<<<kLossBlocks, 256, 0, stream>>>(s->out, C, B * r, r, 1.0f / (float)B, s->g, s->g16, s->g16T, ldT,
                                                    s->partial);
  loss_final_kernel<<<1, 256, 0, stream>>>(s->partial, kLossBlocks, 1.0 / (double)B, s->loss);
  st = scuda(s, cudaGetLastError(), "loss kernels");
  if (st != MSK_OK) return st;
  const bf16* cur16 = s->g16;
  const bf16* cur16T = s->g16T;
  const float* cur = s->g;
  int cur_dim = r;
  for (int l = L - 1; l >= 0; --l) {
    const int in = s->dims[l];
    const bf16* prevT = l > 0 ? s->hT[l - 1] : s->XT;
    // dW_l [out][in] = dz_l^T h_{l-1}: A = dz_l^T [out][B], B = h_{l-1}^T [in][B]
    TcOut ow;
    ow.C = s->grad + s->offW[l];
    ow.ldc = in;
    st = gemm<EPI_F32>(s, cur16T, ldT, cur_dim, prevT, ldT, in, (int)B, ow, true, stream);
    if (st != MSK_OK) return st;
    colsum_kernel<<<blocks_for(cur_dim, 32), dim3(32, 8), 0, stream>>>(cur, (int)B, cur_dim, s->grad + s->offB[l]);
    st = scuda(s, cudaGetLastError(), "bias gradient");
    if (st != MSK_OK) return st;
    if (l == 0) break;
    // dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1}): A = dz_l [B][out], B = W_l^T [in][out]
    TcOut od;
    od.C = s->dz[l & 1];
    od.ldc = H;
    od.C16 = s->dz16[l & 1];
    od.ldc16 = H;
    od.CT = s->dz16T[l & 1];
    od.ldct = ldT;
    od.aux = s->z[l - 1];
    od.ldaux = H;
    st = gemm<EPI_GELU_BWD>(s, cur16, cur_dim, (int)B, s->w16T + s->offW[l], cur_dim, in, cur_dim, od, false, stream);
    if (st != MSK_OK) return st;
    cur = od.C;
    cur16 = od.C16;
    cur16T = od.CT;
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
  msk_status st = scuda(s, cudaGetLastError(), "adam kernel");
  return st == MSK_OK ? refresh_transposed_weights(s, stream) : st;
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
    msk_status st = sgrow(s, &s->rs, &s->rs_bytes, (nF + nW + (size_t)P + 1) * sizeof(double), "reference scratch");
    if (st != MSK_OK) return st;
    double* F = reinterpret_cast<double*>(s->rs);
    double* Wt = F + nF;
    long long* order_buf = reinterpret_cast<long long*>(Wt + nW);
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(order_buf + P);
    st = from_ctx(s, launch_brownian_strided(ctx, steps, P, F, first + (uint64_t)o * stride, stride, stream, true));
    if (st == MSK_OK) st = from_ctx(s, launch_omega(ctx, order, steps, P, MSK_F32, F, Wt, stream));
    if (st == MSK_OK)
      st = from_ctx(s, launch_magnus_queued(ctx, steps, P, MSK_F32, Wt, U + (size_t)o * s->n, nullptr, stream,
                                            order_buf, queue));
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

// U [P][n] = mean + c Phi as one tensor-core contraction over K = 3r of the
// split coefficients A' (already in s->iA, P <= infer_batch) with the split basis.
msk_status decode_split(msk_surrogate* s, int64_t P, float* U, cudaStream_t stream) {
  TcOut o;
  o.C = U;
  o.ldc = s->n;
  o.bias = s->mean;
  return gemm<EPI_ADD_MEAN>(s, s->iA, s->ldk, (int)P, s->basis, s->ldk, s->n, 3 * s->cfg.rank, o, false, stream);
}

msk_status decode(msk_surrogate* s, const float* C, int64_t P, float* U, cudaStream_t stream) {
  const int r = s->cfg.rank;
  for (int64_t o = 0; o < P; o += s->cfg.infer_batch) {
    const int64_t Pc = std::min<int64_t>(s->cfg.infer_batch, P - o);
    split_coef_kernel<<<blocks_for(Pc * r), 256, 0, stream>>>(C + o * r, Pc, r, s->iA, s->ldk);
    msk_status st = scuda(s, cudaGetLastError(), "coefficient split");
    if (st == MSK_OK) st = decode_split(s, Pc, U + (size_t)o * s->n, stream);
    if (st != MSK_OK) return st;
  }
  return MSK_OK;
}

msk_status refresh_basis(msk_surrogate* s, cudaStream_t stream) {
  const int64_t cnt = (int64_t)s->cfg.rank * s->n;
  split_basis_kernel<<<blocks_for(cnt), 256, 0, stream>>>(s->phi, s->cfg.rank, s->n, s->basis, s->ldk);
  return scuda(s, cudaGetLastError(), "decode basis");
}

void free_all(msk_surrogate* s) {
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  F(s->mean);
  F(s->phi);
  F(s->w);
  F(s->w16);
  F(s->w16T);
  F(s->grad);
  F(s->am);
  F(s->av);
  for (float* p : s->z) F(p);
  for (bf16* p : s->h) F(p);
  for (bf16* p : s->hT) F(p);
  F(s->XT);
  F(s->out);
  F(s->g);
  F(s->g16);
  F(s->g16T);
  for (int i = 0; i < 2; ++i) {
    F(s->dz[i]);
    F(s->dz16[i]);
    F(s->dz16T[i]);
    F(s->ih[i]);
  }
  F(s->dev_err);
  if (s->ev_in) cudaEventDestroy(s->ev_in);
  if (s->ev_aud) cudaEventDestroy(s->ev_aud);
  if (s->aud) cudaStreamDestroy(s->aud);
  F(s->ws);
  F(s->partial);
  F(s->loss);
  F(s->iX);
  F(s->iA);
  F(s->basis);
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
  if (st == MSK_OK) st = salloc(s, &s->w16T, s->nparam, "transposed bf16 weights");
  if (st == MSK_OK) st = salloc(s, &s->dev_err, 1, "error word");
  if (st == MSK_OK) {
    int lo = 0, hi = 0;
    st = scuda(s, cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
    if (st == MSK_OK) st = scuda(s, cudaStreamCreateWithPriority(&s->aud, cudaStreamNonBlocking, hi), "audit stream");
  }
  if (st == MSK_OK) st = scuda(s, cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming), "event");
  if (st == MSK_OK) st = scuda(s, cudaEventCreateWithFlags(&s->ev_aud, cudaEventDisableTiming), "event");
  if (st == MSK_OK) st = scuda(s, cudaMemset(s->dev_err, 0, sizeof(uint32_t)), "error word");
  if (st == MSK_OK) st = salloc(s, &s->grad, s->nparam, "gradients");
  if (st == MSK_OK) st = salloc(s, &s->am, s->nparam, "Adam m");
  if (st == MSK_OK) st = salloc(s, &s->av, s->nparam, "Adam v");
  s->ldT = (int)((TB + 7) / 8 * 8);
  const int64_t LT = s->ldT;
  s->z.assign(c.layers, nullptr);
  s->h.assign(c.layers, nullptr);
  s->hT.assign(c.layers, nullptr);
  for (int l = 0; l < c.layers && st == MSK_OK; ++l) {
    st = salloc(s, &s->z[l], (size_t)TB * H, "activations");
    if (st == MSK_OK) st = salloc(s, &s->h[l], (size_t)TB * H, "activations");
    if (st == MSK_OK) st = salloc(s, &s->hT[l], (size_t)H * LT, "activations");
  }
  if (st == MSK_OK) st = salloc(s, &s->XT, (size_t)s->in_dim * LT, "transposed features");
  if (st == MSK_OK) st = salloc(s, &s->out, (size_t)TB * r, "outputs");
  if (st == MSK_OK) st = salloc(s, &s->g, (size_t)TB * r, "output gradient");
  if (st == MSK_OK) st = salloc(s, &s->g16, (size_t)TB * r, "output gradient");
  if (st == MSK_OK) st = salloc(s, &s->g16T, (size_t)r * LT, "output gradient");
  for (int i = 0; i < 2 && st == MSK_OK; ++i) {
    st = salloc(s, &s->dz[i], (size_t)TB * H, "backward buffers");
    if (st == MSK_OK) st = salloc(s, &s->dz16[i], (size_t)TB * H, "backward buffers");
    if (st == MSK_OK) st = salloc(s, &s->dz16T[i], (size_t)H * LT, "backward buffers");
    if (st == MSK_OK) st = salloc(s, &s->ih[i], (size_t)IB * H, "inference buffers");
  }
  // split-K workspace: up to 2 * SMs splits of the largest weight gradient
  s->ws_elems = (int64_t)2 * std::max(ctx->num_sms, 1) * std::max<int64_t>(H * H, H * std::max<int64_t>(r, s->in_dim));
  s->ws_elems = std::min<int64_t>(s->ws_elems, (int64_t)16 * H * H + 1);
  if (st == MSK_OK) st = salloc(s, &s->ws, s->ws_elems, "split-K workspace");
  if (st == MSK_OK) st = salloc(s, &s->partial, kLossBlocks, "loss partials");
  if (st == MSK_OK) st = salloc(s, &s->loss, 1, "loss");
  if (st == MSK_OK) st = salloc(s, &s->iX, (size_t)IB * s->in_dim, "inference features");
  s->ldk = (int)((3 * r + 7) / 8 * 8);
  if (st == MSK_OK) st = salloc(s, &s->iA, (size_t)IB * s->ldk, "split coefficients");
  if (st == MSK_OK) st = salloc(s, &s->basis, (size_t)s->n * s->ldk, "decode basis");
  if (st == MSK_OK) st = scuda(s, cudaMemset(s->iA, 0, (size_t)IB * s->ldk * sizeof(bf16)), "split coefficients");
  if (st == MSK_OK) st = scuda(s, cudaMemset(s->basis, 0, (size_t)s->n * s->ldk * sizeof(bf16)), "decode basis");
  if (st == MSK_OK) st = scuda(s, tc_attributes<64>(), "GEMM attributes");
  if (st == MSK_OK) st = scuda(s, tc_attributes<128>(), "GEMM attributes");
  if (st == MSK_OK) st = scuda(s, tc_attributes<256>(), "GEMM attributes");
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
  if (st == MSK_OK) st = refresh_transposed_weights(s, 0);
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
  if (st == MSK_OK) st = refresh_transposed_weights(s, st_);
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
    if (st == MSK_OK) st = refresh_basis(s, stm);
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
  if (st == MSK_OK) st = refresh_basis(s, stm);
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
  if (st == MSK_OK && na_total > 0)
    st = sgrow(s, &s->uref, &s->uref_bytes, (size_t)na_total * s->n * sizeof(float), "audit solutions");
  // The audit's Magnus solves depend only on the paths: they run on the audit
  // stream (ordered after the caller's earlier work) while the serve kernels run
  // on the caller's stream; the audit kernels join both.
  if (st == MSK_OK && na_total > 0) {
    st = scuda(s, cudaEventRecord(s->ev_in, stm), "event");
    if (st == MSK_OK) st = scuda(s, cudaStreamWaitEvent(s->aud, s->ev_in, 0), "event");
    int64_t na_off = 0;
    for (int64_t o = 0; o < paths && st == MSK_OK; o += IB) {
      const int64_t na = (std::min(IB, paths - o) + audit_every - 1) / audit_every;
      st = reference_solve(s, first + (uint64_t)o, (uint64_t)audit_every, na, s->uref + (size_t)na_off * s->n, s->aud);
      na_off += na;
    }
    if (st == MSK_OK) st = scuda(s, cudaEventRecord(s->ev_aud, s->aud), "event");
  }
  for (int64_t o = 0; o < paths && st == MSK_OK; o += IB) {
    const int64_t P = std::min(IB, paths - o);
    float* U = U_dev + (size_t)o * s->n;
    st = features(s, first + (uint64_t)o, P, s->iX, stm);
    if (st == MSK_OK) st = forward_chain(s, s->iX, P, false, nullptr, stm, s->iA);
    if (st == MSK_OK) st = decode_split(s, P, U, stm);
  }
  if (st != MSK_OK || audit_every == 0) return st;
  st = scuda(s, cudaStreamWaitEvent(stm, s->ev_aud, 0), "event");
  int64_t na_done = 0;
  for (int64_t o = 0; o < paths && st == MSK_OK; o += IB) {
    const int64_t P = std::min(IB, paths - o);
    const int64_t na = (P + audit_every - 1) / audit_every;
    audit_kernel<<<(unsigned)na, 256, 0, stm>>>(U_dev + (size_t)o * s->n, s->uref + (size_t)na_done * s->n, na,
                                                audit_every, s->n, tol, s->aerr + na_done,
                                                flags_dev ? flags_dev + o : nullptr);
    st = scuda(s, cudaGetLastError(), "audit kernel");
    na_done += na;
  }
  if (st != MSK_OK) return st;
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

extern "C" msk_status msk_surrogate_set_wait_test(msk_surrogate* s, int on) {
  if (!s) return MSK_ERR_ARG;
  s->wait_test = on ? 1 : 0;
  return MSK_OK;
}

extern "C" msk_status msk_surrogate_sync_status(msk_surrogate* s, void* stream) {
  if (!s) return MSK_ERR_ARG;
  uint32_t e = 0;
  msk_status st = scuda(s, cudaSetDevice(s->ctx->device), "set device");
  if (st == MSK_OK)
    st = scuda(s, cudaMemcpyAsync(&e, s->dev_err, sizeof(e), cudaMemcpyDeviceToHost, (cudaStream_t)stream), "copy");
  if (st == MSK_OK) st = scuda(s, cudaStreamSynchronize((cudaStream_t)stream), "sync");
  if (st == MSK_OK && e) st = sfail(s, MSK_ERR_TIMEOUT, "a tensor-core pipeline wait ran out");
  return st;
}

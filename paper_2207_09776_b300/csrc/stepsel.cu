// Step-size control by the distance of the order-2 and order-3 Magnus results
// (Remark stepSizeControl): both orders come from the same Brownian functionals
// (the order-3 logarithm contains the order-2 one), so a step count K is
// accepted when the two solutions of a set of trajectories agree to a tolerance.
#include <math.h>

#include <algorithm>
#include <vector>

#include "msk_internal.cuh"

extern "C" msk_status msk_select_steps(msk_ctx* ctx, double tol, int k_min, int k_max, int64_t paths, int precision,
                                       int* K_out, double* dist_host, int* n_tried, void* stream) {
  if (!ctx) return MSK_ERR_ARG;
  if (!K_out) return msk_fail(ctx, MSK_ERR_ARG, "null K_out");
  if (!(tol > 0)) return msk_fail(ctx, MSK_ERR_ARG, "tol must be positive");
  if (precision != MSK_F64 && precision != MSK_F32) return msk_fail(ctx, MSK_ERR_ARG, "bad precision");
  if (paths < 1) return msk_fail(ctx, MSK_ERR_ARG, "paths must be >= 1");
  if (k_min < 1 || k_max < k_min) return msk_fail(ctx, MSK_ERR_ARG, "need 1 <= k_min <= k_max");
  std::vector<int> ks;
  for (int64_t k = k_min; k <= k_max && ks.size() < 16; k *= 2)
    if (ctx->n_fine % k == 0) ks.push_back((int)k);
  if (ks.empty()) return msk_fail(ctx, MSK_ERR_ARG, "no candidate step count divides n_fine");
  cudaStream_t s = (cudaStream_t)stream;
  msk_status st = msk_cuda(ctx, cudaSetDevice(ctx->device), "set device");
  if (st != MSK_OK) return st;
  const size_t es = precision == MSK_F64 ? sizeof(double) : sizeof(float);
  const size_t nU = (size_t)paths * ctx->d * ctx->d;
  const int kmax = ks.back();
  const size_t nF = (size_t)paths * kmax * MSK_NF, nW = (size_t)paths * kmax * MSK_NWT;
  // scratch of this call: functionals, two weight sets, two solutions, per-path distances
  void* buf = nullptr;
  const size_t bytes = (nF + 2 * nW + paths) * sizeof(double) + 2 * nU * es + 256;
  st = msk_cuda(ctx, cudaMalloc(&buf, bytes), "step-selection scratch");
  if (st != MSK_OK) return st;
  double* F = reinterpret_cast<double*>(buf);
  double* W2 = F + nF;
  double* W3 = W2 + nW;
  double* dist = W3 + nW;
  char* u2 = reinterpret_cast<char*>(dist + paths);
  u2 += (256 - reinterpret_cast<uintptr_t>(u2) % 256) % 256;
  char* u3 = u2 + nU * es;
  const bool nf32 = precision == MSK_F32;
  std::vector<double> d(paths);
  int chosen = -1, tried = 0;
  for (int K : ks) {
    st = launch_brownian(ctx, K, paths, F, false, s, nf32);
    if (st == MSK_OK) st = launch_omega(ctx, 2, K, paths, precision, F, W2, s);
    if (st == MSK_OK) st = launch_omega(ctx, 3, K, paths, precision, F, W3, s);
    if (st == MSK_OK) st = launch_engine(ctx, false, K, paths, precision, W2, nullptr, u2, nullptr, s);
    if (st == MSK_OK) st = launch_engine(ctx, false, K, paths, precision, W3, nullptr, u3, nullptr, s);
    if (st == MSK_OK)
      st = msk_error(ctx, u2, precision, paths, MSK_REF_BUFFER, u3, precision, 0, dist, nullptr, stream);
    if (st == MSK_OK)
      st = msk_cuda(ctx, cudaMemcpyAsync(d.data(), dist, paths * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    if (st == MSK_OK) st = msk_cuda(ctx, cudaStreamSynchronize(s), "step-selection sync");
    if (st != MSK_OK) break;
    double dk = 0.0;
    for (double v : d) dk = (v == v) ? std::max(dk, v) : INFINITY;   // NaN (blow-up) rejects the step
    if (dist_host) dist_host[tried] = dk;
    ++tried;
    if (dk <= tol) {
      chosen = K;
      break;
    }
  }
  cudaFree(buf);
  if (st != MSK_OK) return st;
  *K_out = chosen > 0 ? chosen : ks.back();
  if (n_tried) *n_tried = tried;
  return MSK_OK;
}

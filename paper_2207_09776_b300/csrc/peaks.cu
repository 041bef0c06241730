// Arithmetic throughput of this GPU's CUDA cores, the denominator of the
// roofline fraction of the ALU-bound stencil engines (whose state stays on
// chip, so HBM bandwidth does not bound them).  No counterpart in the paper.
//
// Every thread runs kChains independent multiply-add chains (enough
// instruction-level parallelism to keep the FMA pipe busy at full occupancy)
// for `iters` rounds; the grid fills every SM several times over.  The result
// depends on every chain and is stored only when it equals a value it cannot
// take, so the compiler keeps all the arithmetic.
#include "msk_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int64_t iters, T a, T b, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345e30) *sink = s;   // never true for the inputs used; keeps the chains live
}

}  // namespace

extern "C" msk_status msk_fma_throughput(int device, int precision, double* tflops_out, void* stream) {
  if (!tflops_out || (precision != MSK_F32 && precision != MSK_F64)) return MSK_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return MSK_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MSK_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)sms * 8;          // 2048 threads per SM, 8 waves of warps
  const int64_t iters = precision == MSK_F32 ? 4096 : 64;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MSK_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MSK_ERR_CUDA;
  }
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {                 // the first launch warms up
    cudaEventRecord(e0, s);
    if (precision == MSK_F32)
      fma_peak_kernel<float><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999f, 1e-7f, nullptr);
    else
      fma_peak_kernel<double><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999, 1e-7, nullptr);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || !(best < 1e30f)) return MSK_ERR_CUDA;
  const double fmas = (double)blocks * kPeakThreads * iters * 16 * kChains;
  *tflops_out = 2.0 * fmas / (best * 1e-3) / 1e12;
  return MSK_OK;
}

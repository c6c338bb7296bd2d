// Measured FMA throughput of this GPU in FP64 and FP32 (msp_fma_rate).  The FP64 block
// kernels of the solve do one FMA per 8-byte value they read, and on this part the FP64
// FMA rate, not the memory, can bound them; the benchmark measures the rate live and
// states every kernel's ceiling against it.
//
// Launch: 8 resident blocks of 256 threads per SM (a multiple of the SM count); every
// thread runs kChains independent FMA chains of kSteps steps each (x = x * a + c with
// |a| < 1, so the values stay finite and the compiler cannot fold the chain), and writes
// their sum so nothing is eliminated.  Timed with CUDA events on the caller's stream
// after one warm-up launch.
#include <cuda_runtime.h>

#include "common.cuh"

namespace msp {
namespace {

constexpr int kChains = 8;
constexpr int kSteps = 2048;
constexpr int kFmaThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kFmaThreads) fma_chains_kernel(T a, T c, T* __restrict__ out) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int s = 0; s < kSteps; ++s) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, c);
  }
  T sum = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) sum += x[k];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = sum;
}

template <typename T>
int fma_rate(double* flops_per_s, cudaStream_t s) {
  int dev = 0, sms = 0;
  MSP_CUDA_TRY(cudaGetDevice(&dev));
  MSP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;
  DevBuf<T> out;
  MSP_TRY(out.alloc((size_t)blocks * kFmaThreads));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MSP_CUDA_TRY(cudaEventCreate(&e0));
  MSP_CUDA_TRY(cudaEventCreate(&e1));
  const T a = (T)0.999, c = (T)1e-3;
  fma_chains_kernel<T><<<blocks, kFmaThreads, 0, s>>>(a, c, out.p);  // warm-up
  int st = launch_check(__FILE__, __LINE__);
  float best = 0.0f;
  for (int rep = 0; rep < 5 && st == MSP_OK; ++rep) {
    cudaEventRecord(e0, s);
    fma_chains_kernel<T><<<blocks, kFmaThreads, 0, s>>>(a, c, out.p);
    st = launch_check(__FILE__, __LINE__);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = MSP_ERR_CUDA;
    float ms = 0.0f;
    if (st == MSP_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f &&
        (best == 0.0f || ms < best))
      best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MSP_OK) return st;
  if (best <= 0.0f) return MSP_ERR_CUDA;
  const double fmas = (double)blocks * kFmaThreads * kChains * kSteps;
  *flops_per_s = 2.0 * fmas / (best * 1e-3);
  return MSP_OK;
}

}  // namespace
}  // namespace msp

extern "C" int msp_fma_rate(int precision, double* flops_per_s, void* stream) {
  if (!flops_per_s) return MSP_ERR_ARG;
  *flops_per_s = 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    if (precision == MSP_PRECISION_FP64) return msp::fma_rate<double>(flops_per_s, s);
    if (precision == MSP_PRECISION_FP32) return msp::fma_rate<float>(flops_per_s, s);
  } catch (...) {
    return MSP_ERR_NOMEM;
  }
  return MSP_ERR_ARG;
}

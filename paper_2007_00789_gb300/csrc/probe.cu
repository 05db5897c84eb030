// Measurement aid: the ALU roof of the FP64 (and FP32) kernels.
//
// GB300 publishes no FP64 rate that this library can take as a measured
// denominator, and the factorization's kernels are bound by the FP64 (or FP32)
// fused multiply-add pipe, not by HBM.  k_fma_chains runs independent FMA
// chains in every thread of a grid that fills every SM; the best of several
// timed launches (CUDA events on one stream) gives the achievable FMA rate.
#include <cuda_runtime.h>

#include <algorithm>

#include "spand.h"

namespace {

constexpr int kChains = 8;

__device__ double g_fma_sink;  // written only if a chain went negative, which it cannot

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // the chains start at >= 0 and stay positive (a, b > 0): the store never
  // happens, but the compiler must keep every chain to decide that
  if (s < (T)0) g_fma_sink = (double)s;
}

template <typename T>
int measure(double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPAND_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPAND_ECUDA;
  const int threads = 256, blocks = sms * 8;
  const int iters = sizeof(T) == 8 ? 2048 : 65536;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SPAND_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = SPAND_ECUDA;
  } else {
    float best = 1e30f;
    for (int rep = 0; rep < 6 && rc == SPAND_OK; ++rep) {
      cudaEventRecord(e0, s);
      k_fma_chains<T><<<blocks, threads, 0, s>>>(iters, (T)0.999999, (T)1e-7);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = SPAND_ECUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);  // the first launch is a warm-up
    }
    if (rc == SPAND_OK) {
      const double flops = 2.0 * kChains * (double)iters * threads * blocks;
      *tflops = flops / (best * 1e-3) / 1e12;
      if (ms_out) *ms_out = best;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (cudaGetLastError() != cudaSuccess) rc = SPAND_ECUDA;
  return rc;
}

}  // namespace

extern "C" int spand_measure_fma_peak(int precision, double* tflops, double* ms) {
  if (!tflops || (precision != 0 && precision != 1)) return SPAND_EINVAL;
  return precision == 0 ? measure<double>(tflops, ms) : measure<float>(tflops, ms);
}

// Fused multiply-add throughput of the GPU in float32 and float64 (sidp_fma_peak).
//
// The paper has no counterpart: this measures the two arithmetic ceilings against which the
// stage kernels are placed (the float32 path's FP32 pipe, the float64 path's FP64 pipe), beside
// the measured HBM bandwidth.  Every thread runs kChains independent fused multiply-add chains
// (enough independent work per warp to cover the pipe latency), every SM holds several CTAs, and
// the launch is timed with CUDA events on the caller's stream.  One FMA counts as 2 flops.
#include <string>

#include <cuda_runtime.h>

#include "sidp.h"
#include "sidp_internal.h"

namespace sidp {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

// Where a chain's result would go if it matched the sentinel (a NaN, so never): the chains stay
// live without any store in practice, and a store, if one happened, stays in bounds.
__device__ double g_peak_sink[1024];

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, T a, T b, T sentinel) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == sentinel) g_peak_sink[blockIdx.x & 1023] = (double)s;
}

template <typename T>
cudaError_t measure(int iters, double* flop_per_s, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, kPeakThreads, 0);
  if (e != cudaSuccess) return e;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  const T a = T(0.999999), b = T(1e-7), nan = T(__builtin_nan(""));
  k_fma_peak<T><<<blocks, kPeakThreads, 0, st>>>(1, a, b, nan);  // warm-up
  cudaEventRecord(e0, st);
  k_fma_peak<T><<<blocks, kPeakThreads, 0, st>>>(iters, a, b, nan);
  cudaEventRecord(e1, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double fmas = (double)blocks * kPeakThreads * (double)iters * 16.0 * kChains;
  *flop_per_s = ms > 0.f ? 2.0 * fmas / (ms * 1e-3) : 0.0;
  return cudaSuccess;
}

}  // namespace
}  // namespace sidp

extern "C" sidp_status sidp_fma_peak(int precision, double* flop_per_s, void* cuda_stream) {
  using namespace sidp;
  if (!flop_per_s || (precision != SIDP_FP64 && precision != SIDP_MIXED)) {
    set_last_error("sidp_fma_peak: null output or unknown precision");
    return SIDP_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // float32: about 40 ms at the nominal rate; float64 runs far fewer iterations (a small
  // fraction of the float32 rate on this GPU)
  const cudaError_t e = (precision == SIDP_MIXED) ? measure<float>(20000, flop_per_s, st)
                                                  : measure<double>(400, flop_per_s, st);
  if (e != cudaSuccess) {
    set_last_error(std::string("sidp_fma_peak: ") + cudaGetErrorString(e));
    return SIDP_ERR_CUDA;
  }
  return SIDP_OK;
}

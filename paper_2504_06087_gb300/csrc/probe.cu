// FMA-rate probe of the SIMT pipes (float32 and float64).
//
// The roofline fractions of the kernels that run on the FP32 or FP64 pipe
// (the restricted log-det contraction, the Gauss-Jordan inverse, the float64
// LU) are quoted against the rate this kernel measures on the device at hand,
// instead of a rate derived from unit counts and clocks.
//
// Each thread runs eight independent multiply-add chains x <- x * a + b for
// `iters` rounds (eight dependent chains hide the pipe latency at full
// occupancy); the chains are written out at the end so no round can be
// dropped.  FLOPs = 2 * 8 * iters * blocks * threads.
#include <cuda_runtime.h>

#include "../../include/fire.h"

namespace {

template <typename T>
__device__ __forceinline__ T fma_rn(T x, T a, T b);

template <>
__device__ __forceinline__ float fma_rn<float>(float x, float a, float b) {
  float y;
  asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(x), "f"(a), "f"(b));
  return y;
}

template <>
__device__ __forceinline__ double fma_rn<double>(double x, double a, double b) {
  double y;
  asm volatile("fma.rn.f64 %0, %1, %2, %3;" : "=d"(y) : "d"(x), "d"(a), "d"(b));
  return y;
}

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* __restrict__ out, long long iters, T a, T b) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  T x0 = (T)(threadIdx.x & 7), x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (long long k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x0 = fma_rn<T>(x0, a, b);
      x1 = fma_rn<T>(x1, a, b);
      x2 = fma_rn<T>(x2, a, b);
      x3 = fma_rn<T>(x3, a, b);
      x4 = fma_rn<T>(x4, a, b);
      x5 = fma_rn<T>(x5, a, b);
      x6 = fma_rn<T>(x6, a, b);
      x7 = fma_rn<T>(x7, a, b);
    }
  }
  out[tid] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

}  // namespace

extern "C" int fire_selftest_fma_rate(int32_t dtype, int64_t iters, int32_t blocks, void* out, void* stream) {
  if ((dtype != 0 && dtype != 1) || iters < 1 || blocks < 1 || !out) return FIRE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // each loop round does four multiply-adds per chain
  const long long rounds = (iters + 3) / 4;
  if (dtype == 0)
    fma_probe_kernel<double><<<blocks, 256, 0, s>>>((double*)out, rounds, 0.9999999, 1e-7);
  else
    fma_probe_kernel<float><<<blocks, 256, 0, s>>>((float*)out, rounds, 0.9999f, 1e-4f);
  return cudaGetLastError() == cudaSuccess ? FIRE_OK : FIRE_ERR_CUDA;
}

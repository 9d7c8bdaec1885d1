// Measured FMA throughput of the device: the ALU roof of the transport sweep
// (FP32 in mixed mode, FP64 in the plain mode).  Each thread runs 8
// independent chains of dependent FMAs; the grid fills every SM.  The result
// goes to a file-scope sink so that the compiler keeps the arithmetic.
#include <cuda_runtime.h>

#include "obte.h"

namespace {

__device__ double g_obte_fma_sink[1];

template <typename T, int ITERS>
__global__ void __launch_bounds__(256) fma_rate_kernel(T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-7;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)-1.2345) g_obte_fma_sink[0] = (double)s;  // never true; keeps the chains live
}

template <typename T>
int measure(int device, double* out) {
  constexpr int ITERS = sizeof(T) == 8 ? 256 : 4096;  // FP64 runs at 1/64 the rate
  if (cudaSetDevice(device) != cudaSuccess) return OBTE_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return OBTE_ECUDA;
  const int blocks = sms * 8, threads = 256;
  cudaStream_t st;
  cudaEvent_t e0, e1;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return OBTE_ECUDA;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_rate_kernel<T, ITERS><<<blocks, threads, 0, st>>>((T)0.999999, (T)1e-7);  // warm-up
  cudaEventRecord(e0, st);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) fma_rate_kernel<T, ITERS><<<blocks, threads, 0, st>>>((T)0.999999, (T)1e-7);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (e != cudaSuccess || ms <= 0.f) return OBTE_ECUDA;
  const double flops = 2.0 * 8.0 * ITERS * (double)blocks * threads * reps;
  *out = flops / (ms * 1e-3);
  return OBTE_OK;
}

}  // namespace

extern "C" int obte_measure_fma_rate(int precision, int device, double* flops_per_s) {
  if (!flops_per_s || (precision != OBTE_FP64 && precision != OBTE_MIXED)) return OBTE_EINVAL;
  return precision == OBTE_FP64 ? measure<double>(device, flops_per_s) : measure<float>(device, flops_per_s);
}

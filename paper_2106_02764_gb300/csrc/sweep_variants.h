// Sweep kernel variants compiled into the library, one list per translation
// unit (compiled in parallel).  X(T, DIM, G, RMAX, HAS_S).
#pragma once

#include "obte_internal.h"

#define OBTE_SWEEP_F2(X) \
  X(float, 2, 8, 4, false) \
  X(float, 2, 16, 4, false) \
  X(float, 2, 8, 8, false) \
  X(float, 2, 16, 2, false) \
  X(float, 2, 8, 2, false) \
  X(float, 2, 4, 4, false) \
  X(float, 2, 16, 1, false)

#define OBTE_SWEEP_F3(X) \
  X(float, 3, 8, 4, false) \
  X(float, 3, 4, 4, false) \
  X(float, 3, 8, 2, false) \
  X(float, 3, 4, 2, false) \
  X(float, 3, 4, 8, false) \
  X(float, 3, 8, 8, false)

#define OBTE_SWEEP_D2(X) \
  X(double, 2, 8, 4, false) \
  X(double, 2, 4, 4, false) \
  X(double, 2, 8, 2, false) \
  X(double, 2, 4, 8, false) \
  X(double, 2, 8, 1, false)

#define OBTE_SWEEP_D3(X) \
  X(double, 3, 4, 4, false) \
  X(double, 3, 4, 2, false) \
  X(double, 3, 8, 2, false) \
  X(double, 3, 4, 8, false)

#define OBTE_SWEEP_S(X) \
  X(float, 2, 8, 4, true) \
  X(float, 2, 16, 2, true) \
  X(float, 2, 8, 2, true) \
  X(float, 2, 16, 1, true) \
  X(float, 2, 4, 4, true) \
  X(double, 2, 8, 2, true) \
  X(double, 2, 4, 4, true) \
  X(double, 2, 8, 1, true) \
  X(double, 2, 4, 8, true)

#define OBTE_SWEEP_VARIANTS(X) OBTE_SWEEP_F2(X) OBTE_SWEEP_F3(X) OBTE_SWEEP_D2(X) OBTE_SWEEP_D3(X) OBTE_SWEEP_S(X)

#define OBTE_SWEEP_NAME(T, D, G, R, S) obte_sweep_##T##_##D##_##G##_##R##_##S
#define OBTE_SWEEP_DECLARE(T, D, G, R, S)                                                        \
  cudaError_t OBTE_SWEEP_NAME(T, D, G, R, S)(const SweepLaunch* L, int threads, int blocks,       \
                                             size_t smem, cudaStream_t st, int* occupancy);
OBTE_SWEEP_VARIANTS(OBTE_SWEEP_DECLARE)

// In a variant translation unit (after including sweep.cuh): the launcher.
// With L == nullptr it only reports blocks per SM through *occupancy.
#define OBTE_SWEEP_DEFINE(T, D, G, R, S)                                                          \
  cudaError_t OBTE_SWEEP_NAME(T, D, G, R, S)(const SweepLaunch* L, int threads, int blocks,       \
                                             size_t smem, cudaStream_t st, int* occupancy) {     \
    auto k = obte::sweep_kernel<T, D, G, R, S>;                                                   \
    static bool configured = false;                                                               \
    if (!configured) {                                                                            \
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                           200 * 1024);                                           \
      if (e != cudaSuccess) return e;                                                             \
      configured = true;                                                                          \
    }                                                                                             \
    if (!L) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, k, threads, smem);    \
    k<<<blocks, threads, smem, st>>>(*L);                                                         \
    return cudaGetLastError();                                                                    \
  }

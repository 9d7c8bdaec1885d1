// 3D block-kernel variants compiled into the library.  X(T, G, RMAX, HAS_S).
#pragma once

#include "obte_internal.h"

#define OBTE_SWEEP3D_VARIANTS(X) \
  X(float, 8, 4, false) \
  X(float, 4, 4, false) \
  X(float, 8, 8, false) \
  X(float, 4, 8, false) \
  X(float, 8, 2, false) \
  X(double, 4, 4, false) \
  X(double, 4, 8, false) \
  X(double, 2, 4, false) \
  X(float, 8, 4, true) \
  X(double, 4, 4, true)

#define OBTE_SWEEP3D_NAME(T, G, R, S) obte_sweep3d_##T##_##G##_##R##_##S
#define OBTE_SWEEP3D_DECLARE(T, G, R, S)                                                     \
  cudaError_t OBTE_SWEEP3D_NAME(T, G, R, S)(const SweepLaunch* L, int threads, size_t smem, \
                                            cudaStream_t st);
OBTE_SWEEP3D_VARIANTS(OBTE_SWEEP3D_DECLARE)

#define OBTE_SWEEP3D_DEFINE(T, G, R, S)                                                       \
  cudaError_t OBTE_SWEEP3D_NAME(T, G, R, S)(const SweepLaunch* L, int threads, size_t smem,  \
                                            cudaStream_t st) {                               \
    auto k = obte::sweep3d_kernel<T, G, R, S>;                                               \
    static bool configured = false;                                                          \
    if (!configured) {                                                                       \
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                           226 * 1024);                                      \
      if (e != cudaSuccess) return e;                                                        \
      configured = true;                                                                     \
    }                                                                                        \
    k<<<L->n_items, threads, smem, st>>>(*L);                                                 \
    return cudaGetLastError();                                                               \
  }

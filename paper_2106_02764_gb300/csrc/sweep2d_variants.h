// 2D warp-kernel variants compiled into the library, one list per translation
// unit.  X(T, G, RMAX, HAS_S, RFIXED).
#pragma once

#include "obte_internal.h"

#define OBTE_SWEEP2D_WF(X) \
  X(float, 8, 8, false, true) \
  X(float, 6, 8, false, true) \
  X(float, 4, 8, false, true) \
  X(float, 4, 4, false, true) \
  X(float, 8, 4, false, true) \
  X(float, 8, 2, false, true) \
  X(float, 8, 3, false, true) \
  X(float, 8, 5, false, true) \
  X(float, 8, 6, false, true) \
  X(float, 16, 4, false, true) \
  X(float, 16, 2, false, true) \
  X(float, 16, 1, false, true) \
  X(float, 8, 1, false, true)

#define OBTE_SWEEP2D_WS(X) \
  X(float, 8, 8, true, true) \
  X(float, 4, 8, true, true) \
  X(float, 4, 4, true, true) \
  X(float, 8, 4, true, true) \
  X(float, 16, 4, true, true) \
  X(float, 16, 2, true, true) \
  X(float, 16, 1, true, true) \
  X(float, 8, 1, true, true) \
  X(double, 4, 8, true, true) \
  X(double, 8, 4, true, true) \
  X(double, 8, 2, true, true) \
  X(double, 8, 1, true, true)

#define OBTE_SWEEP2D_WD(X) \
  X(double, 4, 8, false, true) \
  X(double, 2, 8, false, true) \
  X(double, 8, 4, false, true) \
  X(double, 8, 2, false, true) \
  X(double, 8, 1, false, true)

#define OBTE_SWEEP2D_WB(X) \
  X(float, 8, 8, false, false) \
  X(double, 4, 8, false, false) \
  X(float, 8, 8, true, false) \
  X(double, 4, 8, true, false)

#define OBTE_SWEEP2D_VARIANTS(X) OBTE_SWEEP2D_WF(X) OBTE_SWEEP2D_WS(X) OBTE_SWEEP2D_WD(X) OBTE_SWEEP2D_WB(X)

#define OBTE_SWEEP2D_NAME(T, G, R, S, F) obte_sweep2d_##T##_##G##_##R##_##S##_##F
// blocks == 0: one warp per work item; blocks > 0: that many persistent
// blocks; L == nullptr: only report the warps per block in *wpb
#define OBTE_SWEEP2D_DECLARE(T, G, R, S, F) \
  cudaError_t OBTE_SWEEP2D_NAME(T, G, R, S, F)(const SweepLaunch* L, int blocks, cudaStream_t st, int* wpb);
OBTE_SWEEP2D_VARIANTS(OBTE_SWEEP2D_DECLARE)

#define OBTE_SWEEP2D_DEFINE(T, G, R, S, F)                                                      \
  cudaError_t OBTE_SWEEP2D_NAME(T, G, R, S, F)(const SweepLaunch* L, int blocks, cudaStream_t st, \
                                               int* wpb_out) {                                 \
    constexpr int wpb = obte::WarpCfg<T, G, R>::WPB;                                            \
    if (!L) {                                                                                  \
      *wpb_out = wpb;                                                                          \
      return cudaSuccess;                                                                      \
    }                                                                                          \
    const int need = (L->n_items + wpb - 1) / wpb;                                             \
    const int b = (blocks > 0 && blocks < need) ? blocks : need;                               \
    if (L->flags & (SWEEP_FLUX | SWEEP_RECORD))                                                \
      obte::sweep2d_warp_kernel<T, G, R, S, F, true><<<b, 32 * wpb, 0, st>>>(*L);               \
    else                                                                                       \
      obte::sweep2d_warp_kernel<T, G, R, S, F, false><<<b, 32 * wpb, 0, st>>>(*L);              \
    return cudaGetLastError();                                                                 \
  }

// Two-warp groups (NH = 2, sweep2d_warp_kernel): X(T, G, RMAX), FP32 without
// s(x), rows fill 64 lanes (ny = 64 RMAX), four groups per block of eight
// warps.
#define OBTE_SWEEP2D_W2(X) X(float, 8, 4)

#define OBTE_SWEEP2D_W2_NAME(T, G, R) obte_sweep2d_split_##T##_##G##_##R
#define OBTE_SWEEP2D_W2_DECLARE(T, G, R) \
  cudaError_t OBTE_SWEEP2D_W2_NAME(T, G, R)(const SweepLaunch* L, int blocks, cudaStream_t st, int* wpb);
OBTE_SWEEP2D_W2(OBTE_SWEEP2D_W2_DECLARE)

#define OBTE_SWEEP2D_W2_DEFINE(T, G, R)                                                        \
  cudaError_t OBTE_SWEEP2D_W2_NAME(T, G, R)(const SweepLaunch* L, int blocks, cudaStream_t st, \
                                            int* wpb_out) {                                  \
    constexpr int wpb = obte::WarpCfg<T, G, R, 2>::WPB;                                       \
    if (!L) {                                                                                \
      *wpb_out = wpb;                                                                        \
      return cudaSuccess;                                                                    \
    }                                                                                        \
    if (L->item_counter) return cudaErrorInvalidValue;                                        \
    const int need = (L->n_items + 3) / 4;                                                   \
    const int b = (blocks > 0 && blocks < need) ? blocks : need;                             \
    if (L->flags & (SWEEP_FLUX | SWEEP_RECORD))                                              \
      obte::sweep2d_warp_kernel<T, G, R, false, true, true, 2><<<b, 32 * wpb, 0, st>>>(*L);   \
    else                                                                                     \
      obte::sweep2d_warp_kernel<T, G, R, false, true, false, 2><<<b, 32 * wpb, 0, st>>>(*L);  \
    return cudaGetLastError();                                                               \
  }

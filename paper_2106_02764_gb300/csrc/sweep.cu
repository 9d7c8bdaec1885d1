// Dispatch to the compiled sweep kernel variants (sweep_variants.h).
#include "sweep_variants.h"
#include "sweep2d_variants.h"
#include "sweep3d_variants.h"

static int prec_of(float*) { return 1; }
static int prec_of(double*) { return 0; }

#define OBTE_MATCH(T, D, GG, RR, SS) \
  (precision == prec_of((T*)nullptr) && dim == D && G == GG && RMAX == RR && has_s == SS)

cudaError_t launch_sweep(const SweepLaunch& L, int precision, int dim, int G, int RMAX, bool has_s,
                         int threads, int blocks, size_t smem, cudaStream_t st) {
#define X(T, D, GG, RR, SS) \
  if (OBTE_MATCH(T, D, GG, RR, SS)) return OBTE_SWEEP_NAME(T, D, GG, RR, SS)(&L, threads, blocks, smem, st, nullptr);
  OBTE_SWEEP_VARIANTS(X)
#undef X
  return cudaErrorInvalidValue;
}

bool sweep_variant_exists(int precision, int dim, int G, int RMAX, bool has_s) {
#define X(T, D, GG, RR, SS) \
  if (OBTE_MATCH(T, D, GG, RR, SS)) return true;
  OBTE_SWEEP_VARIANTS(X)
#undef X
  return false;
}

size_t sweep_smem_bytes(int precision, int dim, int G, int RMAX, int threads) {
  const size_t e = precision == 0 ? sizeof(double) : sizeof(float);
  size_t b = 3 * (size_t)threads * G * e;  // exchange [2][threads][G] + scratch [threads][G]
  if (dim == 3) b += 2 * (size_t)threads * RMAX * G * e;
  return b;
}

int sweep_blocks_per_sm(int precision, int dim, int G, int RMAX, bool has_s, int threads,
                        size_t smem) {
  int n = 1;
#define X(T, D, GG, RR, SS)                                                                \
  if (OBTE_MATCH(T, D, GG, RR, SS)) {                                                     \
    if (OBTE_SWEEP_NAME(T, D, GG, RR, SS)(nullptr, threads, 0, smem, nullptr, &n) != cudaSuccess) n = 1; \
    return n;                                                                             \
  }
  OBTE_SWEEP_VARIANTS(X)
#undef X
  return n;
}

#define OBTE_MATCH2D(T, GG, RR, SS, FF) \
  (precision == prec_of((T*)nullptr) && G == GG && RMAX == RR && has_s == SS && rfixed == FF)

cudaError_t launch_sweep2d_warp(const SweepLaunch& L, int precision, int G, int RMAX, bool has_s,
                                bool rfixed, int blocks, cudaStream_t st) {
#define X(T, GG, RR, SS, FF) \
  if (OBTE_MATCH2D(T, GG, RR, SS, FF)) return OBTE_SWEEP2D_NAME(T, GG, RR, SS, FF)(&L, blocks, st, nullptr);
  OBTE_SWEEP2D_VARIANTS(X)
#undef X
  return cudaErrorInvalidValue;
}

int sweep2d_warps_per_block(int precision, int G, int RMAX, bool has_s, bool rfixed) {
  int w = 0;
#define X(T, GG, RR, SS, FF) \
  if (OBTE_MATCH2D(T, GG, RR, SS, FF)) OBTE_SWEEP2D_NAME(T, GG, RR, SS, FF)(nullptr, 0, nullptr, &w);
  OBTE_SWEEP2D_VARIANTS(X)
#undef X
  return w;
}

bool sweep2d_warp_exists(int precision, int G, int RMAX, bool has_s, bool rfixed) {
#define X(T, GG, RR, SS, FF) \
  if (OBTE_MATCH2D(T, GG, RR, SS, FF)) return true;
  OBTE_SWEEP2D_VARIANTS(X)
#undef X
  return false;
}

#define OBTE_MATCH2DS(T, GG, RR) (precision == prec_of((T*)nullptr) && G == GG && RMAX == RR)

cudaError_t launch_sweep2d_split(const SweepLaunch& L, int precision, int G, int RMAX, int blocks,
                                 cudaStream_t st) {
#define X(T, GG, RR) \
  if (OBTE_MATCH2DS(T, GG, RR)) return OBTE_SWEEP2D_W2_NAME(T, GG, RR)(&L, blocks, st, nullptr);
  OBTE_SWEEP2D_W2(X)
#undef X
  return cudaErrorInvalidValue;
}

bool sweep2d_split_exists(int precision, int G, int RMAX) {
#define X(T, GG, RR) \
  if (OBTE_MATCH2DS(T, GG, RR)) return true;
  OBTE_SWEEP2D_W2(X)
#undef X
  return false;
}

#define OBTE_MATCH3D(T, GG, RR, SS) \
  (precision == prec_of((T*)nullptr) && G == GG && RMAX == RR && has_s == SS)

cudaError_t launch_sweep3d(const SweepLaunch& L, int precision, int G, int RMAX, bool has_s,
                           int threads, size_t smem, cudaStream_t st) {
#define X(T, GG, RR, SS) \
  if (OBTE_MATCH3D(T, GG, RR, SS)) return OBTE_SWEEP3D_NAME(T, GG, RR, SS)(&L, threads, smem, st);
  OBTE_SWEEP3D_VARIANTS(X)
#undef X
  return cudaErrorInvalidValue;
}

bool sweep3d_exists(int precision, int G, int RMAX, bool has_s) {
#define X(T, GG, RR, SS) \
  if (OBTE_MATCH3D(T, GG, RR, SS)) return true;
  OBTE_SWEEP3D_VARIANTS(X)
#undef X
  return false;
}

size_t sweep3d_smem_bytes(int precision, int G, int RMAX, int threads) {
  const size_t e = precision == 0 ? sizeof(double) : sizeof(float);
  const size_t nt = RMAX >= 8 ? 256 : 512;  // the kernel's compile-time block stride
  (void)threads;
  // exchange [2][R][G][nt] + scratch [G][nt] + T_L partials by row [2][nt R]
  // FP32: records of two steps [2][R][nt] of 16 bytes
  return (2 * (size_t)RMAX + 1) * G * nt * e + 2 * nt * (size_t)RMAX * e +
         (precision == 1 ? 2 * (size_t)RMAX * nt * 16 : 0);
}

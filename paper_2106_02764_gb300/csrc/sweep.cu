// Instantiation and dispatch of the sweep kernel variants.
#include "sweep.cuh"

namespace {

template <typename T, int DIM, int G, int RMAX>
cudaError_t run(const SweepLaunch& L, int threads, int blocks, size_t smem, cudaStream_t st) {
  auto k = obte::sweep_kernel<T, DIM, G, RMAX>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k<<<blocks, threads, smem, st>>>(L);
  return cudaGetLastError();
}

// (precision, dim, G, RMAX) variants compiled into the library
#define OBTE_SWEEP_VARIANTS(X) \
  X(float, 2, 8, 4)            \
  X(float, 2, 16, 4)           \
  X(float, 2, 8, 8)            \
  X(float, 2, 16, 2)           \
  X(float, 2, 8, 2)            \
  X(float, 2, 4, 4)            \
  X(float, 2, 16, 1)           \
  X(float, 3, 8, 4)            \
  X(float, 3, 4, 4)            \
  X(float, 3, 8, 2)            \
  X(float, 3, 4, 2)            \
  X(float, 3, 4, 8)            \
  X(float, 3, 8, 8)            \
  X(double, 2, 8, 4)           \
  X(double, 2, 4, 4)           \
  X(double, 2, 8, 2)           \
  X(double, 2, 4, 8)           \
  X(double, 2, 8, 1)           \
  X(double, 3, 4, 4)           \
  X(double, 3, 4, 2)           \
  X(double, 3, 8, 2)           \
  X(double, 3, 4, 8)

}  // namespace

static int prec_of(float*) { return 1; }
static int prec_of(double*) { return 0; }

cudaError_t launch_sweep(const SweepLaunch& L, int precision, int dim, int G, int RMAX,
                         int threads, int blocks, size_t smem, cudaStream_t st) {
#define X(T, D, GG, RR)                                                              \
  if (precision == prec_of((T*)nullptr) && dim == D && G == GG && RMAX == RR) \
    return run<T, D, GG, RR>(L, threads, blocks, smem, st);
  OBTE_SWEEP_VARIANTS(X)
#undef X
  return cudaErrorInvalidValue;
}

bool sweep_variant_exists(int precision, int dim, int G, int RMAX) {
#define X(T, D, GG, RR) \
  if (precision == prec_of((T*)nullptr) && dim == D && G == GG && RMAX == RR) return true;
  OBTE_SWEEP_VARIANTS(X)
#undef X
  return false;
}

size_t sweep_smem_bytes(int precision, int dim, int G, int RMAX, int threads) {
  const size_t e = precision == 0 ? sizeof(double) : sizeof(float);
  size_t b = 2 * (size_t)threads * G * e;
  if (dim == 3) b += 2 * (size_t)threads * RMAX * G * e;
  return b;
}

int sweep_blocks_per_sm(int precision, int dim, int G, int RMAX, int threads, size_t smem) {
  int n = 0;
#define X(T, D, GG, RR)                                                                     \
  if (precision == prec_of((T*)nullptr) && dim == D && G == GG && RMAX == RR) {            \
    cudaFuncSetAttribute(obte::sweep_kernel<T, D, GG, RR>,                                 \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);         \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, obte::sweep_kernel<T, D, GG, RR>, \
                                                      threads, smem) != cudaSuccess)       \
      n = 1;                                                                               \
    return n;                                                                              \
  }
  OBTE_SWEEP_VARIANTS(X)
#undef X
  return 1;
}

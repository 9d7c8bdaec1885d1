// Fourier first guess (App. B, orthogonal-grid subset; Algorithm 1 first line):
// conjugate gradients on the finite-volume heat-conduction system of the
// solid cells, in one cooperative launch.
//
// On a Cartesian grid the secondary (non-orthogonal) flux of App. B vanishes,
// leaving the primary-flux system  sum_j w_a (T_i - T_j) = sum_j w_a J_ij  over
// solid neighbours j (w_a = (h_x / h_a)^2, walls adiabatic), with J_ij the jump
// of the applied temperature difference across the periodic x plane (R^P of
// App. B: the image across the low side is hotter by dT).  The matrix is
// symmetric positive semidefinite with the constant vector as null space and
// the right-hand side sums to zero, so CG converges to a solution; its mean is
// removed at the end.  CG starts from the linear profile -dT (x + 1/2) / nx.
#include <cooperative_groups.h>

#include "obte_internal.h"

namespace cg = cooperative_groups;

namespace {



template <typename T>
__device__ __forceinline__ T apply_A(const CGArgs& a, const T* v, int c, uint8_t code, int x, int y,
                                     int z) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const T vc = v[c];
  T acc = T(0);
  if (!(code & CODE_WALL_XM)) acc += (T)a.wx * (vc - v[c - x + (x > 0 ? x - 1 : nx - 1)]);
  if (!(code & CODE_WALL_XP)) acc += (T)a.wx * (vc - v[c - x + (x < nx - 1 ? x + 1 : 0)]);
  if (!(code & CODE_WALL_YM)) acc += (T)a.wy * (vc - v[c + nx * ((y > 0 ? y - 1 : ny - 1) - y)]);
  if (!(code & CODE_WALL_YP)) acc += (T)a.wy * (vc - v[c + nx * ((y < ny - 1 ? y + 1 : 0) - y)]);
  if (a.dim == 3) {
    if (!(code & CODE_WALL_ZM)) acc += (T)a.wz * (vc - v[c + nx * ny * ((z > 0 ? z - 1 : nz - 1) - z)]);
    if (!(code & CODE_WALL_ZP)) acc += (T)a.wz * (vc - v[c + nx * ny * ((z < nz - 1 ? z + 1 : 0) - z)]);
  }
  return acc;
}

// sum of the grid's per-block partials, done by warp 0 of every block and
// broadcast through shared memory (same order in every block)
__device__ double sum_partials(const double* part, int n, double* bc) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *bc = s;
  }
  __syncthreads();
  return *bc;
}

__device__ double block_reduce(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) s += red[i];
  return s;
}

template <typename T>
__global__ void fourier_cg_kernel(CGArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[32];
  __shared__ double bc;
  const int n = a.nx * a.ny * a.nz;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  T* x = reinterpret_cast<T*>(a.x);
  T* r = reinterpret_cast<T*>(a.r);
  T* p = reinterpret_cast<T*>(a.p);
  T* q = reinterpret_cast<T*>(a.q);
  double* part0 = a.part;
  double* part1 = a.part + gridDim.x;

  // x0 = linear profile; r = b - A x0; p = r
  for (int c = tid; c < n; c += stride) {
    const int xi = c % a.nx;
    x[c] = (a.code[c] & CODE_SOLID) ? (T)(-a.dT * ((xi + 0.5) / a.nx - 0.5)) : T(0);
  }
  grid.sync();
  double rr_l = 0.0, bb_l = 0.0;
  for (int c = tid; c < n; c += stride) {
    const uint8_t code = a.code[c];
    T rc = T(0);
    if (code & CODE_SOLID) {
      const int xi = c % a.nx, yi = (c / a.nx) % a.ny, zi = c / (a.nx * a.ny);
      double b = 0.0;
      if (xi == 0 && !(code & CODE_WALL_XM)) b += a.wx * a.dT;
      if (xi == a.nx - 1 && !(code & CODE_WALL_XP)) b -= a.wx * a.dT;
      rc = (T)b - apply_A<T>(a, x, c, code, xi, yi, zi);
      bb_l += b * b;
    }
    r[c] = rc;
    p[c] = rc;
    rr_l += (double)rc * (double)rc;
  }
  double s = block_reduce(rr_l, red);
  double s2 = block_reduce(bb_l, red);
  if (threadIdx.x == 0) {
    part0[blockIdx.x] = s;
    part1[blockIdx.x] = s2;
  }
  grid.sync();
  double rr = sum_partials(part0, gridDim.x, &bc);
  double bb = sum_partials(part1, gridDim.x, &bc);
  grid.sync();
  const double stop = a.tol * a.tol * bb;
  int it = 0;
  while (it < a.max_iter && rr > stop && bb > 0.0) {
    // q = A p, p.q
    double pq_l = 0.0;
    for (int c = tid; c < n; c += stride) {
      const uint8_t code = a.code[c];
      T qc = T(0);
      if (code & CODE_SOLID) {
        const int xi = c % a.nx, yi = (c / a.nx) % a.ny, zi = c / (a.nx * a.ny);
        qc = apply_A<T>(a, p, c, code, xi, yi, zi);
      }
      q[c] = qc;
      pq_l += (double)p[c] * (double)qc;
    }
    s = block_reduce(pq_l, red);
    if (threadIdx.x == 0) part0[blockIdx.x] = s;
    grid.sync();
    const double pq = sum_partials(part0, gridDim.x, &bc);
    if (!(pq > 0.0)) break;  // uniform across blocks
    const double alpha = rr / pq;
    double rn_l = 0.0;
    for (int c = tid; c < n; c += stride) {
      x[c] += (T)alpha * p[c];
      const T rc = r[c] - (T)alpha * q[c];
      r[c] = rc;
      rn_l += (double)rc * (double)rc;
    }
    s = block_reduce(rn_l, red);
    if (threadIdx.x == 0) part1[blockIdx.x] = s;
    grid.sync();
    const double rn = sum_partials(part1, gridDim.x, &bc);
    const double beta = rn / rr;
    rr = rn;
    for (int c = tid; c < n; c += stride) p[c] = r[c] + (T)beta * p[c];
    ++it;
    grid.sync();
  }
  // remove the mean over solid cells
  double sum_l = 0.0, cnt_l = 0.0;
  for (int c = tid; c < n; c += stride)
    if (a.code[c] & CODE_SOLID) {
      sum_l += (double)x[c];
      cnt_l += 1.0;
    }
  s = block_reduce(sum_l, red);
  s2 = block_reduce(cnt_l, red);
  if (threadIdx.x == 0) {
    part0[blockIdx.x] = s;
    part1[blockIdx.x] = s2;
  }
  grid.sync();
  const double sum = sum_partials(part0, gridDim.x, &bc);
  const double cnt = sum_partials(part1, gridDim.x, &bc);
  const double mean = cnt > 0 ? sum / cnt : 0.0;
  for (int c = tid; c < n; c += stride)
    a.T_out[c] = (a.code[c] & CODE_SOLID) ? (double)x[c] - mean : 0.0;
  if (tid == 0) *a.iters_out = it;
}

// One thread block per geometry: the same CG with block barriers only (no
// grid synchronisation), so many geometries solve in one launch.
template <typename T>
__global__ void __launch_bounds__(1024) fourier_cg_block_kernel(const CGArgs* jobs) {
  const CGArgs& a = jobs[blockIdx.x];
  __shared__ double red[32];
  const int n = a.nx * a.ny * a.nz;
  const int t0 = threadIdx.x, st = blockDim.x;
  T* x = reinterpret_cast<T*>(a.x);
  T* r = reinterpret_cast<T*>(a.r);
  T* p = reinterpret_cast<T*>(a.p);
  T* q = reinterpret_cast<T*>(a.q);
  __shared__ double bval[2];
  auto bsum = [&](double v) -> double {  // block sum, valid in every thread
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) s += red[i];
      bval[0] = s;
    }
    __syncthreads();
    return bval[0];
  };
  for (int c = t0; c < n; c += st) {
    const int xi = c % a.nx;
    x[c] = (a.code[c] & CODE_SOLID) ? (T)(-a.dT * ((xi + 0.5) / a.nx - 0.5)) : T(0);
  }
  __syncthreads();
  double rr_l = 0.0, bb_l = 0.0;
  for (int c = t0; c < n; c += st) {
    const uint8_t code = a.code[c];
    T rc = T(0);
    if (code & CODE_SOLID) {
      const int xi = c % a.nx, yi = (c / a.nx) % a.ny, zi = c / (a.nx * a.ny);
      double b = 0.0;
      if (xi == 0 && !(code & CODE_WALL_XM)) b += a.wx * a.dT;
      if (xi == a.nx - 1 && !(code & CODE_WALL_XP)) b -= a.wx * a.dT;
      rc = (T)b - apply_A<T>(a, x, c, code, xi, yi, zi);
      bb_l += b * b;
    }
    r[c] = rc;
    p[c] = rc;
    rr_l += (double)rc * (double)rc;
  }
  double rr = bsum(rr_l);
  const double bb = bsum(bb_l);
  const double stop = a.tol * a.tol * bb;
  int it = 0;
  while (it < a.max_iter && rr > stop && bb > 0.0) {
    double pq_l = 0.0;
    for (int c = t0; c < n; c += st) {
      const uint8_t code = a.code[c];
      T qc = T(0);
      if (code & CODE_SOLID) {
        const int xi = c % a.nx, yi = (c / a.nx) % a.ny, zi = c / (a.nx * a.ny);
        qc = apply_A<T>(a, p, c, code, xi, yi, zi);
      }
      q[c] = qc;
      pq_l += (double)p[c] * (double)qc;
    }
    const double pq = bsum(pq_l);
    if (!(pq > 0.0)) break;
    const double alpha = rr / pq;
    double rn_l = 0.0;
    for (int c = t0; c < n; c += st) {
      x[c] += (T)alpha * p[c];
      const T rc = r[c] - (T)alpha * q[c];
      r[c] = rc;
      rn_l += (double)rc * (double)rc;
    }
    const double rn = bsum(rn_l);
    const double beta = rn / rr;
    rr = rn;
    for (int c = t0; c < n; c += st) p[c] = r[c] + (T)beta * p[c];
    __syncthreads();
    ++it;
  }
  double sum_l = 0.0, cnt_l = 0.0;
  for (int c = t0; c < n; c += st)
    if (a.code[c] & CODE_SOLID) {
      sum_l += (double)x[c];
      cnt_l += 1.0;
    }
  const double sum = bsum(sum_l);
  const double cnt = bsum(cnt_l);
  const double mean = cnt > 0 ? sum / cnt : 0.0;
  for (int c = t0; c < n; c += st) a.T_out[c] = (a.code[c] & CODE_SOLID) ? (double)x[c] - mean : 0.0;
  if (t0 == 0) *a.iters_out = it;
}

}  // namespace

CGArgs make_cg_args(const GeomDev& g, double hx, double hy, double hz, int max_iter, double tol,
                    double* T_out, int* iters_out, double* work, int blocks_max) {
  CGArgs a;
  a.code = g.code;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.dim = g.dim;
  a.py = g.py;
  a.pz = g.pz;
  a.wx = 1.0;
  a.wy = (hx / hy) * (hx / hy);
  a.wz = g.dim == 3 ? (hx / hz) * (hx / hz) : 0.0;
  a.dT = g.dT;
  a.max_iter = max_iter;
  a.tol = tol;
  const size_t n = (size_t)g.n_cells;
  a.x = work;
  a.r = work + n;
  a.p = work + 2 * n;
  a.q = work + 3 * n;
  a.part = work + 4 * n;
  a.T_out = T_out;
  a.iters_out = iters_out;
  (void)blocks_max;
  return a;
}

cudaError_t launch_fourier_cg_blocks(const CGArgs* jobs_dev, int n_jobs, int precision,
                                     cudaStream_t st) {
  if (precision == 0) fourier_cg_block_kernel<double><<<n_jobs, 1024, 0, st>>>(jobs_dev);
  else fourier_cg_block_kernel<float><<<n_jobs, 1024, 0, st>>>(jobs_dev);
  return cudaGetLastError();
}

size_t fourier_work_doubles(int n_cells, int blocks_max) {
  return 4 * (size_t)n_cells + 2 * (size_t)blocks_max + 8;
}

cudaError_t launch_fourier_cg(const GeomDev& g, double hx, double hy, double hz, int precision,
                              int max_iter, double tol, double* T_out, int* iters_out,
                              double* work, int blocks_max, cudaStream_t st) {
  CGArgs a = make_cg_args(g, hx, hy, hz, max_iter, tol, T_out, iters_out, work, blocks_max);
  const size_t n = (size_t)g.n_cells;
  const int threads = 256;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void* kern = precision == 0 ? (void*)fourier_cg_kernel<double> : (void*)fourier_cg_kernel<float>;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e != cudaSuccess) return e;
  int blocks = sms * (per_sm < 2 ? per_sm : 2);
  const int need = (int)((n + threads - 1) / threads);
  if (blocks > need) blocks = need;
  if (blocks > blocks_max) blocks = blocks_max;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(kern, blocks, threads, args, 0, st);
}

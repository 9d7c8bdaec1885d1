// Anderson acceleration of the source iteration (Algorithm 1's fixed point).
//
// The iteration state x = (T_L over all cells, T_w over wall faces, the row
// values carried between sweeps) is mapped by one sweep + finalisation to
// g(x).  Anderson mixing (type II, window m) replaces x_{k+1} = g(x_k) by
//     x_{k+1} = g_k - sum_i gamma_i (g_{i+1} - g_i),
//     gamma = argmin || f_k - sum_i gamma_i (f_{i+1} - f_i) ||,  f = g(x) - x,
// over the last m differences.  The fixed point is unchanged (f = 0 there);
// only the trajectory is.
//
// The row-value part of the state (most of its length) is combined in the
// sweep precision; T_L, T_w, the reductions and the solve stay FP64.
//
// Per iteration (after the finalisation):
//   aa_residual_kernel: f_k = g_k - x_k into history slot, dots f_k . F_j for
//     every slot as per-block partials;
//   aa_solve_kernel: sums the partials, updates the Gram matrix and solves
//     the normal equations for gamma (Gaussian elimination with partial
//     pivoting, Tikhonov-regularised), giving the mixing coefficients c_j of
//     x_{k+1} = sum_j c_j (X_j + F_j);
//   aa_mix_kernel: x_{k+1} into the state and into the next history slot, and
//     the sweep inputs derived from it (s T_L, wall temperatures per side,
//     octant records).
#include <math.h>

#include "obte_internal.h"
#include "records.cuh"

namespace {

template <typename T>
struct AAView {
  // slot s of the FP64 part (T_L then T_w) and of the row-value part
  static __device__ double* xd(const GeomDev& g, int s) { return g.aa_xd + (size_t)s * g.aa_nd; }
  static __device__ double* fd(const GeomDev& g, int s) { return g.aa_fd + (size_t)s * g.aa_nd; }
  static __device__ T* xt(const GeomDev& g, int s) {
    return reinterpret_cast<T*>(g.aa_xt) + (size_t)s * g.aa_nt;
  }
  static __device__ T* ft(const GeomDev& g, int s) {
    return reinterpret_cast<T*>(g.aa_ft) + (size_t)s * g.aa_nt;
  }
};

__device__ __forceinline__ double state_d(const GeomDev& g, long i) {
  return i < g.n_cells ? g.TL[i] : g.Tw[i - g.n_cells];
}

// Solve the m x m system A y = b (row-major, in place) by Gaussian elimination
// with partial pivoting; returns false if a pivot vanishes.
__device__ bool small_solve(double* A, double* b, int m) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(A[r * 8 + c]) > fabs(A[piv * 8 + c])) piv = r;
    if (!(fabs(A[piv * 8 + c]) > 0.0)) return false;
    if (piv != c) {
      for (int k = 0; k < m; ++k) {
        const double t = A[c * 8 + k];
        A[c * 8 + k] = A[piv * 8 + k];
        A[piv * 8 + k] = t;
      }
      const double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    for (int r = c + 1; r < m; ++r) {
      const double f = A[r * 8 + c] / A[c * 8 + c];
      for (int k = c; k < m; ++k) A[r * 8 + k] -= f * A[c * 8 + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = m - 1; c >= 0; --c) {
    double s = b[c];
    for (int k = c + 1; k < m; ++k) s -= A[c * 8 + k] * b[k];
    b[c] = s / A[c * 8 + c];
    if (!isfinite(b[c])) return false;
  }
  return true;
}

template <typename T>
__global__ void aa_residual_kernel(const GeomDev* geoms) {
  const GeomDev& g = geoms[blockIdx.y];
  if (g.aa_m <= 0 || *(volatile int*)g.done) return;
  const int S = g.aa_m + 1;            // history slots
  const int k = *g.aa_k;               // Anderson step (0 = first sweep)
  const int cur = k % S;
  __shared__ double red[8][32];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  const int nvalid = k + 1 < S ? k + 1 : S;  // slots holding residuals after this step
  // slot j of the window (j = 0: this step) -> its base pointers
  const double* fdj[8];
  const T* ftj[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int sl = (k - j + S * 8) % S;
    fdj[j] = AAView<T>::fd(g, sl);
    ftj[j] = AAView<T>::ft(g, sl);
  }
  // FP64 part (T_L, T_w): few elements, FP64 products and sums
  double dots[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) dots[j] = 0.0;
  double* fcur = AAView<T>::fd(g, cur);
  const double* xcur = AAView<T>::xd(g, cur);
  const long nd = g.aa_nd;
  for (long i = tid; i < nd; i += stride) {
    const double f = state_d(g, i) - xcur[i];
    fcur[i] = f;
    dots[0] += f * f;
#pragma unroll
    for (int j = 1; j < 8; ++j)
      if (j < nvalid) dots[j] += f * fdj[j][i];
  }
  // row values: products and the thread / warp sums in the sweep precision,
  // widened once per warp
  T* ftc = AAView<T>::ft(g, cur);
  const T* xtc = AAView<T>::xt(g, cur);
  const T* front = reinterpret_cast<const T*>(g.front);
  T tdots[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) tdots[j] = T(0);
  const long nt = g.aa_nt;
  for (long i = tid; i < nt; i += stride) {
    const T f = front[i] - xtc[i];
    ftc[i] = f;
    tdots[0] = fma(f, f, tdots[0]);
#pragma unroll
    for (int j = 1; j < 8; ++j)
      if (j < nvalid) tdots[j] = fma(f, ftj[j][i], tdots[j]);
  }
  const unsigned FULL = 0xffffffffu;
  const bool any_d = __any_sync(FULL, (long)(tid - (threadIdx.x & 31)) < nd);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    T t = tdots[j];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    double v = (double)t;
    if (any_d) {
      double d = dots[j];
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(FULL, d, o);
      v += d;
    }
    if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double v = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) v += red[threadIdx.x][w];
    g.blk_part[(size_t)blockIdx.x * 8 + threadIdx.x] = v;
  }
}

// After aa_residual_kernel (one block of 8 warps per geometry): warp j sums
// dot j over the block partials; thread 0 updates the Gram matrix and solves
// for the mixing coefficients.
__global__ void aa_solve_kernel(const GeomDev* geoms, int nblocks) {
  const GeomDev& g = geoms[blockIdx.x];
  if (g.aa_m <= 0 || *(volatile int*)g.done) return;
  __shared__ double dv[8];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double v = 0.0;
  for (int b = lane; b < nblocks; b += 32) v += g.blk_part[(size_t)b * 8 + w];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) dv[w] = v;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int S = g.aa_m + 1;
  const int k = *g.aa_k;
  const int cur = k % S;
  const int nvalid = k + 1 < S ? k + 1 : S;
  // Gram matrix of the residual history (slot indices), then gamma
  double* gram = g.aa_gram;  // [S][S] by slot
  for (int j = 0; j < nvalid; ++j) {
    const int sl = (k - j + S * 8) % S;
    gram[cur * S + sl] = dv[j];
    gram[sl * S + cur] = dv[j];
  }
  // logical order oldest .. newest: slot(l) = (k - (nvalid - 1) + l) mod S
  const int mk = nvalid - 1;  // number of differences
  double coef[8];
  for (int l = 0; l < 8; ++l) coef[l] = 0.0;
  coef[mk] = 1.0;
  if (mk > 0) {
    double A[64], b[8];
    auto G = [&](int l1, int l2) {
      const int s1 = (k - mk + l1 + S * 8) % S, s2 = (k - mk + l2 + S * 8) % S;
      return gram[s1 * S + s2];
    };
    double tr = 0.0;
    for (int i = 0; i < mk; ++i) {
      for (int j = 0; j < mk; ++j)
        A[i * 8 + j] = G(i + 1, j + 1) - G(i + 1, j) - G(i, j + 1) + G(i, j);
      b[i] = G(i + 1, mk) - G(i, mk);
      tr += A[i * 8 + i];
    }
    for (int i = 0; i < mk; ++i) A[i * 8 + i] += 1e-12 * tr + 1e-300;
    if (small_solve(A, b, mk)) {
      // x_{k+1} = G_mk - sum_i gamma_i (G_{i+1} - G_i)
      for (int i = 0; i < mk; ++i) {
        coef[i + 1] -= b[i];
        coef[i] += b[i];
      }
    }
  }
  for (int l = 0; l < 8; ++l) g.aa_coef[l] = coef[l];
}

// x_{k+1} = sum_l coef_l (X_l + F_l) over the window; written to the state, to
// the next history slot, and to the sweep inputs (s T_L, wall temperatures).
template <typename T>
__global__ void aa_mix_kernel(const GeomDev* geoms) {
  const GeomDev& g = geoms[blockIdx.y];
  if (g.aa_m <= 0 || *(volatile int*)g.done) return;
  const int S = g.aa_m + 1;
  const int k = *g.aa_k;
  const int nvalid = k + 1 < S ? k + 1 : S;
  const int mk = nvalid - 1;
  const int nxt = (k + 1) % S;
  double c[8];
  T ct[8];
  const double *xdl[8], *fdl[8];
  const T *xtl[8], *ftl[8];
  for (int l = 0; l < 8; ++l) {
    c[l] = l <= mk ? g.aa_coef[l] : 0.0;
    ct[l] = (T)c[l];
    const int sl = (k - mk + l + S * 8) % S;
    xdl[l] = AAView<T>::xd(g, sl);
    fdl[l] = AAView<T>::fd(g, sl);
    xtl[l] = AAView<T>::xt(g, sl);
    ftl[l] = AAView<T>::ft(g, sl);
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  T* src = reinterpret_cast<T*>(g.src);
  T* twc = reinterpret_cast<T*>(g.twc);
  double* xn = AAView<T>::xd(g, nxt);
  const bool recs = g.rec4 != nullptr;
  for (long i = tid; i < g.aa_nd; i += stride) {
    double v = 0.0;
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (l <= mk) v += c[l] * (xdl[l][i] + fdl[l][i]);
    if (i < g.n_cells) {
      if (!(g.code[i] & CODE_SOLID)) v = 0.0;
      g.TL[i] = v;
      const T sv = (T)(g.s ? g.s[i] * v : v);
      src[i] = sv;
      if (recs) obte::rec_put_src<T>(g, (int)i, sv);
    } else {
      const long f = i - g.n_cells;
      g.Tw[f] = v;
      const int cell = g.wall_cell[f], sd = g.wall_side[f];
      twc[(size_t)cell * 6 + sd] = (T)v;
      if (recs) obte::rec_put_wall<T>(g, cell, sd, (T)v);
    }
    xn[i] = v;
  }
  // row values in the sweep precision
  T* front = reinterpret_cast<T*>(g.front);
  T* xtn = AAView<T>::xt(g, nxt);
  for (long i = tid; i < g.aa_nt; i += stride) {
    T v = T(0);
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (l <= mk) v = fma(ct[l], xtl[l][i] + ftl[l][i], v);
    front[i] = v;
    xtn[i] = v;
  }
}

// advance the Anderson step counter (one thread per geometry)
__global__ void aa_step_kernel(const GeomDev* geoms, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const GeomDev& g = geoms[i];
    if (g.aa_m > 0 && !*(volatile int*)g.done) *g.aa_k += 1;
  }
}

// history slot 0 <- the state at iteration 0
template <typename T>
__global__ void aa_init_kernel(const GeomDev* geoms) {
  const GeomDev& g = geoms[blockIdx.y];
  if (g.aa_m <= 0) return;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  double* x0 = AAView<T>::xd(g, 0);
  for (long i = tid; i < g.aa_nd; i += stride) x0[i] = state_d(g, i);
  T* xt0 = AAView<T>::xt(g, 0);
  const T* front = reinterpret_cast<const T*>(g.front);
  for (long i = tid; i < g.aa_nt; i += stride) xt0[i] = front[i];
  if (tid == 0) {
    *g.aa_k = 0;
  }
}

}  // namespace

cudaError_t launch_anderson_init(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                                 cudaStream_t st) {
  dim3 grid(blocks, n_geoms);
  if (precision == 0) aa_init_kernel<double><<<grid, 256, 0, st>>>(geoms_dev);
  else aa_init_kernel<float><<<grid, 256, 0, st>>>(geoms_dev);
  return cudaGetLastError();
}

cudaError_t launch_anderson_step(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                                 cudaStream_t st) {
  dim3 grid(blocks, n_geoms);
  if (blocks > kMaxPartBlocks) return cudaErrorInvalidValue;
  if (precision == 0) {
    aa_residual_kernel<double><<<grid, 256, 0, st>>>(geoms_dev);
    aa_solve_kernel<<<n_geoms, 256, 0, st>>>(geoms_dev, blocks);
    aa_mix_kernel<double><<<grid, 256, 0, st>>>(geoms_dev);
  } else {
    aa_residual_kernel<float><<<grid, 256, 0, st>>>(geoms_dev);
    aa_solve_kernel<<<n_geoms, 256, 0, st>>>(geoms_dev, blocks);
    aa_mix_kernel<float><<<grid, 256, 0, st>>>(geoms_dev);
  }
  aa_step_kernel<<<(n_geoms + 127) / 128, 128, 0, st>>>(geoms_dev, n_geoms);
  return cudaGetLastError();
}

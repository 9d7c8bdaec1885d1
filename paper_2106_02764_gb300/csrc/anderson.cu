// Anderson acceleration of the source iteration (Algorithm 1's fixed point).
//
// The iteration state x = (T_L over all cells, T_w over wall faces, the row
// values carried between sweeps) is mapped by one sweep + finalisation to
// g(x).  Anderson mixing (type II, window m) replaces x_{k+1} = g(x_k) by
//     x_{k+1} = g_k - sum_i gamma_i (g_{i+1} - g_i),
//     gamma = argmin || f_k - sum_i gamma_i (f_{i+1} - f_i) ||,  f = g(x) - x,
// over the last m differences, i.e. x_{k+1} = sum_l c_l g_l with
// coefficients c summing to one.  The fixed point is unchanged (f = 0 there);
// only the trajectory is.
//
// Storage per part (FP64: T_L then T_w; sweep precision: the row values,
// most of the length): history slots G_l = g(x_l) and F_l = f_l, and the
// current iterate X = x_k.  The row-value part is combined in the sweep
// precision (16-byte vector accesses); the reductions and the solve are FP64.
//
// Per iteration (after the finalisation):
//   aa_residual_kernel: F_k = g_k - X and G_k = g_k into history slot k mod
//     (m + 1), and the dots F_k . F_j for every slot as per-block partials;
//   aa_solve_kernel (one block): sums the partials, updates the Gram matrix,
//     solves the regularised normal equations for gamma (one warp, Gaussian
//     elimination with partial pivoting, a row per lane) and advances the
//     step counter;
//   aa_mix_kernel: x_{k+1} = sum_l c_l G_l into the state, into X, and into
//     the sweep inputs derived from it (s T_L, wall temperatures per side,
//     octant records, row values).
#include <math.h>

#include "obte_internal.h"
#include "records.cuh"

namespace {

template <typename T>
struct AAView {
  static __device__ double* gd(const GeomDev& g, int s) { return g.aa_gd + (size_t)s * g.aa_nd; }
  static __device__ double* fd(const GeomDev& g, int s) { return g.aa_fd + (size_t)s * g.aa_nd; }
  static __device__ T* gt(const GeomDev& g, int s) {
    return reinterpret_cast<T*>(g.aa_gt) + (size_t)s * g.aa_nt;
  }
  static __device__ T* ft(const GeomDev& g, int s) {
    return reinterpret_cast<T*>(g.aa_ft) + (size_t)s * g.aa_nt;
  }
};

// 16-byte vectors of the sweep precision
template <typename T>
struct V16;
template <>
struct V16<float> {
  static constexpr int N = 4;
  using type = float4;
  static __device__ __forceinline__ void get(const float4& v, float* a) {
    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
  }
  static __device__ __forceinline__ float4 make(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }
};
template <>
struct V16<double> {
  static constexpr int N = 2;
  using type = double2;
  static __device__ __forceinline__ void get(const double2& v, double* a) {
    a[0] = v.x; a[1] = v.y;
  }
  static __device__ __forceinline__ double2 make(const double* a) { return make_double2(a[0], a[1]); }
};

__device__ __forceinline__ double state_d(const GeomDev& g, long i) {
  return i < g.n_cells ? g.TL[i] : g.Tw[i - g.n_cells];
}

template <typename T>
__global__ void aa_residual_kernel(const GeomDev* geoms) {
  const GeomDev g = geoms[blockIdx.y];
  if (g.aa_m <= 0 || *(volatile int*)g.done) return;
  const int S = g.aa_m + 1;            // history slots
  const int k = g.aa_k[0];             // Anderson step (0 = first sweep)
  const int cur = k % S;
  __shared__ double red[8][32];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  const int nvalid = k + 1 < S ? k + 1 : S;  // slots holding residuals after this step
  // FP64 part (T_L, T_w): few elements, FP64 products and sums
  double dots[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) dots[j] = 0.0;
  {
    const double* fdj[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) fdj[j] = AAView<T>::fd(g, (k - j + S * 8) % S);
    double* fcur = AAView<T>::fd(g, cur);
    double* gcur = AAView<T>::gd(g, cur);
    const double* X = g.aa_xcd;
    const long nd = g.aa_nd;
    for (long i = tid; i < nd; i += stride) {
      const double gv = state_d(g, i);
      const double f = gv - X[i];
      fcur[i] = f;
      gcur[i] = gv;
      dots[0] += f * f;
#pragma unroll
      for (int j = 1; j < 8; ++j)
        if (j < nvalid) dots[j] += f * fdj[j][i];
    }
  }
  // row values: products and the thread / warp sums in the sweep precision,
  // widened once per warp
  T tdots[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) tdots[j] = T(0);
  {
    const T* ftj[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) ftj[j] = AAView<T>::ft(g, (k - j + S * 8) % S);
    T* ftc = AAView<T>::ft(g, cur);
    T* gtc = AAView<T>::gt(g, cur);
    const T* X = reinterpret_cast<const T*>(g.aa_xct);
    const T* front = reinterpret_cast<const T*>(g.front);
    const long nt = g.aa_nt;
    constexpr int N = V16<T>::N;
    using VT = typename V16<T>::type;
    if (nt % N == 0) {
      const long nv = nt / N;
      for (long u = tid; u < nv; u += stride) {
        T gv[N], xv[N], f[N];
        V16<T>::get(reinterpret_cast<const VT*>(front)[u], gv);
        V16<T>::get(reinterpret_cast<const VT*>(X)[u], xv);
#pragma unroll
        for (int e = 0; e < N; ++e) {
          f[e] = gv[e] - xv[e];
          tdots[0] = fma(f[e], f[e], tdots[0]);
        }
        reinterpret_cast<VT*>(ftc)[u] = V16<T>::make(f);
        reinterpret_cast<VT*>(gtc)[u] = V16<T>::make(gv);
#pragma unroll
        for (int j = 1; j < 8; ++j)
          if (j < nvalid) {
            T fj[N];
            V16<T>::get(reinterpret_cast<const VT*>(ftj[j])[u], fj);
#pragma unroll
            for (int e = 0; e < N; ++e) tdots[j] = fma(f[e], fj[e], tdots[j]);
          }
      }
    } else {
      for (long i = tid; i < nt; i += stride) {
        const T gv = front[i];
        const T f = gv - X[i];
        ftc[i] = f;
        gtc[i] = gv;
        tdots[0] = fma(f, f, tdots[0]);
#pragma unroll
        for (int j = 1; j < 8; ++j)
          if (j < nvalid) tdots[j] = fma(f, ftj[j][i], tdots[j]);
      }
    }
  }
  const unsigned FULL = 0xffffffffu;
  const bool any_d = __any_sync(FULL, (long)(tid - (threadIdx.x & 31)) < g.aa_nd);
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

// After aa_residual_kernel, one block of 8 warps per geometry: warp j sums
// dot j over the block partials; warp 0 then updates the Gram matrix, solves
// for gamma and writes the mixing coefficients; the step counter advances
// (aa_k[1] keeps the step being mixed).
__global__ void aa_solve_kernel(const GeomDev* geoms, int nblocks) {
  const GeomDev g = geoms[blockIdx.x];
  if (g.aa_m <= 0 || *(volatile int*)g.done) return;
  __shared__ double dv[8];
  const unsigned FULL = 0xffffffffu;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double v = 0.0;
  for (int b = lane; b < nblocks; b += 32) v += g.blk_part[(size_t)b * 8 + w];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  if (lane == 0) dv[w] = v;
  __syncthreads();
  if (w != 0) return;
  const int S = g.aa_m + 1;
  const int k = g.aa_k[0];
  const int cur = k % S;
  const int nvalid = k + 1 < S ? k + 1 : S;
  double* gram = g.aa_gram;  // [S][S] by slot
  if (lane < nvalid) {
    const int sl = (k - lane + S * 8) % S;
    gram[cur * S + sl] = dv[lane];
    gram[sl * S + cur] = dv[lane];
  }
  __syncwarp();
  // logical order oldest .. newest: slot(l) = (k - mk + l) mod S
  const int mk = nvalid - 1;  // number of differences
  auto G = [&](int l1, int l2) {
    const int s1 = (k - mk + l1 + S * 8) % S, s2 = (k - mk + l2 + S * 8) % S;
    return gram[s1 * S + s2];
  };
  // lane i < mk holds row i of the normal equations A gamma = b, with
  // A_ij = (f_{i+1} - f_i).(f_{j+1} - f_j), b_i = (f_{i+1} - f_i).f_mk
  double row[7], rhs = 0.0, diag = 0.0;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    row[j] = (lane < mk && j < mk) ? G(lane + 1, j + 1) - G(lane + 1, j) - G(lane, j + 1) + G(lane, j) : 0.0;
    if (j == lane) diag = row[j];
  }
  if (lane < mk) rhs = G(lane + 1, mk) - G(lane, mk);
  double tr = diag;
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(FULL, tr, o);
#pragma unroll
  for (int j = 0; j < 7; ++j)
    if (j == lane) row[j] += 1e-12 * tr + 1e-300;
  bool ok = mk > 0;
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    if (c >= mk || !ok) break;
    // partial pivoting: the row of largest |A_rc| among r >= c
    double a = (lane >= c && lane < mk) ? fabs(row[c]) : -1.0;
    int p = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const double a2 = __shfl_xor_sync(FULL, a, o);
      const int p2 = __shfl_xor_sync(FULL, p, o);
      if (a2 > a || (a2 == a && p2 < p)) {
        a = a2;
        p = p2;
      }
    }
    if (!(a > 0.0)) {
      ok = false;
      break;
    }
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const double rc = __shfl_sync(FULL, row[j], c), rp = __shfl_sync(FULL, row[j], p);
      if (lane == c) row[j] = rp;
      else if (lane == p) row[j] = rc;
    }
    {
      const double bc = __shfl_sync(FULL, rhs, c), bp = __shfl_sync(FULL, rhs, p);
      if (lane == c) rhs = bp;
      else if (lane == p) rhs = bc;
    }
    double piv[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) piv[j] = __shfl_sync(FULL, row[j], c);
    const double pb = __shfl_sync(FULL, rhs, c);
    if (lane > c && lane < mk) {
      const double f = row[c] / piv[c];
#pragma unroll
      for (int j = 0; j < 7; ++j)
        if (j >= c) row[j] -= f * piv[j];
      rhs -= f * pb;
    }
  }
  double gam[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) gam[j] = 0.0;
#pragma unroll
  for (int c = 6; c >= 0; --c) {
    if (c >= mk || !ok) continue;
    double xc = (lane == c) ? rhs / row[c] : 0.0;
    xc = __shfl_sync(FULL, xc, c);
    if (!isfinite(xc)) ok = false;
    gam[c] = xc;
    if (lane < c) rhs -= row[c] * xc;
  }
  if (lane != 0) return;
  // x_{k+1} = G_mk - sum_i gamma_i (G_{i+1} - G_i); plain step if the solve failed
  double coef[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) coef[l] = (l == mk) ? 1.0 : 0.0;
  if (ok) {
#pragma unroll
    for (int i = 0; i < 7; ++i)
      if (i < mk) {
        coef[i + 1] -= gam[i];
        coef[i] += gam[i];
      }
  }
#pragma unroll
  for (int l = 0; l < 8; ++l) g.aa_coef[l] = coef[l];
  g.aa_k[1] = k;
  g.aa_k[0] = k + 1;
}

// x_{k+1} = sum_l coef_l G_l over the window; written to the state, to X, and
// to the sweep inputs (s T_L, wall temperatures, records, row values).
template <typename T>
__global__ void aa_mix_kernel(const GeomDev* geoms) {
  const GeomDev g = geoms[blockIdx.y];
  if (g.aa_m <= 0 || *(volatile int*)g.done) return;
  const int S = g.aa_m + 1;
  const int k = g.aa_k[1];  // the step being mixed
  const int nvalid = k + 1 < S ? k + 1 : S;
  const int mk = nvalid - 1;
  double c[8];
  T ct[8];
  const double* gdl[8];
  const T* gtl[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    c[l] = l <= mk ? g.aa_coef[l] : 0.0;
    ct[l] = (T)c[l];
    const int sl = (k - mk + l + S * 8) % S;
    gdl[l] = AAView<T>::gd(g, sl);
    gtl[l] = AAView<T>::gt(g, sl);
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  T* src = reinterpret_cast<T*>(g.src);
  T* twc = reinterpret_cast<T*>(g.twc);
  double* Xd = g.aa_xcd;
  // deviation form: the records' difference fields are rebuilt from the
  // mixed T_L and T_w by psi_records_kernel after this kernel
  const bool recs = g.rec4 != nullptr && !g.psi;
  for (long i = tid; i < g.aa_nd; i += stride) {
    double v = 0.0;
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (l <= mk) v += c[l] * gdl[l][i];
    if (i < g.n_cells) {
      if (!(g.code[i] & CODE_SOLID)) v = 0.0;
      g.TL[i] = v;
      const T sv = (T)(g.s ? g.s[i] * v : v);
      src[i] = sv;
      if (recs && g.tlq) {  // 2D warp kernel: records at the skewed index of each quadrant
        const int nx = g.nx, ny = g.ny;
        const int x = (int)i % nx, y = (int)i / nx;
        T* rec = reinterpret_cast<T*>(g.rec4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int ip = (q & 1) ? nx - 1 - x : x;
          const int jp = (q & 2) ? ny - 1 - y : y;
          rec[(((size_t)q * nx + (ip + jp) % nx) * ny + jp) * 4] = sv;
        }
      } else if (recs) {
        obte::rec_put_src<T>(g, (int)i, sv);
      }
    } else {
      const long f = i - g.n_cells;
      g.Tw[f] = v;
      const int cell = g.wall_cell[f], sd = g.wall_side[f];
      twc[(size_t)cell * 6 + sd] = (T)v;
      if (recs) obte::rec_put_wall<T>(g, cell, sd, (T)v);
    }
    Xd[i] = v;
  }
  // row values in the sweep precision
  T* front = reinterpret_cast<T*>(g.front);
  T* Xt = reinterpret_cast<T*>(g.aa_xct);
  const long nt = g.aa_nt;
  constexpr int N = V16<T>::N;
  using VT = typename V16<T>::type;
  if (nt % N == 0) {
    const long nv = nt / N;
    for (long u = tid; u < nv; u += stride) {
      T acc[N];
#pragma unroll
      for (int e = 0; e < N; ++e) acc[e] = T(0);
#pragma unroll
      for (int l = 0; l < 8; ++l)
        if (l <= mk) {
          T gl[N];
          V16<T>::get(reinterpret_cast<const VT*>(gtl[l])[u], gl);
#pragma unroll
          for (int e = 0; e < N; ++e) acc[e] = fma(ct[l], gl[e], acc[e]);
        }
      reinterpret_cast<VT*>(front)[u] = V16<T>::make(acc);
      reinterpret_cast<VT*>(Xt)[u] = V16<T>::make(acc);
    }
  } else {
    for (long i = tid; i < nt; i += stride) {
      T v = T(0);
#pragma unroll
      for (int l = 0; l < 8; ++l)
        if (l <= mk) v = fma(ct[l], gtl[l][i], v);
      front[i] = v;
      Xt[i] = v;
    }
  }
}

// X <- the state at iteration 0; step counter 0
template <typename T>
__global__ void aa_init_kernel(const GeomDev* geoms) {
  const GeomDev& g = geoms[blockIdx.y];
  if (g.aa_m <= 0) return;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  for (long i = tid; i < g.aa_nd; i += stride) g.aa_xcd[i] = state_d(g, i);
  T* xt = reinterpret_cast<T*>(g.aa_xct);
  const T* front = reinterpret_cast<const T*>(g.front);
  for (long i = tid; i < g.aa_nt; i += stride) xt[i] = front[i];
  if (tid == 0) {
    g.aa_k[0] = 0;
    g.aa_k[1] = 0;
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
  return cudaGetLastError();
}

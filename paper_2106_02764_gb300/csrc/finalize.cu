// Per-iteration finalisation (FP64): new lattice and wall temperatures,
// kappa_eff, convergence test; state initialisation from the Fourier guess;
// gauge and gradient contraction for the outputs.
#include <math.h>

#include <algorithm>

#include "obte_internal.h"
#include "records.cuh"

namespace {

// block sum (valid in thread 0); every thread of the block calls it
__device__ double obte_block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (lane < nw) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

// T_L <- sum_o a_o T_o (E2), T_w <- wall numerator / denominator (E3), the
// sweep inputs derived from them, and each block's max |dT_L| into its
// partial slot.  Grid: x = blocks per geometry, y = geometry.
template <typename T>
__global__ void finalize_kernel(const GeomDev* geoms) {
  const GeomDev g = geoms[blockIdx.y];
  if (*(volatile int*)g.done) return;
  __shared__ double red[32];
  double dmax = 0.0;
  int nonfin = 0;
  T* src = reinterpret_cast<T*>(g.src);
  const int n_cells = g.n_cells;
  double* __restrict__ TL = g.TL;
  double* __restrict__ TL_acc = g.TL_acc;
  const uint8_t* __restrict__ code = g.code;
  const double* __restrict__ sv = g.s;
  const bool recs = g.rec4 != nullptr;
  const int stride = gridDim.x * blockDim.x;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += stride) {
    if (!(code[c] & CODE_SOLID)) continue;
    double t = 0.0;
    size_t k[4];  // 2D warp kernel: skewed index of the cell in each quadrant
    if (g.tlq3) {  // skewed per-octant partials of the 3D kernel (fixed order)
      double p[8];
      int k3[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        k3[q] = g.rec_idx[(size_t)c * 8 + q];
        p[q] = g.tlq3[k3[q]];
      }
      t = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
      // (the skewed partials are zeroed by tlq_zero_kernel, in their own order)
    } else if (!g.tlq) {  // per-cell accumulator
      t = TL_acc[c];
      TL_acc[c] = 0.0;
    } else {  // skewed per-quadrant partials of the 2D warp kernel
      const int nx = g.nx, ny = g.ny;
      const int x = c % nx, y = c / nx;
      double p[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // all loads first: the zeroing stores come after
        const int ip = (q & 1) ? nx - 1 - x : x;
        const int jp = (q & 2) ? ny - 1 - y : y;
        k[q] = ((size_t)q * nx + (ip + jp) % nx) * ny + jp;
        p[q] = g.tlq[k[q]];
      }
      t += (p[0] + p[1]) + (p[2] + p[3]);
    }
    if (g.psi) {
      // deviation form: the accumulators hold sums of psi = T_o - T_L, so
      // T_L_new = T_L + sum_o a_o psi_o and T_w = T_L,cell + num_psi / den;
      // the cell's walls are done here, while T_L,cell is still the old one
      const double told = TL[c];
      t += told;
      const uint32_t cd = code[c];
      T* twc = reinterpret_cast<T*>(g.twc);
#pragma unroll
      for (int sd = 0; sd < 6; ++sd)
        if (cd & (1u << sd)) {
          const int f = g.wall_id[(size_t)c * 6 + sd];
          const size_t k = (size_t)c * 6 + sd;
          const double w = told + g.wall_acc[k] / g.wall_den[f];
          g.wall_acc[k] = 0.0;
          if (!isfinite(w)) nonfin = 1;
          g.Tw[f] = w;
          twc[k] = (T)w;
        }
    }
    if (!isfinite(t)) nonfin = 1;
    dmax = fmax(dmax, fabs(t - TL[c]));
    TL[c] = t;
    const T v = (T)(sv ? sv[c] * t : t);
    src[c] = v;
    if (recs && !g.psi) {  // deviation form: the records are rebuilt by psi_records_kernel
      if (g.tlq) {  // the records of the 2D warp kernel share the skewed index
        T* rec = reinterpret_cast<T*>(g.rec4);
#pragma unroll
        for (int q = 0; q < 4; ++q) rec[k[q] * 4] = v;
      } else {
        obte::rec_put_src<T>(g, c, v);
      }
    }
  }
  T* twc = reinterpret_cast<T*>(g.twc);
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < (g.psi ? 0 : g.n_walls); f += stride) {
    const int c = g.wall_cell[f], sd = g.wall_side[f];
    const size_t k = (size_t)c * 6 + sd;
    const double w = g.wall_acc[k] / g.wall_den[f];
    g.wall_acc[k] = 0.0;
    if (!isfinite(w)) nonfin = 1;
    g.Tw[f] = w;
    twc[k] = (T)w;
    if (recs) obte::rec_put_wall<T>(g, c, sd, (T)w);
  }
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dmax;
  if (nonfin) atomicOr(g.nonfinite, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) m = fmax(m, red[w]);
    g.blk_part[blockIdx.x] = m;
  }
}

// After finalize_kernel: the skewed T_L partials it read go back to zero in
// their own (coalesced) order; zeroing them per cell in the finalisation
// scatters one 32-byte sector per value (config 2: 13 us of a 0.10 ms
// finalisation, Anderson and records step).  Grid: x = blocks, y = geometry.
__global__ void tlq_zero_kernel(const GeomDev* geoms) {
  const GeomDev& g = geoms[blockIdx.y];
  double* q = g.tlq ? g.tlq : g.tlq3;
  if (!q) return;
  const long n = (long)g.n_cells * (g.tlq ? 4 : 8);
  const long n2 = n / 2;  // double2 stores (the arrays are 16-byte aligned)
  double2* q2 = reinterpret_cast<double2*>(q);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n2; i += (long)gridDim.x * blockDim.x)
    q2[i] = make_double2(0.0, 0.0);
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) q[n - 1] = 0.0;
}

// After finalize_kernel (one warp per geometry): max |dT_L| over the block
// partials, kappa from the hot-face flux, and the stopping test of
// Algorithm 1.
__global__ void finalize_tail_kernel(const GeomDev* geoms, int nblocks) {
  const GeomDev g = geoms[blockIdx.x];
  if (*(volatile int*)g.done) return;
  double m = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) m = fmax(m, g.blk_part[b]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x != 0) return;
  const double delta = m;
  // deviation form: the sweeps summed psi = T_o - T_L; the T_L part of the
  // hot-face flux is K+ S+ + K- S- over the T_L that sweep used
  const double phi_tl = g.psi ? g.kx_pos * g.hot_tl[0] + g.kx_neg * g.hot_tl[1] : 0.0;
  const double kappa = g.kappa_scale * (*g.phi_acc + phi_tl);
  *g.phi_acc = 0.0;
  const int n = *g.iter + 1;
  *g.iter = n;
  if (n - 1 < g.max_hist) g.kappa_hist[n - 1] = kappa;
  const double prevk = (n >= 2 && n - 2 < g.max_hist) ? g.kappa_hist[n - 2] : NAN;
  g.delta_max[1] = delta;   // last iteration's max |dT_L|, for the host
  bool conv = n >= 2 && n >= g.min_iter;
  if (g.tol > 0.0) conv = conv && fabs(kappa - prevk) <= g.tol * fabs(kappa);
  if (g.tol_TL > 0.0) conv = conv && delta <= g.tol_TL;
  if (g.tol <= 0.0 && g.tol_TL <= 0.0) conv = false;
  int done = 0;
  if (*(volatile int*)g.nonfinite || !isfinite(kappa)) done = 3;
  else if (conv) done = 1;
  else if (n >= g.max_iter) done = 2;
  if (done) *(volatile int*)g.done = done;
}

// State at iteration 0 from a full-grid temperature T0 (the Fourier guess):
// T_L, the sweep source, wall temperatures (their cell's value) and the row
// values carried into the first sweep (the value of the cell each row visits
// last, for every ordinate's octant).
// Grid: x = blocks per geometry, y = geometry.
template <typename T>
__global__ void init_state_kernel(const GeomDev* geoms) {
  const GeomDev& g = geoms[blockIdx.y];
  const double* T0 = g.T0;
  const int* octant_of = g.octant_of;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  T* src = reinterpret_cast<T*>(g.src);
  for (int c = tid; c < g.n_cells; c += stride) {
    const bool solid = g.code[c] & CODE_SOLID;
    const double t = solid ? T0[c] : 0.0;
    g.TL[c] = t;
    g.TL_acc[c] = 0.0;
    src[c] = (T)(g.s ? g.s[c] * t : t);
  }
  T* twc = reinterpret_cast<T*>(g.twc);
  for (long i = tid; i < (long)g.n_cells * 6; i += stride) twc[i] = T(0);
  for (int f = tid; f < g.n_walls; f += stride) {
    g.Tw[f] = T0[g.wall_cell[f]];
    g.wall_acc[(size_t)g.wall_cell[f] * 6 + g.wall_side[f]] = 0.0;
  }
  T* front = reinterpret_cast<T*>(g.front);
  const long total = (long)g.n_ord * g.rows;
  for (long i = tid; i < total; i += stride) {
    const int o = (int)(i / g.rows);
    const int row = (int)(i % g.rows);
    const int jp = row % g.ny, kp = row / g.ny;
    const int oc = octant_of[o];
    // the column the row visits last: step nx-1 of the group's wavefront
    const int ip = ((g.nx - 1 + g.ord_d0[o] - jp - (g.dim == 3 ? kp : 0)) % g.nx + g.nx) % g.nx;
    const int x = (oc & 1) ? g.nx - 1 - ip : ip;
    const int y = (oc & 2) ? g.ny - 1 - jp : jp;
    const int z = (g.dim == 3) ? ((oc & 4) ? g.nz - 1 - kp : kp) : 0;
    const int c = x + g.nx * (y + g.ny * z);
    // deviation form: psi = T_o - T_L = 0 on the starting guess
    front[i] = (T)((g.code[c] & CODE_SOLID) && !g.psi ? T0[c] : 0.0);
  }
  if (tid == 0) {
    *g.phi_acc = 0.0;
    g.delta_max[0] = 0.0;
    g.delta_max[1] = 0.0;
    *g.iter = 0;
    *g.done = 0;
    *g.nonfinite = 0;
  }
}

// out[c] = T_L[c] - mean over solid cells (NaN in pores); one block.
__global__ void gauge_kernel(const uint8_t* code, const double* TL, int n, double* out,
                             double* mean_out) {
  __shared__ double red[64];
  __shared__ double s_mean;
  double s = 0.0, k = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    if (code[c] & CODE_SOLID) {
      s += TL[c];
      k += 1.0;
    }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    k += __shfl_xor_sync(0xffffffffu, k, o);
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[w] = s;
    red[32 + w] = k;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nw; ++i) {
      a += red[i];
      b += red[32 + i];
    }
    s_mean = b > 0 ? a / b : 0.0;
    if (mean_out) *mean_out = s_mean;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    out[c] = (code[c] & CODE_SOLID) ? TL[c] - s_mean : NAN;
}

// grad[c] -= jscale * sum_{o in [o0, o1)} a_o T_rev(o)[c] (T_o[c] - T_L[c])
// over recorded fields rec[(o - o0) * n + c]; rev_local maps o - o0 to the
// record slot of the reversed ordinate.  The reversed field is the adjoint
// field of o (see obte_kappa_grad_s).
// With psi the recorded fields are deviations T_o - T_L (deviation-form
// sweeps): then T_o - T_L is the record itself and T_rev = record + T_L.
// Block: 32 consecutive cells (x) times GC_SLICES slices of the records (y);
// each thread takes every GC_SLICES-th record k of its cell (coalesced loads
// across the warp) whose reverse comes later, and adds the terms of both
// ordinates of the pair from the two loaded fields; the slices are added in
// shared memory in a fixed order.  Deviation-form (FP32) records: products
// and the thread's sum in FP32 (the fields themselves are FP32), widened
// once per thread.
constexpr int GC_SLICES = 8;

template <typename T>
__global__ void __launch_bounds__(32 * GC_SLICES) grad_contract_kernel(
    const uint8_t* code, const double* TL, int n, const T* rec, int n_rec, const int* rev_local,
    const double* a_rec, double jscale, double* grad, int psi) {
  __shared__ double part[GC_SLICES][32];
  const int c = blockIdx.x * 32 + threadIdx.x;
  double acc = 0.0;
  if (c < n && (code[c] & CODE_SOLID)) {
    const double tl = TL[c];
    if (sizeof(T) == 4 && psi) {
      const float tlf = (float)tl;
      float accf = 0.f;
      for (int k = threadIdx.y; k < n_rec; k += GC_SLICES) {
        const int rk = rev_local[k];
        if (rk < k) continue;  // the pair's terms were added at rk
        const float f = (float)rec[(size_t)k * n + c];
        if (rk == k) {
          accf = fmaf((float)a_rec[k] * (f + tlf), f, accf);
          continue;
        }
        const float b = (float)rec[(size_t)rk * n + c];
        accf = fmaf((float)a_rec[k] * (b + tlf), f, accf);
        accf = fmaf((float)a_rec[rk] * (f + tlf), b, accf);
      }
      acc = (double)accf;
    } else {
      for (int k = threadIdx.y; k < n_rec; k += GC_SLICES) {
        const int rk = rev_local[k];
        if (rk < k) continue;
        const double f = (double)rec[(size_t)k * n + c];
        const double b = rk == k ? f : (double)rec[(size_t)rk * n + c];
        acc += psi ? a_rec[k] * (b + tl) * f : a_rec[k] * b * (f - tl);
        if (rk != k) acc += psi ? a_rec[rk] * (f + tl) * b : a_rec[rk] * f * (b - tl);
      }
    }
  }
  part[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && c < n && (code[c] & CODE_SOLID)) {
    double t = 0.0;
#pragma unroll
    for (int y = 0; y < GC_SLICES; ++y) t += part[y][threadIdx.x];
    grad[c] -= jscale * t;
  }
}

// Deviation form: each solid cell's record fields 1 .. dim of every octant
// hold the upwind value across that octant's upwind side minus the cell's
// T_L, formed in FP64: T_w - T_L at a wall, otherwise the neighbour's T_L
// (across the x period: +dT at the low side, -dT at the high side) minus the
// cell's.  Grid: x = blocks per geometry, y = geometry.
template <typename T>
__global__ void psi_records_kernel(const GeomDev* geoms) {
  const GeomDev& g = geoms[blockIdx.y];
  if (!g.psi || !g.rec4) return;
  if (blockIdx.x == 0) {
    // S+, S-: T_L at the two ends of the solid-solid faces of the plane x = 0
    // (fixed order: a block sum), for the tail's kappa of the next sweep
    __shared__ double red[32];
    double sp = 0.0, sm = 0.0;
    for (int row = threadIdx.x; row < g.rows; row += blockDim.x) {
      const int c0 = g.nx * row, c1 = c0 + g.nx - 1;
      if ((g.code[c1] & CODE_SOLID) && !(g.code[c1] & CODE_WALL_XP)) {
        sp += g.TL[c1];
        sm += g.TL[c0];
      }
    }
    sp = obte_block_sum(sp, red);
    sm = obte_block_sum(sm, red);
    if (threadIdx.x == 0) {
      g.hot_tl[0] = sp;
      g.hot_tl[1] = sm;
    }
  }
  T* rec = reinterpret_cast<T*>(g.rec4);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nq = g.dim == 3 ? 8 : 4;
  const double* TL = g.TL;
  const int stride = gridDim.x * blockDim.x;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.n_cells; c += stride) {
    const uint32_t cd = g.code[c];
    if (!(cd & CODE_SOLID)) continue;
    const int x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
    const double tl = TL[c];
    auto side = [&](int sd, int nb, double jump) -> double {
      if (cd & (1u << sd)) return g.Tw[g.wall_id[(size_t)c * 6 + sd]] - tl;
      return TL[nb] + jump - tl;
    };
    const int row = nx * (y + ny * z);
    double d[6];
    d[0] = side(0, (x == 0 ? nx - 1 : x - 1) + row, x == 0 ? g.dT : 0.0);
    d[1] = side(1, (x == nx - 1 ? 0 : x + 1) + row, x == nx - 1 ? -g.dT : 0.0);
    d[2] = side(2, x + nx * ((y == 0 ? ny - 1 : y - 1) + ny * z), 0.0);
    d[3] = side(3, x + nx * ((y == ny - 1 ? 0 : y + 1) + ny * z), 0.0);
    d[4] = d[5] = 0.0;
    if (g.dim == 3) {
      d[4] = side(4, x + nx * (y + ny * (z == 0 ? nz - 1 : z - 1)), 0.0);
      d[5] = side(5, x + nx * (y + ny * (z == nz - 1 ? 0 : z + 1)), 0.0);
    }
    for (int q = 0; q < nq; ++q) {
      T* r = rec + (size_t)g.rec_w * g.rec_idx[(size_t)c * nq + q];
      // octant bit a set: p_a < 0, the upwind side is the + side
      r[1] = (T)d[(q & 1) ? 1 : 0];
      r[2] = (T)d[(q & 2) ? 3 : 2];
      if (g.rec_w == 8) r[3] = (T)d[(q & 4) ? 5 : 4];
    }
  }
}

// Skewed per-octant cell records of the 2D warp and 3D kernels (layout in
// obte_internal.h): source, wall temperatures through the upwind sides, packed
// cell index and octant flags; and each cell's record index per octant, by
// which the finalisation and the Anderson step keep the records current.
template <typename T>
__global__ void build_records_kernel(const GeomDev* geoms) {
  const GeomDev& g = geoms[blockIdx.y];
  if (!g.rec4) return;
  const T* src = reinterpret_cast<const T*>(g.src);
  const T* twc = reinterpret_cast<const T*>(g.twc);
  T* rec = reinterpret_cast<T*>(g.rec4);
  const int stride = gridDim.x * blockDim.x;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.n_cells; c += stride) {
    const int x = c % g.nx, y = (c / g.nx) % g.ny, z = c / (g.nx * g.ny);
    const uint32_t code = g.code[c];
    const int nq = g.dim == 3 ? 8 : 4;
    for (int q = 0; q < nq; ++q) {
      const int ip = (q & 1) ? g.nx - 1 - x : x;
      const int jp = (q & 2) ? g.ny - 1 - y : y;
      const int kp = (q & 4) ? g.nz - 1 - z : z;
      const size_t k = ((size_t)q * g.nx + (ip + jp + kp) % g.nx) * g.rows + jp + (size_t)g.ny * kp;
      g.rec_idx[(size_t)c * nq + q] = (int)k;
      const uint32_t in_x = (q & 1) ? CODE_WALL_XP : CODE_WALL_XM;
      const uint32_t in_y = (q & 2) ? CODE_WALL_YP : CODE_WALL_YM;
      const uint32_t in_z = (q & 4) ? CODE_WALL_ZP : CODE_WALL_ZM;
      const uint32_t out_x = (q & 1) ? CODE_WALL_XM : CODE_WALL_XP;
      const uint32_t out_y = (q & 2) ? CODE_WALL_YM : CODE_WALL_YP;
      const uint32_t out_z = (q & 4) ? CODE_WALL_ZM : CODE_WALL_ZP;
      uint32_t packed = (uint32_t)c;
      if (code & in_x) packed |= REC_WIN_X;
      if (code & in_y) packed |= REC_WIN_Y;
      if (g.dim == 3 && (code & in_z)) packed |= REC_WIN_Z;
      if (ip == 0 && !(code & in_x)) packed |= REC_JUMP;
      if (code & CODE_SOLID) packed |= REC_SOLID;
      if (code & out_x) packed |= REC_WOUT_X;
      if (code & out_y) packed |= REC_WOUT_Y;
      if (g.dim == 3 && (code & out_z)) packed |= REC_WOUT_Z;
      if (ip == 0) packed |= REC_FIRST;
      if (ip == g.nx - 1) packed |= REC_LAST;
      T* r = rec + (size_t)g.rec_w * k;
      const T pk = sizeof(T) == 4 ? (T)__uint_as_float(packed) : (T)__longlong_as_double((long long)packed);
      // deviation form (3D): field 0 holds the packed word too (no source
      // field is read), so one 16-byte load gives the packed word and the
      // three wall / difference fields
      r[0] = (g.psi && g.rec_w == 8) ? pk : src[c];
      // x field: the upwind wall temperature, or +-dT on the jump column
      r[1] = (packed & REC_JUMP) ? (T)((q & 1) ? -g.dT : g.dT) : twc[(size_t)c * 6 + ((q & 1) ? 1 : 0)];
      r[2] = twc[(size_t)c * 6 + ((q & 2) ? 3 : 2)];
      if (g.rec_w == 4) {
        r[3] = pk;
      } else {
        r[3] = twc[(size_t)c * 6 + ((q & 4) ? 5 : 4)];
        r[4] = pk;
        r[5] = T(0);
        r[6] = T(0);
        r[7] = T(0);
      }
    }
  }
}

// Ordinate sharding (Sec. 3: directions spread over processors; the only
// exchange per iteration is a sum of the moment partials).  Export: the
// moment partials of the sweep that just ran over this context's share of the
// ordinates, in one compact FP64 vector
//   out[c]                   T_L numerator sum_o a_o T_o of cell c (pores 0)
//   out[n_cells + f]         E3 numerator of wall face f
//   out[n_cells + n_walls]   hot-face flux
// with the accumulators zeroed behind them.  Import: the summed vector back
// into the accumulators (the T_L numerator into quadrant 0 of the skewed
// partials when the 2D warp kernel keeps them there), ready for the
// finalisation.  One geometry; grid-stride loops.
__device__ __forceinline__ size_t skew_index(const GeomDev& g, int c, int q) {
  const int x = c % g.nx, y = c / g.nx;
  const int ip = (q & 1) ? g.nx - 1 - x : x;
  const int jp = (q & 2) ? g.ny - 1 - y : y;
  return ((size_t)q * g.nx + (ip + jp) % g.nx) * g.ny + jp;
}

__global__ void shard_export_kernel(const GeomDev* geoms, double* out) {
  const GeomDev g = geoms[0];
  const int stride = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int c = tid; c < g.n_cells; c += stride) {
    double t = 0.0;
    if (g.tlq3) {
      double p[8];
      int k3[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        k3[q] = g.rec_idx[(size_t)c * 8 + q];
        p[q] = g.tlq3[k3[q]];
      }
      t = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
#pragma unroll
      for (int q = 0; q < 8; ++q) g.tlq3[k3[q]] = 0.0;
    } else if (!g.tlq) {
      t = g.TL_acc[c];
      g.TL_acc[c] = 0.0;
    } else {
      size_t k[4];
      double p[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        k[q] = skew_index(g, c, q);
        p[q] = g.tlq[k[q]];
      }
      t = (p[0] + p[1]) + (p[2] + p[3]);
#pragma unroll
      for (int q = 0; q < 4; ++q) g.tlq[k[q]] = 0.0;
    }
    out[c] = (g.code[c] & CODE_SOLID) ? t : 0.0;
  }
  for (int f = tid; f < g.n_walls; f += stride) {
    const size_t k = (size_t)g.wall_cell[f] * 6 + g.wall_side[f];
    out[g.n_cells + f] = g.wall_acc[k];
    g.wall_acc[k] = 0.0;
  }
  if (tid == 0) {
    out[g.n_cells + g.n_walls] = *g.phi_acc;
    *g.phi_acc = 0.0;
  }
}

__global__ void shard_import_kernel(const GeomDev* geoms, const double* in) {
  const GeomDev g = geoms[0];
  if (*(volatile int*)g.done) return;
  const int stride = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int c = tid; c < g.n_cells; c += stride) {
    if (g.tlq3) g.tlq3[g.rec_idx[(size_t)c * 8]] = in[c];
    else if (g.tlq) g.tlq[skew_index(g, c, 0)] = in[c];
    else g.TL_acc[c] = in[c];
  }
  for (int f = tid; f < g.n_walls; f += stride)
    g.wall_acc[(size_t)g.wall_cell[f] * 6 + g.wall_side[f]] = in[g.n_cells + f];
  if (tid == 0) *g.phi_acc = in[g.n_cells + g.n_walls];
}

}  // namespace

cudaError_t launch_shard_export(const GeomDev* geoms_dev, double* out, int blocks, cudaStream_t st) {
  shard_export_kernel<<<blocks, 256, 0, st>>>(geoms_dev, out);
  return cudaGetLastError();
}

cudaError_t launch_shard_import(const GeomDev* geoms_dev, const double* in, int blocks,
                                cudaStream_t st) {
  shard_import_kernel<<<blocks, 256, 0, st>>>(geoms_dev, in);
  return cudaGetLastError();
}

cudaError_t launch_build_records(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                                 cudaStream_t st) {
  dim3 grid(blocks, n_geoms);
  if (precision == 0) build_records_kernel<double><<<grid, 256, 0, st>>>(geoms_dev);
  else build_records_kernel<float><<<grid, 256, 0, st>>>(geoms_dev);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                            cudaStream_t st) {
  if (blocks > kMaxPartBlocks) return cudaErrorInvalidValue;
  dim3 grid(blocks, n_geoms);
  if (precision == 0) finalize_kernel<double><<<grid, 256, 0, st>>>(geoms_dev);
  else finalize_kernel<float><<<grid, 256, 0, st>>>(geoms_dev);
  tlq_zero_kernel<<<grid, 256, 0, st>>>(geoms_dev);
  finalize_tail_kernel<<<n_geoms, 32, 0, st>>>(geoms_dev, blocks);
  return cudaGetLastError();
}

template <typename T>
__global__ void init_twc_kernel(const GeomDev* geoms) {
  const GeomDev& g = geoms[blockIdx.y];
  T* twc = reinterpret_cast<T*>(g.twc);
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < g.n_walls; f += gridDim.x * blockDim.x)
    twc[(size_t)g.wall_cell[f] * 6 + g.wall_side[f]] = (T)g.Tw[f];
}

cudaError_t launch_init_state(const GeomDev* geoms_dev, int n_geoms, long max_work, int max_walls,
                              int precision, cudaStream_t st) {
  const dim3 grid((unsigned)std::max<long>(1, std::min<long>((max_work + 255) / 256, 4096)),
                  (unsigned)n_geoms);
  const dim3 wgrid((unsigned)std::max(1, std::min((max_walls + 255) / 256, 1024)), (unsigned)n_geoms);
  if (precision == 0) {
    init_state_kernel<double><<<grid, 256, 0, st>>>(geoms_dev);
    init_twc_kernel<double><<<wgrid, 256, 0, st>>>(geoms_dev);
  } else {
    init_state_kernel<float><<<grid, 256, 0, st>>>(geoms_dev);
    init_twc_kernel<float><<<wgrid, 256, 0, st>>>(geoms_dev);
  }
  return cudaGetLastError();
}

cudaError_t launch_psi_records(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                               cudaStream_t st) {
  if (precision == 0) return cudaSuccess;  // FP64 sweeps carry T_o
  dim3 grid(blocks, n_geoms);
  psi_records_kernel<float><<<grid, 256, 0, st>>>(geoms_dev);
  return cudaGetLastError();
}

cudaError_t launch_gauge(const uint8_t* code, const double* TL, int n, double* out,
                         double* mean_out, cudaStream_t st) {
  gauge_kernel<<<1, 1024, 0, st>>>(code, TL, n, out, mean_out);
  return cudaGetLastError();
}

cudaError_t launch_grad_contract2(const uint8_t* code, const double* TL, int n, const void* rec,
                                  int n_rec, const int* rev_local, const double* a_rec,
                                  double jscale, double* grad, int precision, int psi,
                                  cudaStream_t st) {
  const int blocks = (n + 31) / 32;
  const dim3 thr(32, GC_SLICES);
  if (precision == 0)
    grad_contract_kernel<double><<<blocks, thr, 0, st>>>(code, TL, n, (const double*)rec, n_rec,
                                                         rev_local, a_rec, jscale, grad, psi);
  else
    grad_contract_kernel<float><<<blocks, thr, 0, st>>>(code, TL, n, (const float*)rec, n_rec,
                                                        rev_local, a_rec, jscale, grad, psi);
  return cudaGetLastError();
}

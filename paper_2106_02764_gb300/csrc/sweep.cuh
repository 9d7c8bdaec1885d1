// Upwind transport sweep of one ordinate group per thread block (Eq. iter2 of
// App. A, one source-iteration pass of Algorithm 1), with the moment
// reductions fused into the epilogue.
//
// Frame.  Every group holds ordinates of one octant (signs of p_x, p_y, p_z).
// Coordinates are mirrored per octant (i' = x or nx-1-x, ...) so that the
// upwind neighbours of cell (i', j', k') are always (i'-1, j', k'),
// (i', j'-1, k') and (i', j', k'-1).
//
// Wavefront.  Row (j', k') -- the line of cells along x -- visits column
//     i'(d) = (d + d0 - j' - k') mod nx        at step d = 0 .. nx-1,
// d0 being a per-group start offset.  The x neighbour of a cell was visited by
// the same row one step earlier (or, for the row's first column, in the
// previous iteration), and the y and z neighbours were visited by the rows
// below one step earlier (or in the previous iteration at d = 0).  The
// periodic wrap in x is therefore immediate except on one skewed cut per row,
// and the wrap in y (z) is immediate when ny (nz) is a multiple of nx.  Values
// that cross the cut come from the previous iteration: they are the row values
// left in `front` by the previous sweep.  Like the walls and T_L of Eq. iter2
// they are lagged; the fixed point is unchanged.  Every thread is busy at every
// step (no wavefront fill or drain), and groups of one octant start at
// different columns, so their moment atomics land on different cells.
//
// Threads.  Thread t owns R consecutive rows (R divides ny) j' = jb R ..
// jb R + R-1 of plane k' (jb = t mod tpp, k' = t / tpp) and keeps their values
// for all G ordinates of the group in registers.  Rows are updated top-down
// inside a step, so the row below still holds the previous step's value; only
// the lowest row needs the value of the thread below, exchanged through shared
// memory (2D); in 3D every row also needs the row of the plane below.  One
// barrier per step; the exchange buffers are double-buffered by step parity.
//
// Epilogue per solid cell (right-hand side of the next iteration, hot-contact
// flux of App. A):
//   T_L numerator   sum_g a_g T_g               -> FP64 atomic per cell
//   wall numerator  sum_g |K_g . n| T_g  (out-of-cell faces that are walls)
//   hot-face flux   sum_g K_gx (T_g + [p_x > 0] dT)  at the x = 0 plane
// The within-group sums run in the sweep precision (float in mixed mode) and
// are promoted to double once per cell per group.  The periodic jump term
// beta_x dT / (1 + D) is formed in double once per ordinate.
#pragma once

#include <stdint.h>

#include "obte_internal.h"

namespace obte {

template <typename T>
__device__ __forceinline__ T ld(const void* p, int i) {
  return __ldg(reinterpret_cast<const T*>(p) + i);
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Exact binary32 -> binary64 conversion by re-encoding the IEEE 754 fields on
// the integer pipe (sign kept, exponent re-biased by 1023 - 127, mantissa
// shifted into the wider field); Inf / NaN keep their class.  Zeros and
// subnormals (exponent field 0, magnitude below 1.2e-38, rare) take the
// hardware conversion, which is exact for them too.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t m = u & 0x7fffffu;
  uint32_t hi, lo;
  if (e == 0u) {
    if (m != 0u) return (double)f;
    hi = sign;
    lo = 0u;
  } else {
    const uint32_t ed = (e == 0xffu) ? 0x7ffu : e + 896u;
    hi = sign | (ed << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen(double d) { return d; }

__device__ __forceinline__ double block_sum(double v, double* red) {
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
  return s;  // valid in thread 0
}

// Rare per-cell work, kept out of the unrolled update so that the hot loop
// stays small: wall numerators, hot-face flux, and the flux / record passes.
// The cell's G values are read from the thread's scratch row in shared memory.
// Returns the hot-face flux contribution (added to the thread's phi).
template <typename T, int DIM, int G>
__device__ __noinline__ double cell_epilogue(const GeomDev& gm, const T* __restrict__ val,
                                             int cell, uint8_t code, int x, int ip, int o0,
                                             int cnt, int sx, int sy, int sz, int flags,
                                             double kx_sum) {
  const int nx = gm.nx;
  const double dT = gm.dT;
  const uint8_t out_x_bit = sx > 0 ? CODE_WALL_XP : CODE_WALL_XM;
  const uint8_t out_y_bit = sy > 0 ? CODE_WALL_YP : CODE_WALL_YM;
  const uint8_t out_z_bit = sz > 0 ? CODE_WALL_ZP : CODE_WALL_ZM;
  const int out_x_side = sx > 0 ? 1 : 0;
  const int out_y_side = sy > 0 ? 3 : 2;
  const int out_z_side = sz > 0 ? 5 : 4;
  double sxk = 0.0, syk = 0.0, szk = 0.0;  // sum_g |K_ga| T_g
  for (int g = 0; g < cnt; ++g) {
    const double v = (double)val[g];
    sxk += (double)ld<T>(gm.kxa, o0 + g) * v;
    syk += (double)ld<T>(gm.kya, o0 + g) * v;
    if (DIM == 3) szk += (double)ld<T>(gm.kza, o0 + g) * v;
  }
  if (code & out_x_bit) atomicAdd(gm.wall_acc + cell * 6 + out_x_side, sxk);
  if (code & out_y_bit) atomicAdd(gm.wall_acc + cell * 6 + out_y_side, syk);
  if (DIM == 3 && (code & out_z_bit)) atomicAdd(gm.wall_acc + cell * 6 + out_z_side, szk);
  // the x = 0 plane is the out-of-cell x face of the last column i' = nx-1
  const bool hot = (ip == nx - 1) && !(code & out_x_bit);
  double phi = 0.0;
  if (hot) phi = (double)sx * sxk + (sx > 0 ? dT * kx_sum : 0.0);
  if (flags & SWEEP_FLUX) {
    atomicAdd(gm.J_acc + 3 * cell + 0, (double)sx * sxk);
    atomicAdd(gm.J_acc + 3 * cell + 1, (double)sy * syk);
    if (DIM == 3) atomicAdd(gm.J_acc + 3 * cell + 2, (double)sz * szk);
    if (!(code & out_x_bit)) {
      const int sec = sx > 0 ? (x + 1) % nx : x;
      const bool jmp = sx > 0 && x == nx - 1;
      atomicAdd(gm.phi_sec + sec, (double)sx * sxk + (jmp ? dT * kx_sum : 0.0));
    }
    if (hot)
      for (int g = 0; g < cnt; ++g) {
        const double k = (double)sx * (double)ld<T>(gm.kxa, o0 + g);
        atomicAdd(gm.phi_bin + gm.mbin[o0 + g], k * ((double)val[g] + (sx > 0 ? dT : 0.0)));
      }
  }
  if (flags & SWEEP_RECORD) {
    T* rec = reinterpret_cast<T*>(gm.rec);
    for (int g = 0; g < cnt; ++g) {
      const int sl = gm.rec_slot[o0 + g];
      if (sl >= 0) rec[(size_t)sl * gm.n_cells + cell] = val[g];
    }
  }
  return phi;
}

template <typename T, int DIM, int G, int RMAX, bool HAS_S>
__global__ void __launch_bounds__((DIM == 3 && RMAX < 8) ? 512 : 256, 1) sweep_kernel(const SweepLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int s_item;
  const int nthr = blockDim.x;
  const int t = threadIdx.x;
  T* xtop = reinterpret_cast<T*>(smem_raw);               // [2][nthr][G]
  T* scratch = xtop + 2 * nthr * G;                        // [nthr][G]
  T* xall = scratch + nthr * G;                            // [2][nthr][RMAX][G]  (DIM == 3)
  const int flags = L.flags;
  const bool rare_pass = (flags & (SWEEP_FLUX | SWEEP_RECORD)) != 0;

  int item = blockIdx.x;
  for (;;) {
    if (L.item_counter) {
      __syncthreads();
      if (t == 0) s_item = atomicAdd(L.item_counter, 1);
      __syncthreads();
      item = s_item;
    }
    if (item >= L.n_items) return;
    const WorkItem wi = L.items[item];
    const GeomDev& gm = L.geoms[wi.geom];
    if (*(volatile const int*)gm.done) {
      if (!L.item_counter) return;
      continue;
    }
    const int nx = gm.nx, ny = gm.ny, nz = gm.nz, R = gm.R, tpp = gm.tpp;
    const int rows = gm.rows;
    const int sx = (wi.octant & 1) ? -1 : 1;
    const int sy = (wi.octant & 2) ? -1 : 1;
    const int sz = (wi.octant & 4) ? -1 : 1;
    const int o0 = wi.o0, cnt = wi.count, d0 = wi.d0;
    const double dT = gm.dT;
    const int jb = t % tpp, kp = t / tpp;
    const int j0 = jb * R;
    // the host picks R = RMAX dividing ny: a thread owns all RMAX rows or none
    const int nr = (kp < nz && j0 < ny) ? RMAX : 0;
    const uint8_t* __restrict__ codev = gm.code;
    const T* __restrict__ srcv = reinterpret_cast<const T*>(gm.src);
    const double* __restrict__ Twv = gm.Tw;
    const int* __restrict__ widv = gm.wall_id;
    const double* __restrict__ sv_ptr = gm.s;
    double* TLacc = gm.TL_acc;

    // per-ordinate coefficients.  HAS_S: A0 = D, AX = beta_x, ...; otherwise
    // premultiplied by 1/(1+D): A0 = 1/(1+D), AX = beta_x/(1+D), ...
    // JX = AX * (+-dT): the periodic jump term, formed in double.
    T A0[G], AX[G], AY[G], AZ[G], AW[G], JX[G];
    double kx_sum = 0.0;  // sum_g K_gx (signed), jump part of the hot-face flux
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const bool ok = g < cnt;
      const int o = o0 + (ok ? g : 0);
      const double a0 = ok ? (double)ld<T>(HAS_S ? gm.diag : gm.inv, o) : 0.0;
      double ax = ok ? (double)ld<T>(gm.bx, o) : 0.0;
      double ay = ok ? (double)ld<T>(gm.by, o) : 0.0;
      double az = (DIM == 3 && ok) ? (double)ld<T>(gm.bz, o) : 0.0;
      if (!HAS_S) {
        ax *= a0;
        ay *= a0;
        az *= a0;
      }
      A0[g] = (T)a0;
      AX[g] = (T)ax;
      AY[g] = (T)ay;
      AZ[g] = (T)az;
      AW[g] = ok ? ld<T>(gm.aw, o) : T(0);
      JX[g] = (T)(ax * (double)sx * dT);
      if (ok) kx_sum += (double)sx * (double)ld<T>(gm.kxa, o);
    }

    // row values carried from the previous iteration
    T v[RMAX][G];
    const T* front = reinterpret_cast<const T*>(gm.front);
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
#pragma unroll
      for (int g = 0; g < G; ++g)
        v[r][g] = (r < nr && g < cnt) ? front[(size_t)(o0 + g) * rows + (j0 + r) + ny * kp] : T(0);

    // publish as "step -1" (parity 1)
    if (nr > 0) {
#pragma unroll
      for (int g = 0; g < G; ++g) xtop[(1 * nthr + t) * G + g] = v[RMAX - 1][g];
      if (DIM == 3) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
#pragma unroll
          for (int g = 0; g < G; ++g) xall[((1 * nthr + t) * RMAX + r) * G + g] = v[r][g];
      }
    }
    __syncthreads();

    // neighbours in the exchange buffers
    int tb = -1;  // thread owning the row below row j0 (same plane)
    if (nr > 0) {
      if (jb > 0) tb = t - 1;
      else if (gm.py) tb = kp * tpp + (ny - 1) / R;
    }
    int tz = -1;  // thread owning the same rows in the plane below
    if (DIM == 3 && nr > 0) {
      if (kp > 0) tz = t - tpp;
      else if (gm.pz) tz = (nz - 1) * tpp + jb;
    }

    double phi = 0.0;
    const uint8_t in_x_bit = sx > 0 ? CODE_WALL_XM : CODE_WALL_XP;
    const uint8_t in_y_bit = sy > 0 ? CODE_WALL_YM : CODE_WALL_YP;
    const uint8_t in_z_bit = sz > 0 ? CODE_WALL_ZM : CODE_WALL_ZP;
    const uint8_t out_wall_bits = (uint8_t)((sx > 0 ? CODE_WALL_XP : CODE_WALL_XM) |
                                            (sy > 0 ? CODE_WALL_YP : CODE_WALL_YM) |
                                            (DIM == 3 ? (sz > 0 ? CODE_WALL_ZP : CODE_WALL_ZM) : 0));
    const int in_x_side = sx > 0 ? 0 : 1;
    const int in_y_side = sy > 0 ? 2 : 3;
    const int in_z_side = sz > 0 ? 4 : 5;

    for (int d = 0; d < nx; ++d) {
      const int cur = d & 1, prv = cur ^ 1;
      T dn0[G];
#pragma unroll
      for (int g = 0; g < G; ++g) dn0[g] = (tb >= 0) ? xtop[(prv * nthr + tb) * G + g] : T(0);
#pragma unroll
      for (int rr = 0; rr < RMAX; ++rr) {
        const int r = RMAX - 1 - rr;
        if (r < nr) {
          const int jp = j0 + r;
          const int ip = pmod(d + d0 - jp - (DIM == 3 ? kp : 0), nx);
          const int x = sx > 0 ? ip : nx - 1 - ip;
          const int y = sy > 0 ? jp : ny - 1 - jp;
          const int z = (DIM == 3) ? (sz > 0 ? kp : nz - 1 - kp) : 0;
          const int cell = x + nx * (y + ny * z);
          const uint8_t code = __ldg(codev + cell);
          if (code & CODE_SOLID) {
            const T src = srcv[cell];
            // a wall upstream in x replaces the row's carried value
            if (code & in_x_bit) {
              const T w = (T)Twv[widv[cell * 6 + in_x_side]];
#pragma unroll
              for (int g = 0; g < G; ++g) v[r][g] = w;
            }
            const bool wy = code & in_y_bit;
            const T uyw = wy ? (T)Twv[widv[cell * 6 + in_y_side]] : T(0);
            bool wz = false;
            T uzw = T(0);
            if (DIM == 3) {
              wz = code & in_z_bit;
              if (wz) uzw = (T)Twv[widv[cell * 6 + in_z_side]];
            }
            const bool jump = (ip == 0) && !(code & in_x_bit);
            T sval = T(1);
            if (HAS_S) sval = (T)__ldg(sv_ptr + cell);
            T tl = T(0);
#pragma unroll
            for (int g = 0; g < G; ++g) {
              const T uy = wy ? uyw : (r > 0 ? v[r > 0 ? r - 1 : 0][g] : dn0[g]);
              const T jx = jump ? JX[g] : T(0);
              T acc;
              if (HAS_S) {
                acc = fma(AY[g], uy, src + jx);
                acc = fma(AX[g], v[r][g], acc);
              } else if (sizeof(T) == 4) {
                // delta form T = src + jx + sum_a A_a (u_a - src): the weight
                // of src is 1 - sum_a A_a exactly (float A_a)
                acc = fma(AY[g], uy - src, src + jx);
                acc = fma(AX[g], v[r][g] - src, acc);
              } else {
                acc = fma(AY[g], uy, fma(src, A0[g], jx));
                acc = fma(AX[g], v[r][g], acc);
              }
              if (DIM == 3) {
                const T uz = wz ? uzw : ((tz >= 0) ? xall[((prv * nthr + tz) * RMAX + r) * G + g] : T(0));
                acc = fma(AZ[g], (!HAS_S && sizeof(T) == 4) ? uz - src : uz, acc);
              }
              T val;
              if (HAS_S) {
                if (sizeof(T) == 4) val = (T)__fdividef((float)acc, (float)(sval + A0[g]));
                else val = acc / (sval + A0[g]);
              } else {
                val = acc;
              }
              v[r][g] = val;
              tl = fma(AW[g], val, tl);
            }
            atomicAdd(TLacc + cell, widen(tl));
            if ((code & out_wall_bits) || ip == nx - 1 || rare_pass) {
#pragma unroll
              for (int g = 0; g < G; ++g) scratch[t * G + g] = v[r][g];
              phi += cell_epilogue<T, DIM, G>(gm, scratch + t * G, cell, code, x, ip, o0, cnt, sx,
                                              sy, sz, flags, kx_sum);
            }
          }
        }
      }
      // publish this step's values
      if (nr > 0) {
#pragma unroll
        for (int g = 0; g < G; ++g) xtop[(cur * nthr + t) * G + g] = v[RMAX - 1][g];
        if (DIM == 3) {
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
#pragma unroll
            for (int g = 0; g < G; ++g) xall[((cur * nthr + t) * RMAX + r) * G + g] = v[r][g];
        }
      }
      __syncthreads();
    }

    // carry the row values to the next iteration
    T* frontw = reinterpret_cast<T*>(gm.front);
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (r < nr && g < cnt) frontw[(size_t)(o0 + g) * rows + (j0 + r) + ny * kp] = v[r][g];

    const double ps = block_sum(phi, red);
    if (t == 0 && ps != 0.0) atomicAdd(gm.phi_acc, ps);
    if (!L.item_counter) return;
  }
}

}  // namespace obte

// Upwind transport sweep of one ordinate group per thread block (Eq. iter2 of
// App. A, one source-iteration pass of Algorithm 1), with the moment
// reductions fused into the epilogue.
//
// Frame.  Every group holds ordinates of one octant (signs of p_x, p_y, p_z).
// Coordinates are mirrored per octant (i' = x or nx-1-x, ...) so that the
// upwind neighbours of cell (i', j', k') are always (i'-1, j', k'),
// (i', j'-1, k') and (i', j', k'-1).
//
// Wavefront.  Row (j', k') -- the line of cells along x -- processes column
//     i'(d) = (d - j' - k') mod nx        at step d = 0 .. nx-1.
// The x neighbour of a cell was processed by the same row one step earlier
// (or, for the first column visited, in the previous iteration), and the y
// and z neighbours were processed by the rows below one step earlier (or in
// the previous iteration at d = 0).  The periodic wrap in x is therefore
// immediate everywhere except on one skewed cut per row, and the wrap in y
// (z) is immediate when ny (nz) is a multiple of nx.  Values that cross the
// cut come from the previous iteration: they are the row values left in
// `front` by the previous sweep.  Like the walls and T_L of Eq. iter2 they are
// lagged; the fixed point is unchanged.  Every thread is busy at every step
// (no wavefront fill or drain).
//
// Threads.  Thread t owns R consecutive rows (R divides ny) j' = jb R .. jb R + R-1 of plane
// k' (jb = t mod tpp, k' = t / tpp) and keeps their values for all G
// ordinates of the group in registers.  Rows are updated top-down inside a
// step, so the row below still holds the previous step's value; only the
// lowest row needs the value of the thread below, exchanged through shared
// memory (2D), and in 3D every row needs the row of the plane below.  One
// barrier per step; the exchange buffers are double-buffered by step parity.
//
// Epilogue per solid cell (Eq. iter2 right-hand side of the next iteration,
// hot-contact flux of App. A):
//   T_L numerator   sum_g a_g T_g               -> FP64 atomic per cell
//   wall numerator  sum_g |K_g . n| T_g  (out-of-cell faces that are walls)
//   hot-face flux   sum_g K_gx (T_g + [p_x > 0] dT)  at the x = 0 plane
// The within-group sums run in the sweep precision (float in mixed mode) and
// are promoted to double once per cell per group.
#pragma once

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

template <typename T, int DIM, int G, int RMAX>
__global__ void __launch_bounds__(DIM == 3 ? 512 : 256) sweep_kernel(const SweepLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int s_item;
  const int nthr = blockDim.x;
  const int t = threadIdx.x;
  T* xtop = reinterpret_cast<T*>(smem_raw);  // [2][nthr][G]
  T* xall = xtop + 2 * nthr * G;             // [2][nthr][RMAX][G]   (DIM == 3)
  const bool has_s = (L.flags & SWEEP_HAS_S) != 0;
  const bool flux = (L.flags & SWEEP_FLUX) != 0;
  const bool record = (L.flags & SWEEP_RECORD) != 0;

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
    const int o0 = wi.o0, cnt = wi.count;
    const double dT = gm.dT;
    const int jb = t % tpp, kp = t / tpp;
    const int j0 = jb * R;
    // the host picks R = RMAX dividing ny: a thread owns all RMAX rows or none
    const int nr = (kp < nz && j0 < ny) ? RMAX : 0;

    // per-ordinate coefficients.  no s: A0 = 1/(1+D), AX = beta_x/(1+D), ...
    // with s: A0 = D, AX = beta_x, ...  (premultiplied tables vs raw tables)
    T A0[G], AX[G], AY[G], AZ[G], AW[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const bool ok = g < cnt;
      const int o = o0 + (ok ? g : 0);
      A0[g] = ok ? ld<T>(has_s ? gm.diag : gm.inv, o) : T(0);
      AX[g] = ok ? ld<T>(gm.bx, o) : T(0);
      AY[g] = ok ? ld<T>(gm.by, o) : T(0);
      AZ[g] = (DIM == 3 && ok) ? ld<T>(gm.bz, o) : T(0);
      AW[g] = ok ? ld<T>(gm.aw, o) : T(0);
      if (ok && !has_s) {  // premultiply by 1 / (1 + D)
        AX[g] *= A0[g];
        AY[g] *= A0[g];
        AZ[g] *= A0[g];
      }
    }
    double kx_sum = 0.0;  // sum_g K_gx (signed), for the jump part of the hot-face flux
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < cnt) kx_sum += (double)sx * (double)ld<T>(gm.kxa, o0 + g);

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
    const uint8_t out_x_bit = sx > 0 ? CODE_WALL_XP : CODE_WALL_XM;
    const uint8_t in_y_bit = sy > 0 ? CODE_WALL_YM : CODE_WALL_YP;
    const uint8_t out_y_bit = sy > 0 ? CODE_WALL_YP : CODE_WALL_YM;
    const uint8_t in_z_bit = sz > 0 ? CODE_WALL_ZM : CODE_WALL_ZP;
    const uint8_t out_z_bit = sz > 0 ? CODE_WALL_ZP : CODE_WALL_ZM;
    const int in_x_side = sx > 0 ? 0 : 1, out_x_side = 1 - in_x_side;
    const int in_y_side = sy > 0 ? 2 : 3, out_y_side = 5 - in_y_side;
    const int in_z_side = sz > 0 ? 4 : 5, out_z_side = 9 - in_z_side;
    const T* srcv = reinterpret_cast<const T*>(gm.src);

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
        const int ip = pmod(d - jp - (DIM == 3 ? kp : 0), nx);
        const int x = sx > 0 ? ip : nx - 1 - ip;
        const int y = sy > 0 ? jp : ny - 1 - jp;
        const int z = (DIM == 3) ? (sz > 0 ? kp : nz - 1 - kp) : 0;
        const int cell = x + nx * (y + ny * z);
        const uint8_t code = __ldg(gm.code + cell);
        if (code & CODE_SOLID) {
        const T src = srcv[cell];
        const bool wx = code & in_x_bit, wy = code & in_y_bit;
        const bool wz = (DIM == 3) && (code & in_z_bit);
        const T uxw = wx ? (T)gm.Tw[gm.wall_id[cell * 6 + in_x_side]] : T(0);
        const T uyw = wy ? (T)gm.Tw[gm.wall_id[cell * 6 + in_y_side]] : T(0);
        const T uzw = wz ? (T)gm.Tw[gm.wall_id[cell * 6 + in_z_side]] : T(0);
        const bool jump = (ip == 0) && !wx;
        const double jdt = (double)sx * dT;
        const T sv = has_s ? (T)__ldg(gm.s + cell) : T(1);
        T tl = T(0);
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const T ux = wx ? uxw : v[r][g];
          T uy;
          if (wy) uy = uyw;
          else if (r > 0) uy = v[r > 0 ? r - 1 : 0][g];
          else uy = dn0[g];
          T base;
          if (!has_s) {
            base = jump ? (T)((double)src * (double)A0[g] + (double)AX[g] * jdt) : src * A0[g];
          } else {
            base = jump ? (T)((double)src + (double)AX[g] * jdt) : src;
          }
          T acc = fma(AX[g], ux, fma(AY[g], uy, base));
          if (DIM == 3) {
            const T uz = wz ? uzw : ((tz >= 0) ? xall[((prv * nthr + tz) * RMAX + r) * G + g] : T(0));
            acc = fma(AZ[g], uz, acc);
          }
          const T val = has_s ? acc / (sv + A0[g]) : acc;
          v[r][g] = val;
          tl = fma(AW[g], val, tl);
        }
        atomicAdd(gm.TL_acc + cell, (double)tl);

        // walls the group's ordinates leave into
        if (code & out_x_bit) {
          T s = T(0);
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (g < cnt) s = fma(ld<T>(gm.kxa, o0 + g), v[r][g], s);
          atomicAdd(gm.wall_acc + gm.wall_id[cell * 6 + out_x_side], (double)s);
        }
        if (code & out_y_bit) {
          T s = T(0);
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (g < cnt) s = fma(ld<T>(gm.kya, o0 + g), v[r][g], s);
          atomicAdd(gm.wall_acc + gm.wall_id[cell * 6 + out_y_side], (double)s);
        }
        if (DIM == 3 && (code & out_z_bit)) {
          T s = T(0);
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (g < cnt) s = fma(ld<T>(gm.kza, o0 + g), v[r][g], s);
          atomicAdd(gm.wall_acc + gm.wall_id[cell * 6 + out_z_side], (double)s);
        }
        // hot-contact face: the x = 0 plane is the out-of-cell x face of i' = nx-1
        const bool hot = (ip == nx - 1) && !(code & out_x_bit);
        if (hot) {
          T s = T(0);
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (g < cnt) s = fma(ld<T>(gm.kxa, o0 + g), v[r][g], s);
          phi += (double)sx * (double)s + (sx > 0 ? dT * kx_sum : 0.0);
        }
        if (flux) {
          T jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
          for (int g = 0; g < G; ++g) {
            if (g < cnt) {
              jx = fma(ld<T>(gm.kxa, o0 + g), v[r][g], jx);
              jy = fma(ld<T>(gm.kya, o0 + g), v[r][g], jy);
              if (DIM == 3) jz = fma(ld<T>(gm.kza, o0 + g), v[r][g], jz);
            }
          }
          atomicAdd(gm.J_acc + 3 * cell + 0, (double)sx * (double)jx);
          atomicAdd(gm.J_acc + 3 * cell + 1, (double)sy * (double)jy);
          if (DIM == 3) atomicAdd(gm.J_acc + 3 * cell + 2, (double)sz * (double)jz);
          if (!(code & out_x_bit)) {
            const int sec = sx > 0 ? (x + 1) % nx : x;
            const bool jmp = sx > 0 && x == nx - 1;
            atomicAdd(gm.phi_sec + sec, (double)sx * (double)jx + (jmp ? dT * kx_sum : 0.0));
          }
          if (hot) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
              if (g < cnt) {
                const double k = (double)sx * (double)ld<T>(gm.kxa, o0 + g);
                atomicAdd(gm.phi_bin + gm.mbin[o0 + g], k * ((double)v[r][g] + (sx > 0 ? dT : 0.0)));
              }
            }
          }
        }
        if (record) {
          T* rec = reinterpret_cast<T*>(gm.rec);
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int sl = (g < cnt) ? __ldg(gm.rec_slot + o0 + g) : -1;
            if (sl >= 0) rec[(size_t)sl * gm.n_cells + cell] = v[r][g];
          }
        }
        }  // solid
        }  // r < nr
      }
      // publish this step's values
      if (nr > 0) {
#pragma unroll
        for (int g = 0; g < G; ++g) xtop[(cur * nthr + t) * G + g] = v[RMAX - 1][g];
        if (DIM == 3) {
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
            if (r < nr)
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

// 3D upwind transport sweep, one ordinate group per thread block (Eq. iter2 of
// App. A, one source-iteration pass of Algorithm 1), moments fused.
//
// Wavefront as in sweep.cuh: in the frame mirrored per octant, row (j', k')
// visits column i' = (d + d0 - j' - k') mod nx at step d; the x neighbour is
// the row's own previous value, the y and z neighbours are the rows below one
// step earlier.  Thread t owns R consecutive rows j' of plane k' = t / tpp and
// keeps their values for the G ordinates of the group in registers; rows are
// updated top-down inside a step, so the row below in y still holds its
// previous-step value.  At the end of every step each thread publishes its
// R x G values to shared memory, laid out [row][ordinate][thread] so that
// neighbouring threads touch neighbouring banks; after one barrier the thread
// above in z (and, for the lowest row, the thread above in y) reads them.
//
// Data layout.  All cells visited at step d lie on one diagonal
// s = (i' + j' + k') mod nx = (d + d0) mod nx of the octant frame, so the
// finalisation stores every cell's record {s T_L, T_w through the upwind x,
// y and z sides, packed cell / code / column flags} per octant at
// [s][j' + ny k']: a thread's rows of one step are contiguous records, copied
// one step ahead (FP32: by cp.async into shared memory, FP64: loaded into
// registers).  The T_L moment goes by row through shared memory into a skewed
// per-octant FP64 accumulator.
//
// FP32 groups run in deviation form like the 2D warp kernel (sweep2d.cuh):
// row values psi = T_o - T_L, record fields holding the upwind value minus
// the cell's T_L, moments of psi, T_L added back in FP64; their records keep
// the packed word in field 0, so a row's record is one 16-byte copy, which
// each thread makes for its own rows one step ahead into shared memory
// (config 3: 3.01 ms per launch with a 16-byte plus a 4-byte load held one
// step ahead in registers, 2.41 with one 16-byte load, 2.17 with the copies
// and the skewed T_L accumulator).
//
// Cells update branch-free (pore values never reach a solid cell, whose faces
// towards a pore are walls); atomics and the rare epilogue (walls the
// ordinates leave into, the hot-contact column, flux / record passes; sums in
// the sweep precision, widened exactly) are predicated on solid cells.
#pragma once

#include <type_traits>

#include "sweep.cuh"

namespace obte {

__device__ __forceinline__ void cp16_3d(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void commit_3d() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait_3d() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T>
__device__ __forceinline__ uint32_t rec3_bits(T v);
template <>
__device__ __forceinline__ uint32_t rec3_bits<float>(float v) { return __float_as_uint(v); }
template <>
__device__ __forceinline__ uint32_t rec3_bits<double>(double v) { return (uint32_t)__double_as_longlong(v); }

// Rare per-cell epilogue (3D); the cell's G values are at val[g * stride].
template <typename T, int G>
__device__ __noinline__ double cell_epilogue_3d(const GeomDev& gm, const T* val, int stride, int cell,
                                                uint32_t packed, bool last, int o0, int cnt, int sx,
                                                int sy, int sz, int flags, double kx_sum) {
  const int nx = gm.nx;
  const double dT = gm.dT;
  const bool out_x = packed & REC_WOUT_X, out_y = packed & REC_WOUT_Y, out_z = packed & REC_WOUT_Z;
  T sxk = T(0), syk = T(0), szk = T(0);
  for (int g = 0; g < cnt; ++g) {
    const T v = val[g * stride];
    sxk = fma(ld<T>(gm.kxa, o0 + g), v, sxk);
    syk = fma(ld<T>(gm.kya, o0 + g), v, syk);
    szk = fma(ld<T>(gm.kza, o0 + g), v, szk);
  }
  const double dx = widen(sxk), dy = widen(syk), dz = widen(szk);
  if (out_x) atomicAdd(gm.wall_acc + cell * 6 + (sx > 0 ? 1 : 0), dx);
  if (out_y) atomicAdd(gm.wall_acc + cell * 6 + (sy > 0 ? 3 : 2), dy);
  if (out_z) atomicAdd(gm.wall_acc + cell * 6 + (sz > 0 ? 5 : 4), dz);
  // deviation form (FP32): every signed flux sum gains T_L sum_g K_g
  constexpr bool PSI = sizeof(T) == 4;
  const double tl = PSI ? gm.TL[cell] : 0.0;
  const bool hot = last && !out_x;
  double phi = 0.0;
  if (hot) phi = (sx > 0 ? dx : -dx) + (sx > 0 ? dT * kx_sum : 0.0) + tl * kx_sum;
  if (flags & SWEEP_FLUX) {
    const int x = cell % nx;
    double ky_sum = 0.0, kz_sum = 0.0;
    if (PSI)
      for (int g = 0; g < cnt; ++g) {
        ky_sum += (double)sy * (double)ld<T>(gm.kya, o0 + g);
        kz_sum += (double)sz * (double)ld<T>(gm.kza, o0 + g);
      }
    atomicAdd(gm.J_acc + 3 * cell + 0, (sx > 0 ? dx : -dx) + tl * kx_sum);
    atomicAdd(gm.J_acc + 3 * cell + 1, (sy > 0 ? dy : -dy) + tl * ky_sum);
    atomicAdd(gm.J_acc + 3 * cell + 2, (sz > 0 ? dz : -dz) + tl * kz_sum);
    if (!out_x) {
      const int sec = sx > 0 ? (x + 1) % nx : x;
      const bool jmp = sx > 0 && x == nx - 1;
      atomicAdd(gm.phi_sec + sec, (sx > 0 ? dx : -dx) + (jmp ? dT * kx_sum : 0.0) + tl * kx_sum);
    }
    if (hot)
      for (int g = 0; g < cnt; ++g) {
        const double k = (double)sx * (double)ld<T>(gm.kxa, o0 + g);
        atomicAdd(gm.phi_bin + gm.mbin[o0 + g],
                  k * ((double)val[g * stride] + tl + (sx > 0 ? dT : 0.0)));
      }
  }
  if (flags & SWEEP_RECORD) {
    T* rec = reinterpret_cast<T*>(gm.rec);
    for (int g = 0; g < cnt; ++g) {
      const int sl = gm.rec_slot[o0 + g];
      if (sl >= 0) rec[(size_t)sl * gm.n_cells + cell] = val[g * stride];
    }
  }
  return phi;
}

// threads per block the kernel is built for (the launch bound); the exchange
// buffers use it as a compile-time stride
template <int RMAX>
struct Sweep3DCfg {
  static constexpr int NT = RMAX >= 8 ? 256 : 512;
};

template <typename T, int G, int RMAX, bool HAS_S>
__global__ void __launch_bounds__(Sweep3DCfg<RMAX>::NT, 1) sweep3d_kernel(const SweepLaunch L) {
  constexpr int NT = Sweep3DCfg<RMAX>::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ __align__(16) T kcoef[3][G];  // |K_gx|, |K_gy|, |K_gz| of the group (rare path only)
  const int nthr = NT;
  const int t = threadIdx.x;
  T* scratch = reinterpret_cast<T*>(smem_raw) + 2 * RMAX * G * NT;  // [G][NT] after the exchange
  const int flags = L.flags;
  const bool rare_pass = (flags & (SWEEP_FLUX | SWEEP_RECORD)) != 0;
  // FP32 without s(x), G even: ordinates in pairs (float2) through the paired
  // FP32 instructions; the exchange buffer then holds pairs, [b][r][h][thread]
  constexpr bool X2 = sizeof(T) == 4 && !HAS_S && (G % 2 == 0);
  constexpr int GV = X2 ? G / 2 : G;
  using VV = typename std::conditional<X2, float2, T>::type;
  VV* xall2 = reinterpret_cast<VV*>(smem_raw);
  auto XP = [&](int b, int r, int h, int th) -> VV& { return xall2[((b * RMAX + r) * GV + h) * NT + th]; };

  const int item = blockIdx.x;
  if (item >= L.n_items) return;
  const WorkItem wi = L.items[item];
  const GeomDev& gm = L.geoms[wi.geom];
  if (*(volatile const int*)gm.done) return;
  const int nx = gm.nx, ny = gm.ny, nz = gm.nz, tpp = gm.tpp;
  const int rows = gm.rows;
  const int q = wi.octant & 7;
  const int sx = (q & 1) ? -1 : 1;
  const int sy = (q & 2) ? -1 : 1;
  const int sz = (q & 4) ? -1 : 1;
  const int o0 = wi.o0, cnt = wi.count, d0 = wi.d0;
  const double dT = gm.dT;
  const int jb = t % tpp, kp = t / tpp;
  const int j0 = jb * RMAX;
  const bool active = kp < nz;
  const int row0 = j0 + ny * kp;
  const T* __restrict__ recq = reinterpret_cast<const T*>(gm.rec4) + (size_t)q * nx * rows * 8;
  double* tl_acc = gm.TL_acc;
  const double* __restrict__ sv_ptr = gm.s;
  // T_L partials in the skewed order of the records ([s][row] of the
  // octant): a step's rows go through shared memory, by row, so that the
  // FP64 atomics of 32 consecutive rows are one coalesced request; they are
  // issued one step later, after the next step's rows
  double* tlq3 = gm.tlq3 ? gm.tlq3 + (size_t)q * nx * rows : nullptr;
  constexpr int NTR = NT * RMAX;  // rows of a block, at most
  T* tlb = scratch + G * NT;      // [2][NTR] after the scratch
  auto flush_rows = [&](int buf, int sd) {
    const T* b = tlb + buf * NTR;
    double* dst = tlq3 + (size_t)sd * rows;
    for (int row = t; row < rows; row += blockDim.x) {  // threads launched: a multiple of 32 <= NT
      const T v = b[row];
      if (v != T(0)) atomicAdd(dst + row, widen(v));
    }
  };

  T A0[G], AX[G], AY[G], AZ[G], AW[G], JX[G];
  double kx_sum = 0.0;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const bool ok = g < cnt;
    const int o = o0 + (ok ? g : 0);
    const double a0 = ok ? (double)ld<T>(HAS_S ? gm.diag : gm.inv, o) : 0.0;
    double ax = ok ? (double)ld<T>(gm.bx, o) : 0.0;
    double ay = ok ? (double)ld<T>(gm.by, o) : 0.0;
    double az = ok ? (double)ld<T>(gm.bz, o) : 0.0;
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

  if (t < G) {
    const bool ok = t < cnt;
    kcoef[0][t] = ok ? ld<T>(gm.kxa, o0 + t) : T(0);
    kcoef[1][t] = ok ? ld<T>(gm.kya, o0 + t) : T(0);
    kcoef[2][t] = ok ? ld<T>(gm.kza, o0 + t) : T(0);
  }
  const int out_side_x = sx > 0 ? 1 : 0, out_side_y = sy > 0 ? 3 : 2, out_side_z = sz > 0 ? 5 : 4;
  double* wacc = gm.wall_acc;

  VV v[RMAX][GV];
  auto VG = [&](int r, int g) -> T& {
    if constexpr (X2) return (g & 1) ? v[r][g >> 1].y : v[r][g >> 1].x;
    else return v[r][g];
  };
  VV AXv[GV], AYv[GV], AZv[GV], AWv[GV];
#pragma unroll
  for (int h = 0; h < GV; ++h) {
    if constexpr (X2) {
      AXv[h] = make_float2(AX[2 * h], AX[2 * h + 1]);
      AYv[h] = make_float2(AY[2 * h], AY[2 * h + 1]);
      AZv[h] = make_float2(AZ[2 * h], AZ[2 * h + 1]);
      AWv[h] = make_float2(AW[2 * h], AW[2 * h + 1]);
    }
  }
  const T* front = reinterpret_cast<const T*>(gm.front);
#pragma unroll
  for (int r = 0; r < RMAX; ++r)
#pragma unroll
    for (int g = 0; g < G; ++g)
      VG(r, g) = (active && g < cnt) ? front[(size_t)(o0 + g) * rows + row0 + r] : T(0);
#pragma unroll
  for (int r = 0; r < RMAX; ++r)
#pragma unroll
    for (int h = 0; h < GV; ++h) XP(1, r, h, t) = v[r][h];

  int tb = -1;  // thread owning the row below j0 (same plane)
  if (active) {
    if (jb > 0) tb = t - 1;
    else if (gm.py) tb = kp * tpp + (tpp - 1);
  }
  int tz = -1;  // thread owning the same rows in the plane below
  if (active) {
    if (kp > 0) tz = t - tpp;
    else if (gm.pz) tz = (nz - 1) * tpp + jb;
  }
  double phi = 0.0;
  // hot-face flux of the thread's rows, in the sweep precision (each row
  // crosses the hot column once per sweep), widened once at the end
  T hot_sum = T(0);
  int n_hot = 0;
  int s = d0;
  // Film walls beyond the last plane: every cell of plane nz - 1 leaves into
  // the wall, every step.  Their wall fluxes are taken one step late from the
  // published row values by ny helper threads (one row each) instead of by
  // the tpp threads of that plane (R rows each), which would pace the step.
  const bool defer_z = !rare_pass && !gm.pz && nz > 1;
  const bool z_owner = defer_z && kp == nz - 1;
  auto top_plane_walls = [&](int buf, int sd) {
    const int jj = t;  // row of plane nz - 1
    if (jj >= ny) return;
    const int th = (nz - 1) * tpp + jj / RMAX, r = jj % RMAX;
    const int row = jj + ny * (nz - 1);
    const uint32_t packed = rec3_bits<T>(__ldg(recq + ((size_t)sd * rows + row) * 8 + 4));
    if (!(packed & REC_SOLID) || !(packed & REC_WOUT_Z)) return;
    T sk;
    if constexpr (X2) {
      const float2* K2 = reinterpret_cast<const float2*>(kcoef[2]);
      float2 a = make_float2(0.f, 0.f), b = a;
#pragma unroll
      for (int h = 0; h < GV; ++h) {
        if (h & 1) b = __ffma2_rn(K2[h], XP(buf, r, h, th), b);
        else a = __ffma2_rn(K2[h], XP(buf, r, h, th), a);
      }
      sk = (a.x + b.x) + (a.y + b.y);
    } else {
      sk = T(0);
#pragma unroll
      for (int g = 0; g < G; ++g) sk = fma(kcoef[2][g], XP(buf, r, g, th), sk);
    }
    atomicAdd(wacc + (size_t)(packed & REC_CELL_MASK) * 6 + out_side_z, widen(sk));
  };

  // sum_g K_g T_g of register row r (wall and hot-face fluxes): paired FP32
  // products in two chains
  auto kdot = [&](const T* K, int r) -> T {
    if constexpr (X2) {
      const float2* K2 = reinterpret_cast<const float2*>(K);
      float2 a = make_float2(0.f, 0.f), b = a;
#pragma unroll
      for (int h = 0; h < GV; ++h) {
        if (h & 1) b = __ffma2_rn(K2[h], v[r][h], b);
        else a = __ffma2_rn(K2[h], v[r][h], a);
      }
      return (a.x + b.x) + (a.y + b.y);
    } else {
      T sk = T(0);
#pragma unroll
      for (int g = 0; g < G; ++g) sk = fma(K[g], VG(r, g), sk);
      return sk;
    }
  };
  // FP32: each thread copies its own rows' 16-byte records one step ahead
  // into shared memory ([buffer][row r][thread], conflict-free 16-byte
  // loads) and reads them back in the step; FP64 loads them into registers
  constexpr bool SREC = sizeof(T) == 4;
  float4* rsm = reinterpret_cast<float4*>(tlb + 2 * NTR);
  auto copy_recs = [&](int sd, int buf) {
    if (active)
#pragma unroll
      for (int r = 0; r < RMAX; ++r)
        cp16_3d(&rsm[(buf * RMAX + r) * NT + t], recq + ((size_t)sd * rows + row0 + r) * 8);
    commit_3d();
  };
  // records of the first step
  T rc[SREC ? 1 : RMAX][5];
  auto load_recs = [&](int sd, T (&dst)[SREC ? 1 : RMAX][5]) {
    if constexpr (!SREC) {
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (active) {
        const T* p = recq + ((size_t)sd * rows + row0 + r) * 8;
        if (sizeof(T) == 4) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(p));
          dst[r][0] = T(0);
          dst[r][1] = (T)a.y;
          dst[r][2] = (T)a.z;
          dst[r][3] = (T)a.w;
          dst[r][4] = (T)a.x;  // deviation form: the packed word sits in field 0
        } else {
          for (int f = 0; f < 5; ++f) dst[r][f] = __ldg(p + f);
        }
      } else {
        for (int f = 0; f < 5; ++f) dst[r][f] = T(0);
      }
    }
    }
  };
  if constexpr (SREC) copy_recs(s, 0);
  else load_recs(s, rc);
  __syncthreads();

  for (int d = 0; d < nx; ++d) {
    const int cur = d & 1, prv = cur ^ 1;
    const int s_next = (s + 1 == nx) ? 0 : s + 1;
    if constexpr (SREC) {
      if (d + 1 < nx) copy_recs(s_next, cur ^ 1);
      else commit_3d();
      wait_3d<1>();  // this step's records (this thread's own copies)
    }

    if (defer_z && d > 0) top_plane_walls(prv, s == 0 ? nx - 1 : s - 1);
    const int s_prev = s == 0 ? nx - 1 : s - 1;
    if (active) {
      VV dny[GV];
#pragma unroll
      for (int h = 0; h < GV; ++h) {
        if constexpr (X2) dny[h] = (tb >= 0) ? XP(prv, RMAX - 1, h, tb) : make_float2(0.f, 0.f);
        else dny[h] = (tb >= 0) ? XP(prv, RMAX - 1, h, tb) : T(0);
      }
      uint32_t pk[RMAX];
      T tls[RMAX];
      // branch-free update of all rows (top row first: the row below in y
      // still holds its previous value)
#pragma unroll
      for (int rr = 0; rr < RMAX; ++rr) {
        const int r = RMAX - 1 - rr;
        T src, twx, twy, twz;
        uint32_t packed;
        if constexpr (SREC) {
          const float4 a = rsm[(cur * RMAX + r) * NT + t];
          src = T(0);
          twx = (T)a.y;
          twy = (T)a.z;
          twz = (T)a.w;
          packed = __float_as_uint(a.x);  // deviation form: the packed word sits in field 0
        } else {
          src = rc[SREC ? 0 : r][0];
          twx = rc[SREC ? 0 : r][1];
          twy = rc[SREC ? 0 : r][2];
          twz = rc[SREC ? 0 : r][3];
          packed = rec3_bits<T>(rc[SREC ? 0 : r][4]);
        }
        const bool wx = packed & REC_WIN_X, wy = packed & REC_WIN_Y, wz = packed & REC_WIN_Z;
        const bool jump = packed & REC_JUMP;
        T sval = T(1);
        if (HAS_S) sval = (T)__ldg(sv_ptr + (packed & REC_CELL_MASK));
        if constexpr (X2) {
          // u = m T + t per direction: the upwind value, the wall
          // temperature (m = 0), or the value across the jump (the record's
          // x field holds +-dT on the jump column)
          // deviation form: u_a - T_L,cell = m_a psi_a + t_a (record fields
          // t_a: upwind T_L or T_w minus the cell's, the jump included);
          // psi = sum_a A_a (u_a - T_L), whose weight of T_L is exactly
          // 1 - sum_a A_a whatever the float rounding of the A_a
          const float mx = wx ? 0.f : 1.f, my = wy ? 0.f : 1.f, mz = wz ? 0.f : 1.f;
          const float2 mx2 = make_float2(mx, mx), tx2 = make_float2(twx, twx);
          const float2 my2 = make_float2(my, my), ty2 = make_float2(twy, twy);
          const float2 mz2 = make_float2(mz, mz), tz2 = make_float2(twz, twz);
          float2 tlp = make_float2(0.f, 0.f);
#pragma unroll
          for (int h = 0; h < GV; ++h) {
            const float2 ux = __ffma2_rn(mx2, v[r][h], tx2);  // u_x - T_L,cell
            const float2 ud = r > 0 ? v[r > 0 ? r - 1 : 0][h] : dny[h];
            const float2 uy = __ffma2_rn(my2, ud, ty2);
            const float2 uzv = (tz >= 0) ? XP(prv, r, h, tz) : make_float2(0.f, 0.f);
            const float2 uz = __ffma2_rn(mz2, uzv, tz2);
            float2 acc = __fmul2_rn(AXv[h], ux);
            acc = __ffma2_rn(AYv[h], uy, acc);
            acc = __ffma2_rn(AZv[h], uz, acc);
            v[r][h] = acc;
            tlp = __ffma2_rn(AWv[h], acc, tlp);
          }
          pk[r] = packed;
          tls[r] = tlp.x + tlp.y;
        } else {
        T tl = T(0), tl2 = T(0);
#pragma unroll
        for (int g = 0; g < G; ++g) {
          // FP32: deviation form (u_a - T_L = m_a psi_a + t_a); FP64: T_o,
          // the jump premultiplied (JX)
          constexpr bool PSI = sizeof(T) == 4;
          const T ub = r > 0 ? VG(r > 0 ? r - 1 : 0, g) : dny[g];
          const T uzb = (tz >= 0) ? XP(prv, r, g, tz) : T(0);
          const T ux = PSI ? (wx ? T(0) : VG(r, g)) + twx : (wx ? twx : VG(r, g));
          const T uy = PSI ? (wy ? T(0) : ub) + twy : (wy ? twy : ub);
          const T uz = PSI ? (wz ? T(0) : uzb) + twz : (wz ? twz : uzb);
          const T jx = (!PSI && jump) ? JX[g] : T(0);
          T acc;
          if (PSI) acc = T(0);
          else if (HAS_S) acc = src + jx;
          else acc = fma(src, A0[g], jx);
          acc = fma(AZ[g], uz, fma(AY[g], uy, fma(AX[g], ux, acc)));
          T val;
          if (HAS_S) {
            if (sizeof(T) == 4) val = (T)__fdividef((float)acc, (float)(sval + A0[g]));
            else val = acc / (sval + A0[g]);
          } else {
            val = acc;
          }
          VG(r, g) = val;
          if (g & 1) tl2 = fma(AW[g], val, tl2);
          else tl = fma(AW[g], val, tl);
        }
        pk[r] = packed;
        tls[r] = tl + tl2;
        }
      }
      uint32_t rare_mask = 0;
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        const bool rare =
            rare_pass || (pk[r] & (REC_WOUT_X | REC_WOUT_Y | (z_owner ? 0u : (uint32_t)REC_WOUT_Z) | REC_LAST));
        rare_mask |= (((pk[r] & REC_SOLID) && rare) ? 1u : 0u) << r;
      }
      // cells leaving into a wall, the hot-contact column, flux / record passes
      if (rare_mask) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
          if (!((rare_mask >> r) & 1u)) continue;
          const uint32_t packed = pk[r];
          const int cell = (int)(packed & REC_CELL_MASK);
          const bool last = packed & REC_LAST;
          if (rare_pass) {
#pragma unroll
            for (int g = 0; g < G; ++g) scratch[g * nthr + t] = VG(r, g);
            phi += cell_epilogue_3d<T, G>(gm, scratch + t, nthr, cell, packed, last, o0, cnt, sx,
                                          sy, sz, flags, kx_sum);
            continue;
          }
          if (packed & (REC_WOUT_X | REC_LAST)) {
            const T sk = kdot(kcoef[0], r);
            if (packed & REC_WOUT_X) {
              atomicAdd(wacc + (size_t)cell * 6 + out_side_x, widen(sk));
            } else {
              hot_sum += sk;
              ++n_hot;
            }
          }
          if (packed & REC_WOUT_Y) {
            const T sk = kdot(kcoef[1], r);
            atomicAdd(wacc + (size_t)cell * 6 + out_side_y, widen(sk));
          }
          if ((packed & REC_WOUT_Z) && !z_owner) {
            const T sk = kdot(kcoef[2], r);
            atomicAdd(wacc + (size_t)cell * 6 + out_side_z, widen(sk));
          }
        }
      }
      if (tlq3) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r) tlb[cur * NTR + row0 + r] = (pk[r] & REC_SOLID) ? tls[r] : T(0);
      } else {
        // moment atomics after all rows (a generic-address atomic between
        // rows would keep later shared-memory loads from moving ahead of it)
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (pk[r] & REC_SOLID) atomicAdd(tl_acc + (pk[r] & REC_CELL_MASK), widen(tls[r]));
      }
#pragma unroll
      for (int r = 0; r < RMAX; ++r)
#pragma unroll
        for (int h = 0; h < GV; ++h) XP(cur, r, h, t) = v[r][h];
    }
    // the previous step's partials (written before the barrier that ended it)
    if (tlq3 && d > 0) flush_rows(prv, s_prev);
    if constexpr (!SREC) {
      if (d + 1 < nx) load_recs(s_next, rc);
    }
    s = s_next;
    __syncthreads();
  }

  // the last step's plane nz - 1 (its values were published before the
  // loop's final barrier; s is one past the last diagonal) and its partials
  if (defer_z) top_plane_walls((nx - 1) & 1, s == 0 ? nx - 1 : s - 1);
  if (tlq3) flush_rows((nx - 1) & 1, s == 0 ? nx - 1 : s - 1);
  {
    const double dk = widen(hot_sum);
    phi += sx > 0 ? dk : -dk;
    if (sx > 0) phi += (double)n_hot * dT * kx_sum;
  }
  T* frontw = reinterpret_cast<T*>(gm.front);
#pragma unroll
  for (int r = 0; r < RMAX; ++r)
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (active && g < cnt) frontw[(size_t)(o0 + g) * rows + row0 + r] = VG(r, g);
  const double ps = block_sum(phi, red);
  if (t == 0 && ps != 0.0) atomicAdd(gm.phi_acc, ps);
}

}  // namespace obte

// 2D upwind transport sweep, one ordinate group per warp (Eq. iter2 of App. A,
// one source-iteration pass of Algorithm 1) with the moment reductions fused.
//
// Same wavefront as the block kernel (sweep.cuh): in the frame mirrored per
// quadrant, row j' visits column i'(d) = (d + d0 - j') mod nx at step d; the x
// neighbour is the row's own previous value and the y neighbour the row
// below's previous value.  A whole group lives in one warp: lane l owns R
// consecutive rows (ny / R <= 32 lanes in use), so the row below a lane's
// lowest row is the top row of lane l - 1 (lane tpp - 1 for lane 0 when y is
// periodic) and arrives by a warp shuffle.  No barrier: warps never wait for
// one another.
//
// Data layout.  All cells a warp visits at step d lie on one diagonal
// s = (i' + j') mod nx = (d + d0) mod nx of the quadrant frame.  Every cell
// has one record per quadrant (source s_i T_L,i, the wall temperatures seen
// through its upwind x and y sides, and a packed word with the cell index and
// the quadrant's wall / jump / column flags) at [s][j'], kept current by the
// finalisation, so a lane's R rows of one step are R contiguous records.  They are
// prefetched one step ahead with cp.async into lane-private shared memory.
// The T_L partials of a step go, transposed through shared memory, to skewed
// per-quadrant FP64 accumulators [s][j'], so that one atomic instruction of
// the warp covers 32 consecutive rows.
//
// Cells are updated branch-free (pores too: a pore's value is never read by a
// solid cell, whose faces towards a pore are walls); only the atomics and the
// rare epilogue (walls the ordinates leave into, the hot-contact column, flux /
// record passes) are predicated on the cell being solid.
//
// Precision.  FP32 groups run in deviation form: the row values are
// psi = T_o - T_L of the cell, the records' x / y fields hold the upwind
// value minus the cell's T_L (formed in FP64 by the finalisation), and
// psi = A_x (m_x psi_x + t_x) + A_y (m_y psi_y + t_y), with m = 0 and t the
// wall difference at a wall; the T_L, wall and flux moments are sums of psi,
// and the finalisation adds T_L back in FP64.  FP64 groups carry T_o.
//
// The R rows of a lane sit in the top R of RMAX register rows (slots
// RMAX - R .. RMAX - 1), so the lane's top row is always slot RMAX - 1; with
// RFIXED the host guarantees R == RMAX.
#pragma once

#include <type_traits>

#include "sweep.cuh"

namespace obte {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// the same with compile-time byte offsets on both addresses
template <int SOFF, int GOFF>
__device__ __forceinline__ void cp_async16_off(unsigned smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0+%2], [%1+%3], 16;\n" ::"r"(smem), "l"(gmem), "n"(SOFF),
               "n"(GOFF)
               : "memory");
}
// copies k = K .. KMAX-1 of a coalesced record run: part 32 k + lane, whose
// slot is the lane's offset for k mod KP shifted by 32 (k - k mod KP) / CH
template <int K, int KMAX, int KP, int CH>
struct CpRun {
  static __device__ __forceinline__ void go(const unsigned* pslot, unsigned boff, const char* gl) {
    if constexpr (K < KMAX) {
      cp_async16_off<(K / KP) * KP * 32 / CH * 16, K * 512>(pslot[K % KP] + boff, gl);
      CpRun<K + 1, KMAX, KP, CH>::go(pslot, boff, gl);
    }
  }
};
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint32_t rec_bits(float f) { return __float_as_uint(f); }
__device__ __forceinline__ uint32_t rec_bits(double d) { return (uint32_t)__double_as_longlong(d); }

// Rare per-cell epilogue of the warp kernel, in the sweep precision; sums are
// widened exactly before the FP64 atomics.  Returns the hot-face flux.
template <typename T, int G>
__device__ __noinline__ double cell_epilogue_2d(const GeomDev& gm, const T* __restrict__ val,
                                                int cell, uint32_t packed, bool last, int o0,
                                                int cnt, int sx, int sy, int flags,
                                                double kx_sum) {
  const int nx = gm.nx;
  const double dT = gm.dT;
  const bool out_x = packed & REC_WOUT_X, out_y = packed & REC_WOUT_Y;
  T sxk = T(0), syk = T(0);
  for (int g = 0; g < cnt; ++g) {
    sxk = fma(ld<T>(gm.kxa, o0 + g), val[g], sxk);
    syk = fma(ld<T>(gm.kya, o0 + g), val[g], syk);
  }
  const double dx = widen(sxk), dy = widen(syk);
  if (out_x) atomicAdd(gm.wall_acc + cell * 6 + (sx > 0 ? 1 : 0), dx);
  if (out_y) atomicAdd(gm.wall_acc + cell * 6 + (sy > 0 ? 3 : 2), dy);
  // deviation form (FP32): T_o = psi_o + T_L, so every signed flux sum gains
  // T_L sum_g K_g (kx_sum is sum_g sign(p_x) |K_gx|)
  constexpr bool PSI = sizeof(T) == 4;
  const double tl = PSI ? gm.TL[cell] : 0.0;
  const bool hot = last && !out_x;
  double phi = 0.0;
  if (hot) phi = (sx > 0 ? dx : -dx) + (sx > 0 ? dT * kx_sum : 0.0) + tl * kx_sum;
  if (flags & SWEEP_FLUX) {
    const int x = cell % nx;
    double ky_sum = 0.0;
    if (PSI)
      for (int g = 0; g < cnt; ++g) ky_sum += (double)sy * (double)ld<T>(gm.kya, o0 + g);
    atomicAdd(gm.J_acc + 3 * cell + 0, (sx > 0 ? dx : -dx) + tl * kx_sum);
    atomicAdd(gm.J_acc + 3 * cell + 1, (sy > 0 ? dy : -dy) + tl * ky_sum);
    if (!out_x) {
      const int sec = sx > 0 ? (x + 1) % nx : x;
      const bool jmp = sx > 0 && x == nx - 1;
      atomicAdd(gm.phi_sec + sec, (sx > 0 ? dx : -dx) + (jmp ? dT * kx_sum : 0.0) + tl * kx_sum);
    }
    if (hot)
      for (int g = 0; g < cnt; ++g) {
        const double k = (double)sx * (double)ld<T>(gm.kxa, o0 + g);
        atomicAdd(gm.phi_bin + gm.mbin[o0 + g], k * ((double)val[g] + tl + (sx > 0 ? dT : 0.0)));
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

// Warps per block (every warp owns its own staging buffers; static shared
// memory stays under 48 KB) and the resident blocks per SM the registers are
// budgeted for.  FP32 groups narrower than 8 ordinates hold fewer row values
// per lane and are built one warp per block with a register budget for 12
// (G = 6) or 15 (G = 4) resident warps per SM: more warps hide the latencies
// of a step, and single-warp blocks spread the groups evenly over the SMs.
// NST: record buffers per warp (copies run NST - 1 steps ahead).
// NH = 2: a group spans two warps (rows 0 .. 32 R - 1 and 32 R .. 64 R - 1),
// four groups of one octant and start column per block of eight warps, two
// blocks per SM under a 128-register budget: twice the resident warps of the
// one-warp form at the same ordinates per lane.
template <typename T, int G, int RMAX, int NH = 1>
struct WarpCfg {
  static constexpr bool NARROW = NH == 1 && sizeof(T) == 4 && G < 8 && RMAX >= 8;
  static constexpr int NST = 2;
  static constexpr int WPB = NH == 2 ? 8 : (NARROW ? 1 : ((sizeof(T) == 8 && RMAX >= 8) ? 2 : 4));
  static constexpr int MINB = NH == 2 ? 2 : (NARROW ? (G <= 4 ? 15 : 12) : ((G * (int)sizeof(T) <= 16) ? 4 : 1));
};

// Shared-memory slot of the record of (lane, register row r): each 16-byte
// part c of a record lives in plane c; inside a plane, lane l's rows occupy
// slots l*RMAX .. l*RMAX+RMAX-1 in an order permuted by an XOR of the lane's
// bits, so that the eight lanes of a quarter-warp reading the same r hit
// eight different 16-byte bank groups (the unpermuted layout puts them all
// on the same banks).
// Rows per lane that are not a power of two keep the plain order: for odd
// RMAX the eight lanes already fall on eight bank groups (RMAX l mod 8 is a
// permutation), and 6 leaves two-way conflicts.
template <int RMAX>
__device__ __forceinline__ int rec_slot(int lane, int r) {
  constexpr bool POW2 = (RMAX & (RMAX - 1)) == 0;
  constexpr int SH = RMAX >= 8 ? 0 : (RMAX == 4 ? 1 : (RMAX == 2 ? 2 : 0));
  constexpr int MSK = !POW2 ? 0 : (RMAX >= 8 ? 7 : RMAX - 1);
  return lane * RMAX + (r ^ ((lane >> SH) & MSK));
}

// PASS: a flux / record pass (flags SWEEP_FLUX or SWEEP_RECORD); the
// iteration sweeps are built without the out-of-line epilogue call, so no
// registers are saved around it in the hot loop.
// NH = 2 (RFIXED, FP32 without s(x), ny = 64 RMAX, one item per group, no
// work queue): warps w and w + 4 of a block hold the lower and upper half of
// group w's rows; the row below a half's lowest row comes from the other
// half's top row of the previous step through shared memory, across the
// block barrier every step ends with.  A block whose item list runs out
// keeps its warps in the loop on an empty item (no early exit before a
// barrier).
// Flux / record passes run once per solve or per gradient batch: their
// register budget is not cut for residency (a spilled pass costs more than
// the resident warps it would buy).
template <typename T, int G, int RMAX, bool HAS_S, bool RFIXED, bool PASS, int NH = 1>
__global__ void __launch_bounds__(32 * WarpCfg<T, G, RMAX, NH>::WPB,
                                  (PASS && NH == 1) ? 1 : WarpCfg<T, G, RMAX, NH>::MINB)
    sweep2d_warp_kernel(const SweepLaunch L) {
  constexpr int WPB = WarpCfg<T, G, RMAX, NH>::WPB;
  constexpr int CH = (4 * sizeof(T)) / 16;  // 16-byte parts per record
  constexpr int NST = WarpCfg<T, G, RMAX, NH>::NST;
  static_assert(NH == 1 || (RFIXED && sizeof(T) == 4 && !HAS_S && G % 2 == 0), "two-warp groups: FP32 pairs");
  __shared__ __align__(16) uint4 recbuf[WPB][NST][CH][32 * RMAX];
  // a cell's G values for the out-of-line epilogue (two-warp groups: a
  // thread-local array, which keeps the static shared memory under 48 KB)
  __shared__ __align__(16) T scratch_all[NH == 1 ? WPB : 1][32][G];
  __shared__ __align__(16) T kcoef[WPB][2][G];  // |K_gx|, |K_gy| of the warp's group (rare path only)
  // a step's T_L partials of every warp, by row (two step parities)
  __shared__ __align__(16) T tlbuf[2][WPB][32 * RMAX];
  // two-warp groups: top row of each half, by step parity
  __shared__ __align__(16) T xch[NH == 2 ? 2 : 1][4][2][G];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  T* scratch = &scratch_all[NH == 1 ? wib : 0][lane][0];
  const int flags = L.flags;
  constexpr bool rare_pass = PASS;
  const unsigned FULL = 0xffffffffu;
  const int gi = NH == 2 ? (wib & 3) : wib;    // group of the block
  const int half = NH == 2 ? (wib >> 2) : 0;   // half of the group's rows

  int item = NH == 2 ? blockIdx.x * 4 + gi : blockIdx.x * WPB + wib;
  for (;;) {
    if (L.item_counter) {
      int it = 0;
      if (lane == 0) it = atomicAdd(L.item_counter, 1);
      item = __shfl_sync(FULL, it, 0);
    }
    if (NH == 1 && item >= L.n_items) return;
    WorkItem wi = L.items[item < L.n_items ? item : 0];
    if (item >= L.n_items) wi.count = 0;  // (NH = 2) an empty group
    const GeomDev& gm = L.geoms[wi.geom];
    if (*(volatile const int*)gm.done) {
      if (!L.item_counter) return;
      continue;
    }
    const int nx = gm.nx, ny = gm.ny;
    const int R = RFIXED ? RMAX : gm.R;  // rows per lane, <= RMAX
    const int rb = RMAX - R;             // first register row in use
    const int tpp = gm.tpp;              // lanes in use
    const int q = wi.octant & 3;
    const int sx = (q & 1) ? -1 : 1;
    const int sy = (q & 2) ? -1 : 1;
    const int o0 = wi.o0, cnt = wi.count, d0 = wi.d0;
    const double dT = gm.dT;
    const bool active = NH == 2 || lane < tpp;
    const int jl = lane * R;                   // first row of the lane within the warp's rows
    const int rh = NH == 2 ? half * 32 * RMAX : 0;  // first row of the warp's rows
    const int j0 = rh + jl;
    const T* __restrict__ recq = reinterpret_cast<const T*>(gm.rec4) + (size_t)q * nx * ny * 4;
    double* tl_acc = gm.TL_acc;
    double* tlq = gm.tlq ? gm.tlq + (size_t)q * nx * ny : nullptr;
    const double* __restrict__ sv_ptr = gm.s;
    double* wacc = gm.wall_acc;

    // the jump across the x period: FP32 carries it in the record's x
    // difference; FP64, whose pipe is the narrow one, selects the
    // premultiplied term JX instead
    constexpr bool JSEL = sizeof(T) == 8;
    constexpr bool PSI = !JSEL;  // deviation form (see the file comment)
    T A0[G], AX[G], AY[G], AW[G], JX[JSEL ? G : 1];
    double kx_sum = 0.0;
    __syncwarp();  // the previous item's rare path is done with kcoef
    if (lane < G) {
      const bool ok = lane < cnt;
      kcoef[wib][0][lane] = ok ? ld<T>(gm.kxa, o0 + lane) : T(0);
      kcoef[wib][1][lane] = ok ? ld<T>(gm.kya, o0 + lane) : T(0);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const bool ok = g < cnt;
      const int o = o0 + (ok ? g : 0);
      const double a0 = ok ? (double)ld<T>(HAS_S ? gm.diag : gm.inv, o) : 0.0;
      double ax = ok ? (double)ld<T>(gm.bx, o) : 0.0;
      double ay = ok ? (double)ld<T>(gm.by, o) : 0.0;
      if (!HAS_S) {
        ax *= a0;
        ay *= a0;
      }
      A0[g] = (T)a0;
      AX[g] = (T)ax;
      AY[g] = (T)ay;
      AW[g] = ok ? ld<T>(gm.aw, o) : T(0);
      if (JSEL) JX[JSEL ? g : 0] = (T)(ax * (double)sx * dT);
      if (ok) kx_sum += (double)sx * (double)ld<T>(gm.kxa, o);
    }
    // record-only pass (the adjoint's field records): each solid cell's G
    // values go straight to their record slots; the pass's wall, hot-face
    // and moment sums are not used, so the out-of-line epilogue is skipped
    const bool rec_only = PASS && (flags & (SWEEP_FLUX | SWEEP_RECORD)) == SWEEP_RECORD;
    int rsl[PASS ? G : 1];
    if constexpr (PASS) {
#pragma unroll
      for (int g = 0; g < G; ++g) rsl[g] = (rec_only && g < cnt) ? gm.rec_slot[o0 + g] : -1;
    }

    // Row values.  FP32 without s(x), G even: ordinates in pairs (float2),
    // updated by the paired FP32 instructions of sm_100+ (__ffma2_rn and
    // friends: one instruction per two ordinates, same rounding per lane).
    constexpr bool X2 = sizeof(T) == 4 && !HAS_S && (G % 2 == 0);
    constexpr int GV = X2 ? G / 2 : G;
    using VV = typename std::conditional<X2, float2, T>::type;
    VV v[RMAX][GV];
    auto VG = [&](int r, int g) -> T& {
      if constexpr (X2) return (g & 1) ? v[r][g >> 1].y : v[r][g >> 1].x;
      else return v[r][g];
    };
    VV AXv[GV], AYv[GV], AWv[GV];
#pragma unroll
    for (int h = 0; h < GV; ++h) {
      if constexpr (X2) {
        AXv[h] = make_float2(AX[2 * h], AX[2 * h + 1]);
        AYv[h] = make_float2(AY[2 * h], AY[2 * h + 1]);
        AWv[h] = make_float2(AW[2 * h], AW[2 * h + 1]);
      }
    }
    const T* front = reinterpret_cast<const T*>(gm.front);
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
#pragma unroll
      for (int g = 0; g < G; ++g)
        VG(r, g) = (active && r >= rb && g < cnt) ? front[(size_t)(o0 + g) * ny + j0 + (r - rb)] : T(0);

    // Prefetch the records of diagonal s into buffer b.  With RFIXED the
    // warp's ny records are one contiguous run and part m of it is copied by
    // lane m % 32 (coalesced); otherwise every lane copies its own rows.
    // RFIXED copies: part m = 32 k + lane of the run goes to a slot that
    // repeats with period KP in k up to a shift of 32 KP / CH slots, so two to
    // four lane-constant offsets and compile-time shifts address every copy
    constexpr int KP = CH == 1 ? (RMAX >= 8 ? 2 : 1) : (RMAX >= 8 ? 4 : (RMAX == 4 ? 2 : 1));
    unsigned pslot[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const int m = k * 32 + lane;
      const int jr = m / CH, c = m % CH;
      pslot[k] = (unsigned)__cvta_generic_to_shared(&recbuf[wib][0][c][rec_slot<RMAX>(jr / RMAX, jr % RMAX)]);
    }
    const bool full_run = NH == 2 || ny * CH >= 32 * RMAX * CH;  // every lane copies every k
    auto prefetch = [&](int s, int b) {
      const char* g0 = reinterpret_cast<const char*>(recq + ((size_t)s * ny + rh) * 4);
      if (RFIXED && full_run) {
        CpRun<0, RMAX * CH, KP, CH>::go(pslot, (unsigned)(b * CH * 32 * RMAX * 16), g0 + lane * 16);
      } else if (RFIXED) {
        const int n16 = ny * CH;
#pragma unroll
        for (int k = 0; k < RMAX * CH; ++k) {
          const int m = k * 32 + lane;
          if (m < n16) {
            const int jr = m / CH, c = m % CH;
            cp_async16(&recbuf[wib][b][c][rec_slot<RMAX>(jr / RMAX, jr % RMAX)], g0 + (size_t)m * 16);
          }
        }
      } else if (active) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r >= rb)
#pragma unroll
            for (int c = 0; c < CH; ++c)
              cp_async16(&recbuf[wib][b][c][rec_slot<RMAX>(lane, r)],
                         g0 + ((size_t)(j0 + r - rb) * CH + c) * 16);
      }
      cp_async_commit();
    };

    // sum_g K_g T_g of register row r (wall and hot-face fluxes): paired
    // FP32 products in two chains
    auto kdot = [&](const T* K, const VV* K2r, int r) -> T {
      if constexpr (X2) {
        const float2* K2 = K2r;
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
    const int below = lane > 0 ? lane - 1 : (gm.py ? tpp - 1 : 0);
    const int out_x_side = sx > 0 ? 1 : 0, out_y_side = sy > 0 ? 3 : 2;
    double phi = 0.0;
    // The warp's T_L partials go by row through shared memory so that one
    // atomic instruction covers 32 consecutive rows of the skewed
    // accumulator (8 sectors instead of 32).
    const bool tr_atom = tlq != nullptr;
    // SWEEP_BLOCK_COMBINE: the block's warps hold groups of one octant with
    // one start column, so row j's partials of the four warps are added in
    // shared memory (FP32, fixed order) and each warp issues the atomics of a
    // quarter of the rows: a block barrier per step, a quarter of the atomics
    const bool comb = (WPB == 4 || NH == 2) && RFIXED && full_run && tr_atom &&
                      (flags & SWEEP_BLOCK_COMBINE) && !L.item_counter;
    int par = 0;
    // block-combined moments of a step, done one step later (after the next
    // step's rows, so that their loads overlap that step's arithmetic)
    auto comb_rows = [&](int s_c, int par_c) {
      constexpr int RQ = (8 * RMAX + 31) / 32;
      const int w0 = NH == 2 ? half * 4 : 0;
#pragma unroll
      for (int k = 0; k < RQ; ++k) {
        const int local = 32 * k + lane;
        const int j = gi * 8 * RMAX + local;
        if ((8 * RMAX) % 32 == 0 || local < 8 * RMAX) {
          const T t01 = tlbuf[par_c][w0 + 0][j] + tlbuf[par_c][w0 + 1][j];
          const T t23 = tlbuf[par_c][w0 + 2][j] + tlbuf[par_c][w0 + 3][j];
          atomicAdd(tlq + (size_t)s_c * ny + rh + j, (double)(t01 + t23));
        }
      }
    };
    int s_prev = -1;
    // hot-face flux: each row crosses the hot column once per sweep, so its
    // sum_g K_gx T_g is kept per row in the sweep precision and widened once
    T hot[RMAX];
#pragma unroll
    for (int r = 0; r < RMAX; ++r) hot[r] = T(0);
    int n_hot = 0;
    // Hot column without a branch (FP32 pairs, fixed rows, nx a multiple of
    // the rows per lane): at step d the rows at the hot column are the rows
    // j = d + d0 + 1 (mod nx), all at register row (d + d0 + 1) mod RMAX of
    // their lanes, so every lane adds that register row's K_x dot under a
    // predicate inside the row loop and keeps it where the row is hot
    // (two-warp groups keep the per-row path: the extra registers spill at
    // their 128-register bound)
    const bool uni_hot = NH == 1 && X2 && RFIXED && !PASS && (nx % RMAX == 0) &&
                         ((RMAX & (RMAX - 1)) == 0);
    float hot8 = 0.f;     // this lane's hot-row fluxes of up to RMAX steps
    double hot_d = 0.0;   // and their sum
    // diagonals of steps d .. d + NST - 2 are in flight at the top of step d
    // (they wrap around nx, so the copies past the last step stay in bounds)
    if constexpr (NH == 2) {
      // the other half reads this half's top row of "step -1" at step 0
      if (lane == 31)
#pragma unroll
        for (int g = 0; g < G; ++g) xch[1][gi][half][g] = VG(RMAX - 1, g);
      __syncthreads();
    }
    int s = d0;
    int sf = d0;  // diagonal of the next copy
#pragma unroll
    for (int b = 0; b < NST - 1; ++b) {
      prefetch(sf, b);
      sf = (sf + 1 == nx) ? 0 : sf + 1;
    }
    // 8 ordinates x 8 rows per lane (the widest FP32 form): a second copy of
    // the step loop with the launch-constant conditions of its common case
    // (full warps, block combine, hot column under a predicate) known at
    // compile time, unrolled by two steps so that the buffer parities are
    // constants (about 3 % per launch on a 256 x 256 mesh)
    auto step_loop = [&](auto FASTV) {
      constexpr bool F = decltype(FASTV)::value;
      int cur = 0, bf = NST - 1;  // buffer of step d, buffer of the next copy
#pragma unroll(F ? 2 : 1)
      for (int d = 0; d < nx; ++d) {
        const int s_next = (s + 1 == nx) ? 0 : s + 1;
        if constexpr (F) {
          const char* g0f = reinterpret_cast<const char*>(recq + ((size_t)sf * ny + rh) * 4);
          CpRun<0, RMAX * CH, KP, CH>::go(pslot, (unsigned)(bf * CH * 32 * RMAX * 16), g0f + lane * 16);
          cp_async_commit();
        } else {
          prefetch(sf, bf);
        }
        sf = (sf + 1 == nx) ? 0 : sf + 1;
        bf = (bf + 1 == NST) ? 0 : bf + 1;
        cp_async_wait<NST - 1>();
        __syncwarp();  // parts copied by other lanes are visible
        VV dn0[GV];
#pragma unroll
        for (int h = 0; h < GV; ++h) {
          if constexpr (X2) {
            dn0[h].x = __shfl_sync(FULL, v[RMAX - 1][h].x, below);
            dn0[h].y = __shfl_sync(FULL, v[RMAX - 1][h].y, below);
          } else {
            dn0[h] = __shfl_sync(FULL, v[RMAX - 1][h], below);
          }
        }
        if constexpr (NH == 2) {
          // lane 0: the other half's top row of the previous step (for the
          // lower half across the y period; a wall's record ignores it)
          if (lane == 0) {
            const float2* xo = reinterpret_cast<const float2*>(&xch[(d + 1) & 1][gi][half ^ 1][0]);
#pragma unroll
            for (int h = 0; h < GV; ++h) dn0[h] = xo[h];
          }
        }
        if (F || active) {
          uint32_t pk[RMAX];
          T tls[RMAX];
          // uniform hot column: the hot row of this step is register row rs of
          // whichever lane holds it; its K_x dot accumulates under a predicate
          const int rs = (d + d0 + 1) & (RMAX - 1);
          float2 hk = make_float2(0.f, 0.f);
          uint32_t pkh = 0;
          VV K2v[X2 ? GV : 1];
          if constexpr (X2) {
            if (F || uni_hot) {
#pragma unroll
              for (int h = 0; h < GV; ++h) K2v[h] = reinterpret_cast<const float2*>(kcoef[wib][0])[h];
            }
          }
          // branch-free update of all rows of the step (top row first: the row
          // below still holds its previous value, the y upwind neighbour)
#pragma unroll
          for (int rr = 0; rr < RMAX; ++rr) {
            const int r = RMAX - 1 - rr;
            if (RFIXED || r >= rb) {
              const int slot = rec_slot<RMAX>(lane, r);
              const T* rc0 = reinterpret_cast<const T*>(&recbuf[wib][cur][0][slot]);
              const T* rc1 = reinterpret_cast<const T*>(&recbuf[wib][cur][CH - 1][slot]);
              const T src = rc0[0], twx = rc0[1];
              const T twy = CH == 1 ? rc0[2] : rc1[0];
              const uint32_t packed = rec_bits(CH == 1 ? rc0[3] : rc1[1]);
              const bool wx = packed & REC_WIN_X, wy = packed & REC_WIN_Y;
              const bool jump = packed & REC_JUMP;
              const bool below_in_lane = RFIXED ? (r > 0) : (r > rb);
              T sval = T(1);
              if (HAS_S) sval = (T)__ldg(sv_ptr + (packed & REC_CELL_MASK));
              if constexpr (X2) {
                // deviation form: u_a - T_L,cell = m_a psi_a + t_a, with the
                // upwind row's psi (m = 1, t = its T_L minus this cell's, the
                // jump included on the jump column) or a wall (m = 0, t =
                // T_w - T_L,cell); psi = A_x (u_x - T_L) + A_y (u_y - T_L).
                // The weight of T_L is exactly 1 - A_x - A_y whatever the float
                // rounding of A_x and A_y, and no float value carries T_L
                const float mx = wx ? 0.f : 1.f, my = wy ? 0.f : 1.f;
                const float2 mx2 = make_float2(mx, mx), tx2 = make_float2(twx, twx);
                const float2 my2 = make_float2(my, my), ty2 = make_float2(twy, twy);
                float2 tlp = make_float2(0.f, 0.f);
#pragma unroll
                for (int h = 0; h < GV; ++h) {
                  const float2 ux = __ffma2_rn(mx2, v[r][h], tx2);  // u_x - T_L,cell
                  const float2 ud = below_in_lane ? v[r > 0 ? r - 1 : 0][h] : dn0[h];
                  const float2 uy = __ffma2_rn(my2, ud, ty2);       // u_y - T_L,cell
                  float2 acc = __fmul2_rn(AYv[h], uy);
                  acc = __ffma2_rn(AXv[h], ux, acc);
                  v[r][h] = acc;
                  tlp = __ffma2_rn(AWv[h], acc, tlp);
                  if ((F || uni_hot) && r == rs) hk = __ffma2_rn(K2v[h], acc, hk);
                }
                if ((F || uni_hot) && r == rs) pkh = packed;
                pk[r] = packed;
                tls[r] = tlp.x + tlp.y;
              } else {
              T tl = T(0), tl2 = T(0);  // two partial chains of the T_L moment
              // FP32: the deviation form of the paired path (with s(x):
              // psi = (beta_x (u_x - T_L) + beta_y (u_y - T_L)) / (s + D));
              // FP64 carries T_o, the jump premultiplied (JX)
#pragma unroll
              for (int g = 0; g < G; ++g) {
                const T ux = JSEL ? (wx ? twx : VG(r, g)) : (wx ? T(0) : VG(r, g)) + twx;
                const T ud = below_in_lane ? VG(r > 0 ? r - 1 : 0, g) : dn0[g];
                const T uy = JSEL ? (wy ? twy : ud) : (wy ? T(0) : ud) + twy;
                const T jx = (JSEL && jump) ? JX[JSEL ? g : 0] : T(0);
                T acc;
                if (!JSEL) acc = AY[g] * uy;
                else if (HAS_S) acc = fma(AY[g], uy, src + jx);
                else acc = fma(AY[g], uy, fma(src, A0[g], jx));
                acc = fma(AX[g], ux, acc);
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
          }
          if ((F || comb) && s_prev >= 0) comb_rows(s_prev, par ^ 1);
          // walls per row; the hot column per row too unless uni_hot took it
          const uint32_t RARE = REC_WOUT_X | REC_WOUT_Y | ((F || uni_hot) ? 0u : (uint32_t)REC_LAST);
          uint32_t any = 0;
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
            if (RFIXED || r >= rb) any |= pk[r];
          // cells leaving into a wall, the hot-contact column, flux / record passes
          if ((any & RARE) || rare_pass) {
            const T* KX = kcoef[wib][0];
            const T* KY = kcoef[wib][1];
            // the coefficients once per step (a generic-address atomic between
            // rows would otherwise force them to be reloaded)
            VV KXr[GV], KYr[GV];
            if constexpr (X2) {
#pragma unroll
              for (int h = 0; h < GV; ++h) {
                KXr[h] = reinterpret_cast<const float2*>(KX)[h];
                KYr[h] = reinterpret_cast<const float2*>(KY)[h];
              }
            }
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
              if (!(RFIXED || r >= rb)) continue;
              const uint32_t packed = pk[r];
              if (!(packed & REC_SOLID) || !((packed & RARE) || rare_pass)) continue;
              const int cell = (int)(packed & REC_CELL_MASK);
              const bool last = packed & REC_LAST;
              if constexpr (PASS) {
                if (rec_only) {
                  T* rec = reinterpret_cast<T*>(gm.rec);
#pragma unroll
                  for (int g = 0; g < G; ++g)
                    if (rsl[g] >= 0) rec[(size_t)rsl[g] * gm.n_cells + cell] = VG(r, g);
                  continue;
                }
#pragma unroll
                T loc[NH == 2 ? G : 1];
                T* sc = NH == 2 ? loc : scratch;
                for (int g = 0; g < G; ++g) sc[g] = VG(r, g);
                phi += cell_epilogue_2d<T, G>(gm, sc, cell, packed, last, o0, cnt, sx, sy,
                                              flags, kx_sum);
                continue;
              }
              if (packed & (REC_WOUT_X | ((F || uni_hot) ? 0u : (uint32_t)REC_LAST))) {
                const T sk = kdot(KX, KXr, r);
                if (packed & REC_WOUT_X) {
                  atomicAdd(wacc + (size_t)cell * 6 + out_x_side, widen(sk));
                } else {
                  hot[r] = sk;
                  ++n_hot;
                }
              }
              if (packed & REC_WOUT_Y) {
                const T sy_k = kdot(KY, KYr, r);
                atomicAdd(wacc + (size_t)cell * 6 + out_y_side, widen(sy_k));
              }
            }
          }
          if constexpr (X2 && RFIXED && !PASS) {
            if (F || uni_hot) {
              if ((pkh & (REC_LAST | REC_SOLID | REC_WOUT_X)) == (REC_LAST | REC_SOLID)) {
                hot8 += hk.x + hk.y;
                ++n_hot;
              }
              if (rs == RMAX - 1) {
                hot_d += widen(hot8);
                hot8 = 0.f;
              }
            }
          }
          // the moment atomics come after all rows: a generic-address atomic
          // between two rows would keep the next row's shared-memory loads from
          // being scheduled ahead of it
          if (F || tr_atom) {
#pragma unroll
            for (int r = 0; r < RMAX; ++r)
              if (RFIXED || r >= rb) tlbuf[par][wib][jl + r - rb] = (pk[r] & REC_SOLID) ? tls[r] : T(0);
          } else {
#pragma unroll
            for (int r = 0; r < RMAX; ++r)
              if ((RFIXED || r >= rb) && (pk[r] & REC_SOLID))
                atomicAdd(tl_acc + (pk[r] & REC_CELL_MASK), X2 ? widen(tls[r]) : (double)tls[r]);
          }
        }
        if constexpr (NH == 2) {
          if (lane == 31)
#pragma unroll
            for (int h = 0; h < GV; ++h)
              reinterpret_cast<float2*>(&xch[d & 1][gi][half][0])[h] = v[RMAX - 1][h];
        }
        if (F || comb) {
          __syncthreads();
          s_prev = s;
          par ^= 1;
        } else if (tr_atom) {
          if (NH == 2) __syncthreads();  // the exchange of the top rows
          else __syncwarp();
          double* row = tlq + (size_t)s * ny + rh + lane;
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
            if (RFIXED && full_run ? true : 32 * r + lane < ny)
              atomicAdd(row + 32 * r, (double)tlbuf[par][wib][32 * r + lane]);
          if (NH == 2) par ^= 1;
        } else if (NH == 2) {
          __syncthreads();
        }
        s = s_next;
        cur = (cur + 1 == NST) ? 0 : cur + 1;
        __syncwarp();
      }
    };
    if constexpr (X2 && RFIXED && !PASS && NH == 1 && G == 8 && RMAX == 8) {
      if (comb && uni_hot && tpp == 32) step_loop(std::true_type{});
      else step_loop(std::false_type{});
    } else {
      step_loop(std::false_type{});
    }
    if (comb && s_prev >= 0) comb_rows(s_prev, par ^ 1);  // the last step's moments
    cp_async_wait<0>();  // copies past the last step land before the buffers are reused
    __syncwarp();

    T* frontw = reinterpret_cast<T*>(gm.front);
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (active && r >= rb && g < cnt) frontw[(size_t)(o0 + g) * ny + j0 + (r - rb)] = VG(r, g);

#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const double dk = widen(hot[r]);
      phi += sx > 0 ? dk : -dk;
    }
    hot_d += widen(hot8);
    phi += sx > 0 ? hot_d : -hot_d;
    if (sx > 0) phi += (double)n_hot * dT * kx_sum;
    for (int o = 16; o > 0; o >>= 1) phi += __shfl_xor_sync(FULL, phi, o);
    if (lane == 0 && phi != 0.0) atomicAdd(gm.phi_acc, phi);
    if (!L.item_counter) return;
  }
}

}  // namespace obte

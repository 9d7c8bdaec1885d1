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

#include <algorithm>

#include "obte_internal.h"

namespace cg = cooperative_groups;

namespace {



template <typename T>
__device__ __forceinline__ T apply_A(const CGArgs& a, const T* v, int c, uint8_t code, int x, int y,
                                     int z) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const T vc = v[c];
  const T wx = (T)a.wx, wy = (T)a.wy, wz = (T)a.wz;
  T acc = T(0);
  if (!(code & CODE_WALL_XM)) acc += wx * (vc - v[c - x + (x > 0 ? x - 1 : nx - 1)]);
  if (!(code & CODE_WALL_XP)) acc += wx * (vc - v[c - x + (x < nx - 1 ? x + 1 : 0)]);
  if (!(code & CODE_WALL_YM)) acc += wy * (vc - v[c + nx * ((y > 0 ? y - 1 : ny - 1) - y)]);
  if (!(code & CODE_WALL_YP)) acc += wy * (vc - v[c + nx * ((y < ny - 1 ? y + 1 : 0) - y)]);
  if (a.dim == 3) {
    if (!(code & CODE_WALL_ZM)) acc += wz * (vc - v[c + nx * ny * ((z > 0 ? z - 1 : nz - 1) - z)]);
    if (!(code & CODE_WALL_ZP)) acc += wz * (vc - v[c + nx * ny * ((z < nz - 1 ? z + 1 : 0) - z)]);
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
  // Partial sums go per thread and per warp in the vector precision and in
  // FP64 only across warps and blocks; the CG scalars are formed by thread 0
  // of each block (from the same grid sums, so identical everywhere) and
  // broadcast: GB300's FP64 pipe is 1/64 of FP32 and would otherwise bind.
  __shared__ double sc[2];  // alpha, beta
  __shared__ int sf[2];     // run, p.q > 0
  auto wsum = [&](T u) -> double {  // block sum, valid in thread 0
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = (double)u;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
      for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) t += red[i];
    return t;
  };
  T rr_l = T(0), bb_l = T(0);
  for (int c = tid; c < n; c += stride) {
    const uint8_t code = a.code[c];
    T rc = T(0);
    if (code & CODE_SOLID) {
      const int xi = c % a.nx, yi = (c / a.nx) % a.ny, zi = c / (a.nx * a.ny);
      double b = 0.0;
      if (xi == 0 && !(code & CODE_WALL_XM)) b += a.wx * a.dT;
      if (xi == a.nx - 1 && !(code & CODE_WALL_XP)) b -= a.wx * a.dT;
      rc = (T)b - apply_A<T>(a, x, c, code, xi, yi, zi);
      bb_l += (T)(b * b);
    }
    r[c] = rc;
    p[c] = rc;
    q[c] = T(0);
    rr_l += rc * rc;
  }
  {
    const double s0 = wsum(rr_l);
    const double s1 = wsum(bb_l);
    if (threadIdx.x == 0) {
      part0[blockIdx.x] = s0;
      part1[blockIdx.x] = s1;
    }
  }
  grid.sync();
  // thread 0 keeps rr, stop, it and forms alpha, beta and the run flag
  double rr = 0.0, stop = 0.0;
  int it = 0;
  {
    const double rr0 = sum_partials(part0, gridDim.x, &bc);
    const double bb = sum_partials(part1, gridDim.x, &bc);
    if (threadIdx.x == 0) {
      rr = rr0;
      stop = a.tol * a.tol * bb;
      sc[1] = 0.0;
      sf[0] = (it < a.max_iter && rr > stop && bb > 0.0) ? 1 : 0;
    }
  }
  grid.sync();  // every block has read the partials before they are reused
  // CG with the matrix-vector product carried by recurrence, two grid
  // synchronisations per iteration: with p = r + beta p, A p = A r + beta A p,
  // so the product needs the neighbours' r (final after the r update's
  // synchronisation) and p, q stay cell-local.
  while (sf[0]) {
    // p = r + beta p, q = A r + beta q, and p.q
    const T bt = (T)sc[1];
    T pq_l = T(0);
    for (int c = tid; c < n; c += stride) {
      const uint8_t code = a.code[c];
      T pc = T(0), qc = T(0);
      if (code & CODE_SOLID) {
        const int xi = c % a.nx, yi = (c / a.nx) % a.ny, zi = c / (a.nx * a.ny);
        const T w = apply_A<T>(a, r, c, code, xi, yi, zi);
        pc = r[c] + bt * p[c];
        qc = w + bt * q[c];
      }
      p[c] = pc;
      q[c] = qc;
      pq_l += pc * qc;
    }
    {
      const double s0 = wsum(pq_l);
      if (threadIdx.x == 0) part0[blockIdx.x] = s0;
    }
    grid.sync();
    {
      const double pq = sum_partials(part0, gridDim.x, &bc);
      if (threadIdx.x == 0) {
        sf[1] = pq > 0.0 ? 1 : 0;
        sc[0] = pq > 0.0 ? rr / pq : 0.0;
      }
      __syncthreads();
    }
    if (!sf[1]) break;  // uniform across blocks
    const T al = (T)sc[0];
    T rn_l = T(0);
    for (int c = tid; c < n; c += stride) {
      x[c] += al * p[c];
      const T rc = r[c] - al * q[c];
      r[c] = rc;
      rn_l += rc * rc;
    }
    {
      const double s0 = wsum(rn_l);
      if (threadIdx.x == 0) part1[blockIdx.x] = s0;
    }
    grid.sync();
    {
      const double rn = sum_partials(part1, gridDim.x, &bc);
      if (threadIdx.x == 0) {
        sc[1] = rn / rr;
        rr = rn;
        ++it;
        sf[0] = (it < a.max_iter && rr > stop) ? 1 : 0;
      }
      __syncthreads();
    }
  }
  grid.sync();  // partials read before the mean reuses them
  // remove the mean over solid cells
  double sum_l = 0.0, cnt_l = 0.0;
  for (int c = tid; c < n; c += stride)
    if (a.code[c] & CODE_SOLID) {
      sum_l += (double)x[c];
      cnt_l += 1.0;
    }
  const double s = block_reduce(sum_l, red);
  const double s2 = block_reduce(cnt_l, red);
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
  __shared__ double bval[2];
  __shared__ T sc[2];   // alpha, beta in the vector precision
  __shared__ int sf;    // run
  const int n = a.nx * a.ny * a.nz;
  const int t0 = threadIdx.x, st = blockDim.x;
  T* x = reinterpret_cast<T*>(a.x);
  T* r = reinterpret_cast<T*>(a.r);
  T* p = reinterpret_cast<T*>(a.p);
  T* q = reinterpret_cast<T*>(a.q);
  // block sum, valid in thread 0: per thread and per warp in the vector
  // precision, FP64 across warps; the CG scalars are formed by thread 0 (the
  // FP64 pipe is narrow, a division in every thread would bind it)
  auto bsum = [&](T u) -> double {
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)u;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
      for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) s += red[i];
    return s;
  };
  for (int c = t0; c < n; c += st) {
    const int xi = c % a.nx;
    x[c] = (a.code[c] & CODE_SOLID) ? (T)(-a.dT * ((xi + 0.5) / a.nx - 0.5)) : T(0);
  }
  __syncthreads();
  T rr_l = T(0), bb_l = T(0);
  for (int c = t0; c < n; c += st) {
    const uint8_t code = a.code[c];
    T rc = T(0);
    if (code & CODE_SOLID) {
      const int xi = c % a.nx, yi = (c / a.nx) % a.ny, zi = c / (a.nx * a.ny);
      double b = 0.0;
      if (xi == 0 && !(code & CODE_WALL_XM)) b += a.wx * a.dT;
      if (xi == a.nx - 1 && !(code & CODE_WALL_XP)) b -= a.wx * a.dT;
      rc = (T)b - apply_A<T>(a, x, c, code, xi, yi, zi);
      bb_l += (T)(b * b);
    }
    r[c] = rc;
    p[c] = rc;
    rr_l += rc * rc;
  }
  double rr = bsum(rr_l);  // thread 0
  const double bb = bsum(bb_l);
  const double stop = a.tol * a.tol * bb;
  int it = 0;
  if (threadIdx.x == 0) sf = (it < a.max_iter && rr > stop && bb > 0.0) ? 1 : 0;
  __syncthreads();
  while (sf) {
    T pq_l = T(0);
    for (int c = t0; c < n; c += st) {
      const uint8_t code = a.code[c];
      T qc = T(0);
      if (code & CODE_SOLID) {
        const int xi = c % a.nx, yi = (c / a.nx) % a.ny, zi = c / (a.nx * a.ny);
        qc = apply_A<T>(a, p, c, code, xi, yi, zi);
      }
      q[c] = qc;
      pq_l += p[c] * qc;
    }
    const double pq = bsum(pq_l);
    if (threadIdx.x == 0) {
      sf = pq > 0.0 ? 1 : 0;
      sc[0] = (T)(pq > 0.0 ? rr / pq : 0.0);
    }
    __syncthreads();
    if (!sf) break;
    const T al = sc[0];
    T rn_l = T(0);
    for (int c = t0; c < n; c += st) {
      x[c] += al * p[c];
      const T rc = r[c] - al * q[c];
      r[c] = rc;
      rn_l += rc * rc;
    }
    const double rn = bsum(rn_l);
    if (threadIdx.x == 0) {
      sc[1] = (T)(rn / rr);
      rr = rn;
      ++it;
      sf = (it < a.max_iter && rr > stop) ? 1 : 0;
    }
    __syncthreads();
    const T be = sc[1];
    for (int c = t0; c < n; c += st) p[c] = r[c] + be * p[c];
    __syncthreads();
  }
  T sum_l = T(0), cnt_l = T(0);
  for (int c = t0; c < n; c += st)
    if (a.code[c] & CODE_SOLID) {
      sum_l += x[c];
      cnt_l += T(1);
    }
  const double sum = bsum(sum_l);
  const double cnt = bsum(cnt_l);
  if (threadIdx.x == 0) bval[0] = cnt > 0 ? sum / cnt : 0.0;
  __syncthreads();
  const double mean = bval[0];
  for (int c = t0; c < n; c += st) a.T_out[c] = (a.code[c] & CODE_SOLID) ? (double)x[c] - mean : 0.0;
  if (t0 == 0) *a.iters_out = it;
}


// The same CG on one thread-block cluster.  The rows of cells (lines along
// x) are cut into `ncl` contiguous ranges of `rpc` rows, one per CTA, and the
// four CG vectors live in the CTAs' shared memory; a y / z neighbour row in
// another CTA's range is read through distributed shared memory.  Thread t
// handles column t % nx of rows t / nx, t / nx + 1024 / nx, ... of its range,
// so no cell needs index divisions.  Reductions: each CTA's partial goes to a
// slot in its shared memory, one cluster barrier, then lane k of warp 0 reads
// rank k's partial and a fixed shuffle tree adds them (the same sum in every
// CTA; two slots used alternately, so a barrier per reduction suffices).  No
// grid-wide synchronisation and no global-memory traffic in the iteration.
template <typename T>
__device__ __forceinline__ void cluster_cg(const CGArgs& a, int rpc) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int ncl = (int)cl.num_blocks();
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int cpc = rpc * nx;
  extern __shared__ __align__(16) unsigned char smem_cg[];
  T* xs = reinterpret_cast<T*>(smem_cg);
  T* rs = xs + cpc;
  T* ps = rs + cpc;
  T* qs = ps + cpc;
  uint8_t* cs = reinterpret_cast<uint8_t*>(qs + cpc);
  __shared__ double slot[2][2];
  __shared__ double bcast[2];
  __shared__ double red2[32][2];
  const int rows = ny * nz;
  const int r0g = rank * rpc;                            // first global row of this CTA
  const int nrow = max(0, min(rpc, rows - r0g));         // rows held here
  const int tid = threadIdx.x, nth = blockDim.x;
  const int rstep = nth / nx;                            // rows per pass of the block
  const int xi = tid % nx, rfirst = tid / nx;
  const bool has_col = rfirst < rstep;                   // threads beyond rstep rows idle
  const T wx = (T)a.wx, wy = (T)a.wy, wz = (T)a.wz;       // converted once (FP64 pipe)

  // the vector v at (global row gr, column x): local, or in the owner CTA
  auto rowval = [&](T* vloc, int gr, int x) -> T {
    const int lr = gr - r0g;
    if (lr >= 0 && lr < nrow) return vloc[lr * nx + x];
    const int rk = gr / rpc;
    return cl.map_shared_rank(vloc, rk)[(gr - rk * rpc) * nx + x];
  };
  // (A v) at local row lr, column xi
  auto applyA = [&](T* v, int lr, uint8_t code) -> T {
    const int gr = r0g + lr;
    const int yi = gr % ny, zi = gr / ny;
    const T vc = v[lr * nx + xi];
    T acc = T(0);
    if (!(code & CODE_WALL_XM)) acc += wx * (vc - v[lr * nx + (xi > 0 ? xi - 1 : nx - 1)]);
    if (!(code & CODE_WALL_XP)) acc += wx * (vc - v[lr * nx + (xi < nx - 1 ? xi + 1 : 0)]);
    if (!(code & CODE_WALL_YM)) acc += wy * (vc - rowval(v, zi * ny + (yi > 0 ? yi - 1 : ny - 1), xi));
    if (!(code & CODE_WALL_YP)) acc += wy * (vc - rowval(v, zi * ny + (yi < ny - 1 ? yi + 1 : 0), xi));
    if (a.dim == 3) {
      if (!(code & CODE_WALL_ZM)) acc += wz * (vc - rowval(v, (zi > 0 ? zi - 1 : nz - 1) * ny + yi, xi));
      if (!(code & CODE_WALL_ZP)) acc += wz * (vc - rowval(v, (zi < nz - 1 ? zi + 1 : 0) * ny + yi, xi));
    }
    return acc;
  };
  int sl = 0;
  // cluster-wide sums of (v0, v1), identical in every CTA
  // (partials are summed per thread and per warp in the vector precision,
  // then in FP64: the FP64 pipe of one SM would otherwise bind)
  auto csum = [&](T u0, T u1, double& o0, double& o1) {
    const unsigned FULL = 0xffffffffu;
    for (int o = 16; o > 0; o >>= 1) {
      u0 += __shfl_xor_sync(FULL, u0, o);
      u1 += __shfl_xor_sync(FULL, u1, o);
    }
    const int lane = tid & 31, w = tid >> 5;
    if (lane == 0) {
      red2[w][0] = (double)u0;
      red2[w][1] = (double)u1;
    }
    __syncthreads();
    if (w == 0) {  // this CTA's partial: warp 0 adds the warps' sums
      double t0 = lane < (nth >> 5) ? red2[lane][0] : 0.0;
      double t1 = lane < (nth >> 5) ? red2[lane][1] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(FULL, t0, o);
        t1 += __shfl_xor_sync(FULL, t1, o);
      }
      if (lane == 0) {
        slot[sl][0] = t0;
        slot[sl][1] = t1;
      }
    }
    cl.sync();
    if (w == 0) {  // lane k reads rank k's partial; the same tree in every CTA
      double t0 = 0.0, t1 = 0.0;
      if (lane < ncl) {
        const double* rp = cl.map_shared_rank(&slot[sl][0], lane);
        t0 = rp[0];
        t1 = rp[1];
      }
      for (int o = 16; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(FULL, t0, o);
        t1 += __shfl_xor_sync(FULL, t1, o);
      }
      if (lane == 0) {
        bcast[0] = t0;
        bcast[1] = t1;
      }
    }
    __syncthreads();
    o0 = bcast[0];
    o1 = bcast[1];
    sl ^= 1;
  };

  // x0 = linear profile
  if (has_col)
    for (int lr = rfirst; lr < nrow; lr += rstep) {
      const int l = lr * nx + xi;
      const uint8_t code = a.code[(size_t)(r0g + lr) * nx + xi];
      cs[l] = code;
      xs[l] = (code & CODE_SOLID) ? (T)(-a.dT * ((xi + 0.5) / nx - 0.5)) : T(0);
    }
  cl.sync();
  // r = b - A x0, p = r, q = 0
  T rr_l = T(0), bb_l = T(0);
  if (has_col)
    for (int lr = rfirst; lr < nrow; lr += rstep) {
      const int l = lr * nx + xi;
      const uint8_t code = cs[l];
      T rc = T(0);
      if (code & CODE_SOLID) {
        double b = 0.0;
        if (xi == 0 && !(code & CODE_WALL_XM)) b += a.wx * a.dT;
        if (xi == nx - 1 && !(code & CODE_WALL_XP)) b -= a.wx * a.dT;
        rc = (T)b - applyA(xs, lr, code);
        bb_l += (T)(b * b);
      }
      rs[l] = rc;
      ps[l] = rc;
      qs[l] = T(0);
      rr_l += rc * rc;
    }
  // the CG scalars are formed by thread 0 and broadcast (the FP64 pipe is
  // narrow: a division in every thread would bind it)
  __shared__ double csc[2];  // alpha, beta
  __shared__ int csf[2];     // run, p.q > 0
  double rr = 0.0, stop = 0.0;
  int it = 0;
  {
    double rr0, bb;
    csum(rr_l, bb_l, rr0, bb);
    if (tid == 0) {
      rr = rr0;
      stop = a.tol * a.tol * bb;
      csc[1] = 0.0;
      csf[0] = (it < a.max_iter && rr > stop && bb > 0.0) ? 1 : 0;
    }
    __syncthreads();
  }
  while (csf[0]) {
    // p = r + beta p, q = A r + beta q (the neighbours' r are final), p.q
    const T bt = (T)csc[1];
    T pq_l = T(0);
    if (has_col)
      for (int lr = rfirst; lr < nrow; lr += rstep) {
        const int l = lr * nx + xi;
        const uint8_t code = cs[l];
        T pc = T(0), qc = T(0);
        if (code & CODE_SOLID) {
          const T w = applyA(rs, lr, code);
          pc = rs[l] + bt * ps[l];
          qc = w + bt * qs[l];
        }
        ps[l] = pc;
        qs[l] = qc;
        pq_l += pc * qc;
      }
    double pq, dummy;
    csum(pq_l, T(0), pq, dummy);
    if (tid == 0) {
      csf[1] = pq > 0.0 ? 1 : 0;
      csc[0] = pq > 0.0 ? rr / pq : 0.0;
    }
    __syncthreads();
    if (!csf[1]) break;  // same value in every CTA
    const T al = (T)csc[0];
    T rn_l = T(0);
    if (has_col)
      for (int lr = rfirst; lr < nrow; lr += rstep) {
        const int l = lr * nx + xi;
        xs[l] += al * ps[l];
        const T rc = rs[l] - al * qs[l];
        rs[l] = rc;
        rn_l += rc * rc;
      }
    double rn;
    csum(rn_l, T(0), rn, dummy);
    if (tid == 0) {
      csc[1] = rn / rr;
      rr = rn;
      ++it;
      csf[0] = (it < a.max_iter && rr > stop) ? 1 : 0;
    }
    __syncthreads();
  }
  // remove the mean over solid cells
  T sum_l = T(0), cnt_l = T(0);
  if (has_col)
    for (int lr = rfirst; lr < nrow; lr += rstep) {
      const int l = lr * nx + xi;
      if (cs[l] & CODE_SOLID) {
        sum_l += xs[l];
        cnt_l += T(1);
      }
    }
  double sum, cnt;
  csum(sum_l, cnt_l, sum, cnt);
  const double mean = cnt > 0 ? sum / cnt : 0.0;
  if (has_col)
    for (int lr = rfirst; lr < nrow; lr += rstep) {
      const int l = lr * nx + xi;
      a.T_out[(size_t)(r0g + lr) * nx + xi] = (cs[l] & CODE_SOLID) ? (double)xs[l] - mean : 0.0;
    }
  if (rank == 0 && tid == 0) *a.iters_out = it;
  cl.sync();  // no CTA leaves while others may still read its shared memory
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) fourier_cg_cluster_kernel(CGArgs a, int rpc) {
  cluster_cg<T>(a, rpc);
}

// many geometries: cluster c of the grid solves jobs[c] (rows cut evenly)
template <typename T>
__global__ void __launch_bounds__(1024, 1) fourier_cg_cluster_jobs_kernel(const CGArgs* jobs) {
  cg::cluster_group cl = cg::this_cluster();
  const int ncl = (int)cl.num_blocks();
  const CGArgs a = jobs[blockIdx.x / ncl];
  const int rows = a.ny * a.nz;
  cluster_cg<T>(a, (rows + ncl - 1) / ncl);
}

// Conductive flux through the solid faces of the plane x = 0 (App. B, the
// kappa_fourier equation), in units of kappa_bulk / h_x: the sum over the
// rows whose x = 0 cell is solid with a solid periodic image at x = nx - 1 of
// (T_image + dT - T_cell).  One block, fixed summation order.
__global__ void __launch_bounds__(256) fourier_hot_flux_kernel(const uint8_t* code, const double* T,
                                                                int nx, int rows, double dT,
                                                                double* out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int row = threadIdx.x; row < rows; row += blockDim.x) {
    const size_t c0 = (size_t)row * nx, c1 = c0 + nx - 1;
    const uint8_t k = code[c0];
    if ((k & CODE_SOLID) && !(k & CODE_WALL_XM)) s += T[c1] + dT - T[c0];
  }
  s = block_reduce(s, red);
  if (threadIdx.x == 0) *out = s;
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

// cluster form (FP32 vectors): 16 CTAs (8 where 16 is not available), when
// the four vectors and the codes of a CTA's range fit its shared memory and
// a row fits the block; returns cudaErrorNotSupported otherwise, so that the
// caller uses the grid form
static cudaError_t launch_fourier_cg_cluster(const CGArgs& a, int n, int precision, cudaStream_t st) {
  const size_t e = precision == 0 ? sizeof(double) : sizeof(float);
  void* kern = precision == 0 ? (void*)fourier_cg_cluster_kernel<double> : (void*)fourier_cg_cluster_kernel<float>;
  if (a.nx > 1024) return cudaErrorNotSupported;
  const int rows = n / a.nx;
  for (int ncl : {16, 8}) {
    const int rpc = (rows + ncl - 1) / ncl;  // rows per CTA
    const size_t cpc = (size_t)rpc * a.nx;
    const size_t smem = 4 * e * cpc + cpc;
    if (smem > 200 * 1024) continue;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncl);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ncl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      continue;
    }
    int rpc_arg = rpc;
    void* args[] = {const_cast<CGArgs*>(&a), &rpc_arg};
    if (cudaLaunchKernelExC(&cfg, kern, args) == cudaSuccess) return cudaSuccess;
    cudaGetLastError();  // launch refused: try the next size, then the grid form
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_fourier_cg_cluster_jobs(const CGArgs* jobs_dev, const CGArgs* jobs_host, int n_jobs,
                                           int precision, cudaStream_t st) {
  if (precision == 0 || n_jobs < 1) return cudaErrorNotSupported;
  void* kern = (void*)fourier_cg_cluster_jobs_kernel<float>;
  for (int ncl : {8, 4}) {
    size_t smem = 0;
    bool fits = true;
    for (int j = 0; j < n_jobs; ++j) {
      const CGArgs& a = jobs_host[j];
      if (a.nx > 1024) fits = false;
      const int rpc = (a.ny * a.nz + ncl - 1) / ncl;
      smem = std::max(smem, 4 * sizeof(float) * (size_t)rpc * a.nx + (size_t)rpc * a.nx);
    }
    if (!fits) return cudaErrorNotSupported;
    if (smem > 200 * 1024) continue;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncl * n_jobs);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ncl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      continue;
    }
    const CGArgs* jd = jobs_dev;
    void* args[] = {&jd};
    if (cudaLaunchKernelExC(&cfg, kern, args) == cudaSuccess) return cudaSuccess;
    cudaGetLastError();
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_fourier_cg(const GeomDev& g, double hx, double hy, double hz, int precision,
                              int max_iter, double tol, double* T_out, int* iters_out,
                              double* work, int blocks_max, cudaStream_t st) {
  CGArgs a = make_cg_args(g, hx, hy, hz, max_iter, tol, T_out, iters_out, work, blocks_max);
  const size_t n = (size_t)g.n_cells;
  if (precision != 0) {  // FP64 arithmetic on 16 SMs would bind their FP64 pipes: grid form
    const cudaError_t ec = launch_fourier_cg_cluster(a, (int)n, precision, st);
    if (ec != cudaErrorNotSupported) return ec;
  }
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

cudaError_t launch_fourier_hot_flux(const uint8_t* code, const double* T, int nx, int rows, double dT,
                                   double* out, cudaStream_t st) {
  fourier_hot_flux_kernel<<<1, 256, 0, st>>>(code, T, nx, rows, dT, out);
  return cudaGetLastError();
}

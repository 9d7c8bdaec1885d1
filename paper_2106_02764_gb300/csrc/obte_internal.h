// Internal declarations shared by the libobte translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// ---------------------------------------------------------------------------
// per-cell face codes (kernel frame): a wall bit means that side of a solid
// cell has no solid neighbour (pore or non-periodic boundary)
// ---------------------------------------------------------------------------
enum : uint8_t {
  CODE_WALL_XM = 1u << 0,
  CODE_WALL_XP = 1u << 1,
  CODE_WALL_YM = 1u << 2,
  CODE_WALL_YP = 1u << 3,
  CODE_WALL_ZM = 1u << 4,
  CODE_WALL_ZP = 1u << 5,
  CODE_SOLID = 1u << 6,
};

// Flags of a skewed cell record (bits 22-31 of its packed word), oriented for
// the record's octant: "in" sides are the upwind ones, "out" the downwind ones.
enum : uint32_t {
  REC_CELL_MASK = (1u << 22) - 1,
  REC_WIN_X = 1u << 22,    // upwind x side is a wall
  REC_WIN_Y = 1u << 23,
  REC_WIN_Z = 1u << 24,
  REC_JUMP = 1u << 25,     // first column of the octant frame, x upwind across the jump
  REC_SOLID = 1u << 26,
  REC_WOUT_X = 1u << 27,   // downwind x side is a wall
  REC_WOUT_Y = 1u << 28,
  REC_WOUT_Z = 1u << 29,
  REC_FIRST = 1u << 30,    // i' == 0
  REC_LAST = 1u << 31,     // i' == nx - 1
};

// sweep flags (runtime, uniform)
enum : int {
  SWEEP_HAS_S = 1 << 0,   // per-cell scattering scale: divide per update
  SWEEP_FLUX = 1 << 1,    // also accumulate J per cell, section fluxes, bin fluxes
  SWEEP_RECORD = 1 << 2,  // write every ordinate field to the record buffer
  // 2D warp kernel: the four warps of a block hold four groups of one octant
  // with the same start column, so their T_L partials of a step can be added
  // in shared memory before the atomics (items padded to blocks of four)
  SWEEP_BLOCK_COMBINE = 1 << 3,
};

// One geometry as seen by the device kernels (kernel frame: x = gradient axis).
struct GeomDev {
  int nx, ny, nz, dim;
  int n_cells;            // nx * ny * nz
  int rows;               // ny * nz
  int py, pz;             // periodic flags of y and z
  int R;                  // rows (along y) per thread
  int tpp;                // threads per z-plane = ceil(ny / R)
  int n_ord;              // ordinates
  int n_walls;
  double dT;              // applied jump across the x period
  double kappa_scale;     // L_x / (dT * cells per cross-section)
  const uint8_t* code;    // [n_cells]
  const int* wall_id;     // [n_cells * 6], side order -x +x -y +y -z +z; -1 none
  const double* s;        // [n_cells] scattering scale (nullptr: 1)
  // iteration state
  double* TL;             // [n_cells] lattice temperature (FP64)
  double* TL_acc;         // [n_cells] sum_o a_o T_o of the running sweep
  void* src;              // [n_cells] s_i T_L,i in the sweep precision
  double* Tw;             // [n_walls]
  double* wall_acc;       // [n_cells * 6] numerator of E3 per (cell, side); only wall sides used
  const double* wall_den; // [n_walls]
  const int* wall_cell;   // [n_walls]
  const int* wall_side;   // [n_walls] side of its cell (0..5: -x +x -y +y -z +z)
  void* twc;              // [n_cells * 6] wall temperature seen through each side, sweep precision
  // Skewed cell records and T_L accumulators of the 2D warp and 3D kernels.
  // Octant q's cell (i', j', k') (mirrored frame) has row = j' + ny k' and sits
  // at diagonal s = (i' + j' + k') mod nx:
  //   rec4[((q * nx + s) * rows + row) * rec_w + f]: rec_w = 4 (2D warp kernel)
  //     {s_i T_L,i, T_w in-x side, T_w in-y side, packed};  rec_w = 8 (3D)
  //     (the in-x field holds sign(p_x) dT instead on the jump column, REC_JUMP;
  //     wall fields of sides without a wall hold 0)
  //     {s_i T_L,i, T_w in-x, in-y, in-z sides, packed, 0, 0, 0}
  //     (deviation form: the wall / difference fields u - T_L,cell, and the
  //     packed word also in field 0, so that one 16-byte load serves a row)
  //   packed = cell (bits 0-21) | REC_* flags of octant q (bits 22-31)
  //   rec_idx[c * n_octants + q] = record index (q * nx + s) * rows + row of cell c
  //   tlq[(q * nx + s) * rows + row]: T_L partial sums of the running sweep in
  //     the same skewed order (2D warp kernel; FP64); the finalisation adds
  //     them to TL_acc's
  //   tlq3: the same for the 3D kernel (eight octants, rows = ny nz), read
  //     through rec_idx
  void* rec4;
  int* rec_idx;
  double* tlq;
  double* tlq3;
  int rec_w;              // values per record: 4 (2D warp kernel), 8 (3D kernel); 0: none
  // Deviation form (float record kernels): the sweep carries psi_o = T_o - T_L
  // per cell, the records' wall / neighbour fields hold the FP64 differences
  // u - T_L,cell of the upwind values (neighbour T_L, wall T_w, image T_L
  // +- dT) rounded once, and the moment accumulators receive sums of psi;
  // the finalisation adds T_L back in FP64.  A float sweep that carried T_o
  // itself would quantise the source s T_L to float, and the slowly
  // converging diffusive mode of T_L stalls on that quantum.
  int psi;
  // deviation form: the T_L part of the hot-face flux, K+ S+ + K- S-, with
  // K+- = sum of K_ox over the ordinates with p_x > 0 (< 0) and S+- = sum of
  // T_L over the cells at x = nx - 1 (x = 0) of the solid-solid faces of the
  // plane x = 0; hot_tl[0..1] = S+, S- of the T_L the next sweep uses
  double kx_pos, kx_neg;
  double* hot_tl;
  void* front;            // [n_ord][rows] row values carried between iterations
  double* phi_acc;        // [1] hot-face flux of the running sweep
  // flux pass outputs
  double* J_acc;          // [n_cells * 3]
  double* phi_sec;        // [nx] flux through every x-section
  double* phi_bin;        // [n_mfp] hot-face flux per MFP bin
  // record pass output: rec[rec_slot[o] * n_cells + cell] for rec_slot[o] >= 0
  void* rec;
  const int* rec_slot;
  // ordinate table (sorted by octant), precision of the sweep
  const void* bx; const void* by; const void* bz; const void* diag; const void* inv;
  const void* aw; const void* kxa; const void* kya; const void* kza; const void* kx;
  const int* mbin;        // [n_ord] MFP bin of each sorted ordinate
  const int* ord_d0;      // [n_ord] start step of the group holding each ordinate
  const int* octant_of;   // [n_ord] octant of each sorted ordinate
  const double* T0;       // [n_cells] starting temperature (the Fourier first guess)
  // control
  int* done;              // [1] converged flag
  int* iter;              // [1] iterations run
  double* kappa_hist;     // [max_hist]
  int max_hist;
  double* delta_max;      // [1] max |dT_L| (as FP64 bits, via atomicMax on u64)
  double tol, tol_TL;
  int min_iter, max_iter;
  double* blk_part;       // [kMaxPartBlocks * 8] per-block partials (finalize, Anderson dots)
  // Anderson acceleration (anderson.cu); aa_m = 0: plain source iteration
  int aa_m;               // window (history slots aa_m + 1 <= 8)
  long aa_nd, aa_nt;      // state lengths: FP64 part (T_L, T_w), row values
  double* aa_gd;          // [(aa_m + 1) * aa_nd] history of g(x)
  double* aa_fd;          // [(aa_m + 1) * aa_nd] history of f = g(x) - x
  double* aa_xcd;         // [aa_nd] current iterate
  void* aa_gt;            // [(aa_m + 1) * aa_nt] the same for the row values, sweep precision
  void* aa_ft;            // [(aa_m + 1) * aa_nt]
  void* aa_xct;           // [aa_nt]
  double* aa_gram;        // [(aa_m + 1)^2] residual Gram matrix by slot
  double* aa_coef;        // [8] mixing coefficients
  int* aa_k;              // [2] Anderson step; the step being mixed
  int* nonfinite;         // [1]
};

// A unit of sweep work: ordinates [o0, o0 + count) of one octant of one geometry.
struct WorkItem {
  int geom;
  int octant;   // bit0: p_x < 0, bit1: p_y < 0, bit2: p_z < 0
  int o0;
  int count;
  int d0;       // start step: row j' visits column (d + d0 - j' - k') mod nx
};

struct SweepLaunch {
  const GeomDev* geoms;
  const WorkItem* items;
  int n_items;
  int flags;
  int* item_counter;  // persistent work queue (nullptr: one item per block)
};

// sweep.cu (generic block kernel) and the 2D warp kernel (sweep_w*.cu)
cudaError_t launch_sweep2d_warp(const SweepLaunch& L, int precision, int G, int RMAX, bool has_s,
                                bool rfixed, int blocks, cudaStream_t st);
bool sweep2d_warp_exists(int precision, int G, int RMAX, bool has_s, bool rfixed);
// 3D block kernel (sweep3d.cuh)
cudaError_t launch_sweep3d(const SweepLaunch& L, int precision, int G, int RMAX, bool has_s,
                           int threads, size_t smem, cudaStream_t st);
bool sweep3d_exists(int precision, int G, int RMAX, bool has_s);
size_t sweep3d_smem_bytes(int precision, int G, int RMAX, int threads);
int sweep2d_warps_per_block(int precision, int G, int RMAX, bool has_s, bool rfixed);
// 2D warp kernel with two-warp groups (rows fill 64 lanes; eight warps, four
// groups per block; FP32 without s(x))
cudaError_t launch_sweep2d_split(const SweepLaunch& L, int precision, int G, int RMAX, int blocks,
                                 cudaStream_t st);
bool sweep2d_split_exists(int precision, int G, int RMAX);
cudaError_t launch_sweep(const SweepLaunch& L, int precision, int dim, int G, int RMAX,
                         bool has_s, int threads, int blocks, size_t smem, cudaStream_t st);
size_t sweep_smem_bytes(int precision, int dim, int G, int RMAX, int threads);
bool sweep_variant_exists(int precision, int dim, int G, int RMAX, bool has_s);
int sweep_blocks_per_sm(int precision, int dim, int G, int RMAX, bool has_s, int threads,
                        size_t smem);

// finalize.cu
constexpr int kMaxPartBlocks = 1216;  // blocks of the finalize / Anderson reductions
// finalize_kernel then its one-warp tail (kappa, stopping test)
cudaError_t launch_finalize(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                            cudaStream_t st);
// Anderson acceleration (anderson.cu)
cudaError_t launch_anderson_init(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                                 cudaStream_t st);
cudaError_t launch_anderson_step(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                                 cudaStream_t st);
// build the skewed records and record indices (after the state is initialised)
cudaError_t launch_build_records(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                                 cudaStream_t st);
constexpr int kMaxSkewCells = 1 << 22;
// state at iteration 0 from each geometry's T0, geometries geoms_dev[0 .. n_geoms);
// max_work = max over them of max(6 n_cells, n_ord rows), max_walls likewise
cudaError_t launch_init_state(const GeomDev* geoms_dev, int n_geoms, long max_work, int max_walls,
                              int precision, cudaStream_t st);
// ordinate sharding: the moment partials of a sweep out of / back into the
// accumulators (layout: T_L numerator [n_cells], wall numerators [n_walls],
// hot-face flux [1]); one geometry
cudaError_t launch_shard_export(const GeomDev* geoms_dev, double* out, int blocks, cudaStream_t st);
cudaError_t launch_shard_import(const GeomDev* geoms_dev, const double* in, int blocks,
                                cudaStream_t st);
// deviation form: rebuild the records' upwind-difference fields from T_L and
// T_w (after the finalisation and the Anderson mix); no-op for other geometries
cudaError_t launch_psi_records(const GeomDev* geoms_dev, int n_geoms, int precision, int blocks,
                               cudaStream_t st);
cudaError_t launch_gauge(const uint8_t* code, const double* TL, int n, double* out,
                         double* mean_out, cudaStream_t st);
// psi: the recorded fields are deviations T_o - T_L (deviation-form sweeps)
cudaError_t launch_grad_contract2(const uint8_t* code, const double* TL, int n, const void* rec,
                                  int n_rec, const int* rev_local, const double* a_rec,
                                  double jscale, double* grad, int precision, int psi,
                                  cudaStream_t st);

// fourier.cu
// arguments of one Fourier CG solve
struct CGArgs {
  const uint8_t* code;
  int nx, ny, nz, dim, py, pz;
  double wx, wy, wz, dT;
  int max_iter;
  double tol;
  double* x;
  double* r;
  double* p;
  double* q;
  double* part;   // [2][gridDim]
  double* T_out;  // [n] solution, mean 0, 0 in pores
  int* iters_out;
};
CGArgs make_cg_args(const GeomDev& g, double hx, double hy, double hz, int max_iter, double tol,
                    double* T_out, int* iters_out, double* work, int blocks_max);
// one thread-block cluster per job (FP32; every job's rows must fit the
// cluster's shared memory); cudaErrorNotSupported when it does not apply
cudaError_t launch_fourier_cg_cluster_jobs(const CGArgs* jobs_dev, const CGArgs* jobs_host, int n_jobs,
                                           int precision, cudaStream_t st);
// one block per job (geometries up to kBlockCGMaxCells cells)
cudaError_t launch_fourier_cg_blocks(const CGArgs* jobs_dev, int n_jobs, int precision,
                                     cudaStream_t st);
constexpr int kBlockCGMaxCells = 1 << 18;
cudaError_t launch_fourier_cg(const GeomDev& g, double hx, double hy, double hz, int precision,
                              int max_iter, double tol, double* T_out, int* iters_out,
                              double* work, int blocks_max, cudaStream_t st);
size_t fourier_work_doubles(int n_cells, int blocks_max);
// sum over the hot-contact rows of (T_image + dT - T_cell), one block
cudaError_t launch_fourier_hot_flux(const uint8_t* code, const double* T, int nx, int rows, double dT,
                                   double* out, cudaStream_t st);

/*
 * obte.h -- C ABI of libobte, a GB300 (sm_103a) solver for the steady-state
 * anisotropic-mean-free-path phonon Boltzmann transport equation (aMFP-BTE)
 * on periodic Cartesian voxel meshes, after OpenBTE (G. Romano, arXiv
 * 2106.02764).
 *
 * What is solved (App. A of the paper, upwind finite volumes, Eq. iter2):
 * for every ordinate o = (MFP bin m, direction s) and every solid cell i
 *
 *   (s_i + sum_a Lambda_m |p_a| / h_a) T_oi
 *       - sum_{inflow faces} (Lambda_m |p_a| / h_a) u_o  =  s_i T_Li
 *
 * where u_o is the upwind value across the face: the neighbour's T_o (plus
 * the applied jump +dT / -dT across the low / high side of the periodic x
 * period, the P term of App. A), or the temperature of a diffuse wall face.
 * The lattice temperature is T_L = sum_o a_o T_o with
 * a_o = w_s (kappa_m / Lambda_m^2) / sum_m' (kappa_m' / Lambda_m'^2) (Sec. 2),
 * every wall face thermalises to the flux-weighted mean of the ordinates
 * leaving into it (Sec. 2, R_mu_nu), with flux weights
 * K_o = d_ang kappa_m w_s p_s / Lambda_m, and kappa_eff is the upwinded heat
 * flux through the solid faces of the plane x = 0 (Eq. keff, hot-contact form
 * of App. A) times L_x / (dT * cross-section).  The system is iterated to its
 * fixed point as in Algorithm 1 (Sec. 3), starting from a Fourier solution
 * (App. B).
 *
 * Conventions
 *  - Every function returns an obte_status; obte_last_error() gives a message.
 *  - The caller owns every host array; the library copies what it needs and
 *    keeps no caller pointer.
 *  - Device memory is taken only through obte_device_cfg.alloc/free when they
 *    are given (cudaMalloc/cudaFree otherwise) and work is enqueued on
 *    obte_device_cfg.cuda_stream (a cudaStream_t; NULL = a stream the library
 *    creates).  Functions that return results to host memory synchronise that
 *    stream.
 *  - Call order: create -> create_mesh -> set_material -> [set_scattering_scale]
 *    -> solve -> get_* / kappa_grad_s.  Out of order: OBTE_ESTATE.
 *  - One context per host thread at a time.
 *  - Lengths are in metres, conductivities in W/m/K, temperatures in K.
 */
#ifndef OBTE_H
#define OBTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct obte_ctx obte_ctx;

typedef enum {
  OBTE_OK = 0,
  OBTE_EINVAL = -1,         /* invalid argument (message says which)            */
  OBTE_ESTATE = -2,         /* call out of order                                */
  OBTE_ECUDA = -3,          /* a CUDA call failed                               */
  OBTE_ENOMEM = -4,         /* device allocation failed                         */
  OBTE_NOT_CONVERGED = -5,  /* max_iter reached; results are readable           */
  OBTE_ENONFINITE = -6,     /* NaN or Inf in the inputs or in the iterate       */
  OBTE_ETIMEOUT = -7        /* reserved: a bounded device-side wait expired      */
} obte_status;

typedef enum { OBTE_FP64 = 0, OBTE_MIXED = 1 } obte_precision;

typedef struct {
  void* (*alloc)(size_t bytes, void* user); /* NULL: cudaMalloc                  */
  void (*free)(void* ptr, void* user);      /* NULL: cudaFree                    */
  void* user;
  void* cuda_stream;                        /* cudaStream_t, NULL: library stream */
  int device;                               /* CUDA device ordinal               */
} obte_device_cfg;

typedef struct {
  int precision;        /* obte_precision.  FP64: every step in double.  MIXED:
                           transport sweeps in float, carrying deviations
                           psi = T - T_L: the upwind differences u - T_L of
                           neighbour, wall and periodic-image values (the
                           applied jump dT included) are formed in double
                           and rounded once, psi = sum_a A_a (u_a - T_L), so
                           the weight of T_L is exactly 1 - sum_a A_a and no
                           float value carries T_L itself; T_L, flux, kappa
                           (its jump part dT sum K_x and its T_L part
                           included) and wall sums and the convergence test
                           in double                                          */
  double tol;           /* stop when |kappa_n - kappa_{n-1}| <= tol |kappa_n|
                           (Algorithm 1); <= 0 disables                        */
  double tol_TL;        /* and max_i |T_L,n - T_L,n-1| <= tol_TL (K); <= 0 off  */
  int max_iter;         /* iteration cap; reaching it gives OBTE_NOT_CONVERGED  */
  int min_iter;         /* never stop before this many iterations              */
  int check_every;      /* iterations per CUDA-graph launch between host checks */
  int fourier_max_iter; /* CG iterations for the Fourier first guess (0: auto) */
  double fourier_tol;   /* relative CG residual (0: 1e-3)                      */
  int group_size;       /* ordinates per group (0: chosen by rule, or by an
                           earlier timed choice for the same mesh shape;
                           -1: timed choice among the compiled variants,
                           for a batch among its launch forms)           */
  int rows_per_thread;  /* mesh rows per thread or lane (0: chosen by rule) */
  int use_graph;        /* 1: capture check_every iterations in a CUDA graph   */
  int profile;          /* 1: time every sweep / finalize launch with CUDA
                           events recorded on the solve stream (stats below)   */
  int kernel;           /* 0: automatic, 1: plain block kernel (every dimension),
                           2: 2D warp-per-group kernel, 3: 3D block kernel
                           with skewed cell records                            */
  int accel;            /* Anderson acceleration window (0: plain source
                           iteration as in Algorithm 1; 1..7: mix the last
                           accel iterates of (T_L, T_w, carried row values);
                           same fixed point; with mixing two consecutive
                           kappas can agree by chance, so pair tol with
                           tol_TL at large windows)                            */
} obte_solve_opts;

#define OBTE_MAX_HISTORY 4096

typedef struct {
  int iterations;             /* source iterations run                            */
  int fourier_iterations;     /* CG iterations of the first guess                 */
  int converged;              /* 1 if the stopping test passed                    */
  double kappa_eff;           /* W/m/K                                            */
  double delta_TL;            /* max |T_L,n - T_L,n-1| of the last iteration (K)  */
  double time_fourier_ms;     /* device time of the first guess                   */
  double time_iter_ms;        /* device time of the source iterations             */
  double time_total_ms;       /* device time of obte_solve                        */
  double updates_per_s;       /* N_solid * N_ordinates * iterations / time_iter   */
  int group_size, rows_per_thread, threads_per_block, n_groups;
  int kernel;                 /* 1: block kernel, 2: 2D warp-per-group kernel,
                                 3: 3D block kernel with skewed cell records      */
  int n_sweeps;               /* sweep launches timed when opts.profile = 1       */
  double time_sweep_ms;       /* summed device time of those sweep launches       */
  double time_finalize_ms;    /* summed device time of the finalize launches      */
  int n_history;              /* entries of kappa_history                         */
  double kappa_history[OBTE_MAX_HISTORY];
} obte_solve_stats;

/* Fill opts with defaults: FP64, tol 1e-6, max_iter 2000, check_every 8. */
void obte_default_opts(obte_solve_opts* opts);

/* Create a context on cfg->device.  cfg may be NULL (defaults: device 0). */
int obte_create(obte_ctx** out, const obte_device_cfg* cfg);

/* Mesh and geometry (Sec. 6; App. A, R_ij, R^P_ij, g_si).
 *  dim        2 or 3 (2: nz must be 1 and lz is ignored)
 *  nx,ny,nz   cells per axis; lx,ly,lz domain lengths (m)
 *  solid_mask host uint8 [nz][ny][nx] (x fastest), nonzero = solid, 0 = pore
 *  periodic   host int[3]; 1 = periodic axis, 0 = diffuse walls at both ends
 *  grad_axis  axis of the applied temperature jump (must be periodic)
 *  delta_T    applied jump across one period (K), nonzero
 * After mapping grad_axis to the sweep's x axis, a periodic y (z) axis needs
 * ny (nz) to be a multiple of nx; OBTE_EINVAL otherwise. */
int obte_create_mesh(obte_ctx* ctx, int dim, int nx, int ny, int nz, double lx, double ly,
                     double lz, const uint8_t* solid_mask, const int periodic[3],
                     int grad_axis, double delta_T);

/* Material and angular quadrature (Sec. 5; aMFP interpolation of App. A,
 * F_ml = Lambda_m s_l).
 *  kappa_m, lambda_m  host double[n_mfp]: bin conductivity (W/m/K), MFP (m) > 0
 *  dirs               host double[n_dir][3]: directions; in 2D only x, y are
 *                     used (projected directions may have |p| < 1)
 *  w                  host double[n_dir]: weights, sum 1
 *  angular_dim        2 (in-plane circle) or 3 (sphere-based sets)
 * The direction set must be symmetric under p -> -p and under each axis
 * mirror, as every wall must conserve energy (OBTE_EINVAL otherwise). */
int obte_set_material(obte_ctx* ctx, int n_mfp, const double* kappa_m, const double* lambda_m,
                      int n_dir, const double* dirs, const double* w, int angular_dim);

/* General aMFP material (Sec. 5: the Material module turns mode data into
 * per-ordinate quantities; App. A: F_ml = Lambda_m s_l with the weights D_ml
 * and S_ml interpolated from the modes).  Every ordinate o carries its own
 * vectorial MFP and weight, so MFPs may depend on direction (anisotropic
 * materials) and weights need not factor into bin x direction.
 *  lambda   host double[n_ord]: Lambda_o (m) > 0
 *  dirs     host double[n_ord][3]: s_o (in 2D only x, y are used; projected
 *           directions may have |s| < 1)
 *  weight   host double[n_ord]: W_o >= 0, the C/tau of the modes the ordinate
 *           stands for (any common scale), not all zero
 *  bin      host int[n_ord] in [0, n_bins) or NULL (one bin): the MFP bin of
 *           each ordinate, for obte_get_kappa_bins and the adjoint's pairing
 * Lattice-temperature weights a_o = W_o / sum W (E2); flux weights K_o =
 * W_o Lambda_o s_o, the form for which every ordinate's transport conserves
 * energy (sum_o K_o . grad T_o = -sum_o W_o (T_o - T_L) = 0).  The
 * bin-separable obte_set_material is the case W_o = d_ang (kappa_m /
 * Lambda_m^2) w_s.  Bulk conductivity along axis a: sum_o W_o Lambda_o^2
 * s_oa^2 (the first guess and obte_solve_fourier use these as an axis-aligned
 * tensor).  The set must be mirror-symmetric like obte_set_material's
 * (OBTE_EINVAL otherwise); obte_kappa_grad_s also needs for every ordinate a
 * reversed one (same bin, Lambda and weight, opposite direction).
 * OBTE_ENONFINITE for non-finite input; OBTE_EINVAL for lambda <= 0, a
 * negative weight, an all-zero weight vector, a bin out of range, or no
 * ordinate moving along the gradient axis. */
int obte_set_material_ordinates(obte_ctx* ctx, int n_ord, const double* lambda, const double* dirs,
                                const double* weight, const int* bin, int n_bins);

/* Per-cell scattering scale s_i > 0 multiplying the collision term of every
 * ordinate in cell i (not in the paper; used for sensitivities).
 * s: host double[nz][ny][nx] or NULL (all ones); pore entries are ignored.
 * Needs create_mesh (OBTE_ESTATE otherwise); a solid entry that is not finite
 * gives OBTE_ENONFINITE, one <= 0 OBTE_EINVAL.  Invalidates earlier results. */
int obte_set_scattering_scale(obte_ctx* ctx, const double* s);

/* Fourier first guess then source iteration to the fixed point (Algorithm 1).
 * opts NULL: defaults.  stats may be NULL.  Returns OBTE_NOT_CONVERGED when
 * max_iter is reached (results still readable). */
int obte_solve(obte_ctx* ctx, const obte_solve_opts* opts, obte_solve_stats* stats);

/* Several independent geometries (each its own context on the same device and
 * stream) iterated together: one persistent launch per iteration over a work
 * list of (geometry, ordinate group) items, or in mixed precision one launch
 * per class of geometries with the same rows per lane, the iteration captured
 * in a CUDA graph, per-geometry convergence.  opts->group_size = -1 times the
 * launch forms the batch accepts (class launches, persistent warp queue,
 * persistent block kernel) over a few iterations each, keeps the fastest for
 * this batch shape and solves with it; the timing runs overwrite the
 * contexts' state before the solve.  stats: array of n or NULL. */
int obte_solve_batch(obte_ctx* const* ctxs, int n, const obte_solve_opts* opts,
                     obte_solve_stats* stats);

/* Getters below: ctx or out NULL gives OBTE_EINVAL; before a solve (or after
 * an input change that invalidates it) OBTE_ESTATE.  Arrays are written in
 * the caller's axis order (x fastest), whatever axis the gradient was on. */

/* Lattice temperature of the last solve, gauged to zero mean over the solid
 * cells: host double[nz][ny][nx], NaN in pores. */
int obte_get_T_L(obte_ctx* ctx, double* out);

/* Heat flux J = sum_o K_o T_o (Sec. 2) per cell: host double[nz][ny][nx][dim]
 * (W/m^2), NaN in pores.  Runs one extra sweep the first time it is called. */
int obte_get_flux(obte_ctx* ctx, double* out);

/* kappa_eff of the last solve (W/m/K). */
int obte_get_kappa_eff(obte_ctx* ctx, double* out);

/* Net x-flux through every section x = const of the kernel frame (conservation
 * diagnostic; equal at the fixed point): host double[n_sections], n_sections
 * = cells along the gradient axis.  Runs with obte_get_flux's extra sweep. */
int obte_get_section_flux(obte_ctx* ctx, double* out);

/* d kappa_eff / d s_i for every cell after obte_solve: host double[nz][ny][nx],
 * 0 in pores.  The adjoint of the discrete system is the same upwind transport
 * with every direction reversed (transposed ordinate direction, reverse
 * wavefront order) and the applied jump replaced by the kappa functional; the
 * adjoint fields are produced by sweeps in reversed direction and contracted
 * with the forward fields group by group, so device memory stays bounded by
 * max_field_bytes (0: 1 GiB). */
int obte_kappa_grad_s(obte_ctx* ctx, double* out, size_t max_field_bytes);

/* d kappa_eff / d s_i like obte_kappa_grad_s, for callers that cannot allocate
 * device memory at the time they need it: a service that reserves its whole
 * device-memory budget at start-up and whose allocator refuses new blocks
 * afterwards, or an optimisation loop sharing a full GPU with other jobs,
 * where allocating the recorded fields could fail in the middle of a run.
 * This call allocates nothing: the recorded ordinate fields, the gradient
 * accumulator and the small index tables live in a fixed 32 MiB device array
 * inside the library (held by every GPU that loads the library until the
 * process exits).  The context's own buffers, made by earlier calls, are
 * reused.  out: host double[nz][ny][nx], 0 in pores.  Returns OBTE_EINVAL
 * with a message when the gradient, the ordinate tables and one reversed pair
 * of ordinate fields do not fit in the 32 MiB; larger problems run as several
 * batches of ordinate pairs.  The call blocks the host: it synchronises the
 * context's stream after every batch and copies small index tables from
 * pageable host memory, so that stream must not be under stream capture.  The
 * first call on a device takes the array's device address
 * (cudaGetSymbolAddress).  Every call shares the one array and overwrites it:
 * calls whose work overlaps on the GPU (other threads, other contexts on other
 * streams) race and must be serialised by the caller.  The paper has no
 * counterpart to this entry point. */
int obte_kappa_grad_s_noalloc(obte_ctx* ctx, double* out);

/* Ordinate sharding of one solve across processes or devices (Sec. 3: the
 * paper spreads the phonon directions over MPI processes; within an iteration
 * the ordinates are independent, and the only exchange is a sum of the FP64
 * moment partials).  Each rank holds the whole mesh and material and sweeps
 * the runs of ordinate groups r with r mod n_ranks == rank.  Per iteration:
 *
 *   obte_shard_sweep(ctx, buf)      enqueue this rank's sweep on ctx's stream
 *                                   and write its partials to buf
 *   (caller) sum buf over the ranks (an all-reduce; between contexts on one
 *            device, a device add)
 *   obte_shard_finalize(ctx, sum, &done)
 *                                   T_L, T_w, kappa and the stopping test from
 *                                   the summed partials; blocks until done
 *
 * Every rank computes the same finalisation from the same sums, so all ranks
 * hold the same T_L, T_w and kappa and stop at the same iteration.  buf and
 * sum are device arrays of obte_shard_partials_count(ctx) doubles on ctx's
 * device, owned by the caller:
 *   [0, n_cells)                    T_L numerator sum_o a_o T_o per cell (E2;
 *                                   0 in pores), cell order x fastest
 *   [n_cells, n_cells + n_walls)    E3 numerator of each wall face
 *   [n_cells + n_walls]             hot-face flux through x = 0 (Eq. keff)
 * obte_set_shard (rank in [0, n_ranks)) comes after set_material and before
 * obte_shard_begin; n_ranks = 1 makes the context whole again.  obte_shard_begin
 * takes the solve options like obte_solve, with group_size >= 0 (every rank
 * must pick the same variant) and accel = 0 (the plain source iteration of
 * Algorithm 1), and runs the Fourier first guess.  *done after
 * obte_shard_finalize: 0 running, 1 converged, 2 max_iter reached, 3
 * non-finite (the call then returns OBTE_ENONFINITE).  After any finalize,
 * obte_get_T_L and obte_get_kappa_eff give the (full) current iterate;
 * obte_get_flux, obte_get_section_flux and obte_get_kappa_bins give this
 * rank's ordinates' share, whose sum over the ranks is the full output.  On a
 * sharded context obte_solve, obte_solve_batch and the gradient return
 * OBTE_ESTATE. */
int obte_set_shard(obte_ctx* ctx, int rank, int n_ranks);
size_t obte_shard_partials_count(const obte_ctx* ctx);
int obte_shard_begin(obte_ctx* ctx, const obte_solve_opts* opts);
int obte_shard_sweep(obte_ctx* ctx, double* partials);
int obte_shard_finalize(obte_ctx* ctx, const double* partials, int* done);

/* Per-MFP-bin contribution to kappa_eff (the aMFP analogue of the
 * mode-resolved conductivity, App. A): host double[n_mfp]; sums to kappa_eff.
 * Runs with obte_get_flux's extra sweep. */
int obte_get_kappa_bins(obte_ctx* ctx, double* out);

/* Fourier model alone (App. B; the paper's Fourier-only run): heat
 * conduction with the bulk conductivity (kappa_bulk = sum_m kappa_m for
 * obte_set_material, the axis-aligned tensor of obte_set_material_ordinates)
 * in the solid cells, adiabatic pore and film walls, and the applied jump dT across
 * the gradient period, solved by FP64 conjugate gradients on the device (the
 * solver's first guess run to a tight tolerance).  Needs create_mesh and
 * set_material; leaves the transport solve's state untouched.
 *   tol        relative CG residual, |r| <= tol |b| (0: 1e-12)
 *   max_iter   CG iterations (0: 40 (nx + ny + nz))
 *   kappa_out  host double: kappa_fourier in W/m/K = L / (dT A_sec) x the
 *              conductive flux through the solid faces of the plane x = 0
 *              (App. B, last equation; A_sec the full cross-section)
 *   T_out      host double[nz][ny][nx] or NULL: the temperature, solid-cell
 *              mean 0, NaN in pores
 *   iters_out  host int or NULL: CG iterations taken
 * Device scratch (5 doubles per cell) comes from the context's allocator and
 * is freed before the call returns.  OBTE_NOT_CONVERGED when the residual
 * test is not met within max_iter (the outputs are still written). */
int obte_solve_fourier(obte_ctx* ctx, double tol, int max_iter, double* kappa_out, double* T_out,
                       int* iters_out);

/* Measured FMA throughput of a device, in flop/s (2 per FMA): precision
 * OBTE_MIXED times FP32 FMAs, OBTE_FP64 FP64 FMAs, in a kernel of independent
 * FMA chains over every SM (a few ms).  The ALU roof of the sweep, for the
 * roofline beside the peak derived from unit counts and clocks.  Needs no
 * context; allocates nothing.  The paper has no counterpart (a measurement
 * utility). */
int obte_measure_fma_rate(int precision, int device, double* flops_per_s);

/* Message of the last failing call on ctx ("" if none has failed; "null
 * context" for NULL).  The pointer stays valid until the next failing call on
 * ctx or obte_destroy. */
const char* obte_last_error(const obte_ctx* ctx);

/* Wait for the context's stream, then release every device buffer (through
 * the allocator's free callback where one was given), the cached iteration
 * graph and a stream the library created.  NULL is a no-op. */
void obte_destroy(obte_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* OBTE_H */

// Host implementation of the libobte C ABI (include/obte.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "obte.h"
#include "obte_internal.h"

namespace {

constexpr int kMaxHist = OBTE_MAX_HISTORY;
constexpr int kFourierBlocksMax = 1024;
constexpr double kFourierTolDefault = 1e-3;  // relative CG residual of the first guess

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct obte_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* (*alloc_fn)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* user = nullptr;
  std::string err;
  std::vector<DevBuf> bufs;

  // mesh (kernel frame: x = gradient axis)
  bool has_mesh = false, has_material = false, solved = false;
  int dim = 2, n[3] = {1, 1, 1}, perm[3] = {0, 1, 2}, user_n[3] = {1, 1, 1};
  double len[3] = {0, 0, 0}, h[3] = {1, 1, 1};
  int periodic[3] = {1, 1, 1};
  double dT = 1.0;
  int n_cells = 0, n_solid = 0, n_walls = 0;
  std::vector<uint8_t> code_h;
  std::vector<int> wall_id_h, wall_cell_h, wall_side_h;
  uint8_t* code_d = nullptr;
  int* wall_id_d = nullptr;
  int* wall_cell_d = nullptr;
  int* wall_side_d = nullptr;
  double* s_d = nullptr;
  bool has_s = false;

  // material: sorted ordinate table
  int M = 0, S = 0, O = 0, d_ang = 2;
  std::vector<double> kappa_m, lambda_m;
  std::vector<int> ord_m, ord_s, octant;          // sorted order
  std::vector<double> bx, by, bz, diag, inv, aw, kxa, kya, kza;
  std::vector<double> pk[3];                      // kernel-frame direction per sorted ordinate
  double* wall_den_d = nullptr;
  std::vector<double> wall_den_h;
  void* tab_d[2][9] = {{nullptr}};                // [precision][table]
  int* mbin_d = nullptr;
  int* octant_d = nullptr;
  int* ord_d0_d = nullptr;
  double kappa_scale = 0.0, sum_k_over_l2 = 0.0;
  double w_total = 0.0;                           // sum of the E2 weights before normalisation
  double kappa_axes[3] = {0, 0, 0};               // bulk conductivity along each kernel axis
  std::vector<double> lam_o;                      // Lambda per sorted ordinate
  std::vector<int> rev_o;                         // reversed sorted ordinate, -1 if none

  // solve state
  int precision = -1;
  GeomDev gh{};
  GeomDev* gd = nullptr;
  double* TL = nullptr;
  double* TL_acc = nullptr;
  void* src = nullptr;
  void* twc = nullptr;
  CGArgs* cg_job = nullptr;
  int aa_m_alloc = -1;
  int rec_w_alloc = 0;
  double *aa_xd = nullptr, *aa_fd = nullptr, *aa_small = nullptr;
  void *aa_xt = nullptr, *aa_ft = nullptr;
  int* aa_int = nullptr;
  void* rec4 = nullptr;
  int* rec_idx = nullptr;
  double* tlq = nullptr;
  double* blk_part = nullptr;  // per-block partials of the finalize / Anderson reductions
  double* Tw = nullptr;
  double* wall_acc = nullptr;
  void* front = nullptr;
  double* scal = nullptr;    // phi_acc, delta_max[2]
  int* ctrl = nullptr;       // done, iter, nonfinite
  double* hist = nullptr;
  double* TF = nullptr;
  double* fwork = nullptr;
  int* fiters = nullptr;
  double* J_acc = nullptr;
  double* phi_sec = nullptr;
  double* phi_bin = nullptr;
  bool flux_done = false;
  int G = 0, R = 0, threads = 0;
  bool warp = false;
  bool k3d = false;
  int nh = 1;  // warps per group of the 2D warp kernel
  int items_pad = 1;  // 4: items padded for the warp kernel's block-combined moments
  std::vector<WorkItem> items_h;
  WorkItem* items_d = nullptr;
  double kappa = NAN;
  int last_iters = 0;
  // cached iteration graph (reused by later solves with the same launch shape)
  cudaGraphExec_t it_exec = nullptr;
  std::vector<cudaEvent_t> it_events;
  long long it_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  void drop_graph() {
    if (it_exec) cudaGraphExecDestroy(it_exec);
    it_exec = nullptr;
    for (auto& e : it_events) cudaEventDestroy(e);
    it_events.clear();
  }
  obte_solve_opts last_opts{};
  // ordinate sharding: this context sweeps the runs of work items r with
  // r mod shard_n == shard_rank (obte_set_shard); shard_active after
  // obte_shard_begin
  int shard_rank = 0, shard_n = 1;
  bool shard_active = false;

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (alloc_fn) {
      p = alloc_fn(bytes, user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) bufs.push_back({p, bytes});
    return p;
  }
  void dfree(void* p) {
    if (!p) return;
    bool owned = false;
    for (size_t i = 0; i < bufs.size(); ++i)
      if (bufs[i].p == p) {
        bufs.erase(bufs.begin() + i);
        owned = true;
        break;
      }
    if (!owned) return;  // never free what this context did not allocate
    if (free_fn) free_fn(p, user);
    else cudaFree(p);
  }
  void forget_pointers() {
    code_d = nullptr;
    wall_id_d = nullptr;
    wall_cell_d = nullptr;
    wall_side_d = nullptr;
    twc = nullptr;
    cg_job = nullptr;
    aa_m_alloc = -1;
    rec_w_alloc = 0;
    aa_xd = aa_fd = aa_small = nullptr;
    aa_xt = aa_ft = nullptr;
    aa_int = nullptr;
    rec4 = nullptr;
    rec_idx = nullptr;
    tlq = nullptr;
    blk_part = nullptr;
    s_d = nullptr;
    wall_den_d = nullptr;
    for (auto& a : tab_d)
      for (auto& b : a) b = nullptr;
    mbin_d = octant_d = ord_d0_d = nullptr;
    gd = nullptr;
    TL = TL_acc = Tw = wall_acc = scal = hist = TF = fwork = J_acc = phi_sec = phi_bin = nullptr;
    src = front = nullptr;
    ctrl = fiters = nullptr;
    items_d = nullptr;
    items_h.clear();
    precision = -1;
  }
  template <typename T>
  T* dalloc_t(size_t count) {
    return reinterpret_cast<T*>(dalloc(count * sizeof(T)));
  }
  int fail(int code, const std::string& m) {
    err = m;
    return code;
  }
  int cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return OBTE_ECUDA;
  }
};

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call); \
  } while (0)

#define NEED(ptr)                                                              \
  do {                                                                         \
    if (!(ptr)) return ctx->fail(OBTE_ENOMEM, "device allocation failed: " #ptr); \
  } while (0)

extern "C" void obte_default_opts(obte_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = OBTE_FP64;
  o->tol = 1e-6;
  o->tol_TL = 0.0;
  o->max_iter = 2000;
  o->min_iter = 2;
  o->check_every = 8;
  o->fourier_max_iter = 0;
  o->fourier_tol = 0.0;
  o->group_size = 0;
  o->rows_per_thread = 0;
  o->use_graph = 1;
  o->profile = 0;
  o->kernel = 0;
  o->accel = 0;
}

extern "C" int obte_create(obte_ctx** out, const obte_device_cfg* cfg) {
  if (!out) return OBTE_EINVAL;
  *out = nullptr;
  obte_ctx* ctx = new obte_ctx();
  if (cfg) {
    ctx->device = cfg->device;
    ctx->alloc_fn = cfg->alloc;
    ctx->free_fn = cfg->free;
    ctx->user = cfg->user;
    ctx->stream = reinterpret_cast<cudaStream_t>(cfg->cuda_stream);
  }
  if ((ctx->alloc_fn == nullptr) != (ctx->free_fn == nullptr)) {
    ctx->err = "alloc and free must be given together";
    *out = ctx;
    return OBTE_EINVAL;
  }
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) {
    ctx->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    *out = ctx;
    return OBTE_ECUDA;
  }
  if (!ctx->stream) {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      ctx->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
      *out = ctx;
      return OBTE_ECUDA;
    }
    ctx->own_stream = true;
  }
  *out = ctx;
  return OBTE_OK;
}

extern "C" const char* obte_last_error(const obte_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

static void free_all(obte_ctx* ctx) {
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  while (!ctx->bufs.empty()) ctx->dfree(ctx->bufs.back().p);
  ctx->forget_pointers();
}

extern "C" void obte_destroy(obte_ctx* ctx) {
  if (!ctx) return;
  ctx->drop_graph();
  free_all(ctx);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
extern "C" int obte_create_mesh(obte_ctx* ctx, int dim, int nx, int ny, int nz, double lx,
                                double ly, double lz, const uint8_t* mask, const int periodic[3],
                                int grad_axis, double delta_T) {
  if (!ctx) return OBTE_EINVAL;
  if (dim != 2 && dim != 3) return ctx->fail(OBTE_EINVAL, "dim must be 2 or 3");
  if (dim == 2) {
    if (nz != 1) return ctx->fail(OBTE_EINVAL, "2D mesh needs nz = 1");
    lz = 1.0;
  }
  if (nx < 1 || ny < 1 || nz < 1) return ctx->fail(OBTE_EINVAL, "cell counts must be positive");
  if ((long)nx * ny * nz > (1L << 30)) return ctx->fail(OBTE_EINVAL, "mesh too large");
  if (!(lx > 0) || !(ly > 0) || !(lz > 0) || !std::isfinite(lx) || !std::isfinite(ly) ||
      !std::isfinite(lz))
    return ctx->fail(OBTE_EINVAL, "lengths must be positive and finite");
  if (!mask || !periodic) return ctx->fail(OBTE_EINVAL, "mask and periodic are required");
  if (grad_axis < 0 || grad_axis >= dim) return ctx->fail(OBTE_EINVAL, "grad_axis out of range");
  if (!periodic[grad_axis]) return ctx->fail(OBTE_EINVAL, "the gradient axis must be periodic");
  if (!(delta_T != 0.0) || !std::isfinite(delta_T)) return ctx->fail(OBTE_EINVAL, "delta_T must be nonzero and finite");
  ctx->drop_graph();
  if (ctx->solved || ctx->has_mesh) free_all(ctx);
  ctx->has_mesh = ctx->has_material = ctx->solved = false;
  ctx->precision = -1;
  ctx->flux_done = false;

  const int un[3] = {nx, ny, nz};
  const double ul[3] = {lx, ly, lz};
  // kernel axis k <- user axis perm[k]: gradient first, the others in order
  int perm[3] = {grad_axis, 0, 0};
  int k = 1;
  for (int a = 0; a < 3; ++a)
    if (a != grad_axis) perm[k++] = a;
  if (dim == 2) {  // keep z as the third axis
    perm[0] = grad_axis;
    perm[1] = 1 - grad_axis;
    perm[2] = 2;
  }
  for (int i = 0; i < 3; ++i) {
    ctx->perm[i] = perm[i];
    ctx->n[i] = un[perm[i]];
    ctx->len[i] = ul[perm[i]];
    ctx->periodic[i] = (dim == 2 && i == 2) ? 1 : (periodic[perm[i]] ? 1 : 0);
    ctx->h[i] = ctx->len[i] / ctx->n[i];
    ctx->user_n[i] = un[i];
  }
  ctx->dim = dim;
  ctx->dT = delta_T;
  const int Nx = ctx->n[0], Ny = ctx->n[1], Nz = ctx->n[2];
  if (ctx->periodic[1] && Ny % Nx != 0)
    return ctx->fail(OBTE_EINVAL, "a periodic y axis needs ny to be a multiple of nx (kernel frame)");
  if (dim == 3 && ctx->periodic[2] && Nz % Nx != 0)
    return ctx->fail(OBTE_EINVAL, "a periodic z axis needs nz to be a multiple of nx (kernel frame)");
  ctx->n_cells = Nx * Ny * Nz;

  // solid flags in the kernel frame
  std::vector<uint8_t> solid(ctx->n_cells);
  for (int z = 0; z < Nz; ++z)
    for (int y = 0; y < Ny; ++y)
      for (int x = 0; x < Nx; ++x) {
        int u[3];
        const int kc[3] = {x, y, z};
        for (int i = 0; i < 3; ++i) u[perm[i]] = kc[i];
        const long ui = u[0] + (long)un[0] * (u[1] + (long)un[1] * u[2]);
        solid[x + Nx * (y + Ny * z)] = mask[ui] ? 1 : 0;
      }
  ctx->code_h.assign(ctx->n_cells, 0);
  ctx->wall_id_h.assign((size_t)ctx->n_cells * 6, -1);
  ctx->wall_cell_h.clear();
  ctx->wall_side_h.clear();
  ctx->n_solid = 0;
  for (int z = 0; z < Nz; ++z)
    for (int y = 0; y < Ny; ++y)
      for (int x = 0; x < Nx; ++x) {
        const int c = x + Nx * (y + Ny * z);
        if (!solid[c]) continue;
        ++ctx->n_solid;
        uint8_t code = CODE_SOLID;
        const int kc[3] = {x, y, z};
        for (int a = 0; a < dim; ++a)
          for (int sd = 0; sd < 2; ++sd) {
            int q[3] = {x, y, z};
            q[a] += sd ? 1 : -1;
            bool wall = false;
            if (q[a] < 0 || q[a] >= ctx->n[a]) {
              if (ctx->periodic[a]) q[a] = (q[a] + ctx->n[a]) % ctx->n[a];
              else wall = true;
            }
            if (!wall) wall = !solid[q[0] + Nx * (q[1] + Ny * q[2])];
            if (wall) {
              code |= (uint8_t)(1u << (2 * a + sd));
              ctx->wall_id_h[(size_t)c * 6 + 2 * a + sd] = (int)ctx->wall_cell_h.size();
              ctx->wall_cell_h.push_back(c);
              ctx->wall_side_h.push_back(2 * a + sd);
            }
            (void)kc;
          }
        ctx->code_h[c] = code;
      }
  if (ctx->n_solid == 0) return ctx->fail(OBTE_EINVAL, "the mask has no solid cell");
  ctx->n_walls = (int)ctx->wall_cell_h.size();
  long n_sec = (long)Ny * (dim == 3 ? Nz : 1);
  ctx->kappa_scale = ctx->len[0] / (delta_T * (double)n_sec);

  cudaSetDevice(ctx->device);
  ctx->code_d = ctx->dalloc_t<uint8_t>(ctx->n_cells);
  ctx->wall_id_d = ctx->dalloc_t<int>((size_t)ctx->n_cells * 6);
  ctx->wall_cell_d = ctx->dalloc_t<int>(std::max(1, ctx->n_walls));
  ctx->wall_side_d = ctx->dalloc_t<int>(std::max(1, ctx->n_walls));
  NEED(ctx->wall_side_d);
  NEED(ctx->code_d);
  NEED(ctx->wall_id_d);
  NEED(ctx->wall_cell_d);
  CK(cudaMemcpyAsync(ctx->code_d, ctx->code_h.data(), ctx->n_cells, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->wall_id_d, ctx->wall_id_h.data(), sizeof(int) * ctx->n_cells * 6,
                     cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->n_walls) {
    CK(cudaMemcpyAsync(ctx->wall_cell_d, ctx->wall_cell_h.data(), sizeof(int) * ctx->n_walls,
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->wall_side_d, ctx->wall_side_h.data(), sizeof(int) * ctx->n_walls,
                       cudaMemcpyHostToDevice, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->has_s = false;
  ctx->s_d = nullptr;
  ctx->has_mesh = true;
  return OBTE_OK;
}

extern "C" int obte_set_scattering_scale(obte_ctx* ctx, const double* s) {
  if (!ctx) return OBTE_EINVAL;
  if (!ctx->has_mesh) return ctx->fail(OBTE_ESTATE, "create_mesh first");
  ctx->solved = false;
  ctx->flux_done = false;
  if (!s) {
    ctx->has_s = false;
    return OBTE_OK;
  }
  std::vector<double> sk(ctx->n_cells, 1.0);
  const int Nx = ctx->n[0], Ny = ctx->n[1];
  for (int c = 0; c < ctx->n_cells; ++c) {
    const int kc[3] = {c % Nx, (c / Nx) % Ny, c / (Nx * Ny)};
    int u[3];
    for (int i = 0; i < 3; ++i) u[ctx->perm[i]] = kc[i];
    const long ui = u[0] + (long)ctx->user_n[0] * (u[1] + (long)ctx->user_n[1] * u[2]);
    const double v = s[ui];
    if (ctx->code_h[c] & CODE_SOLID) {
      if (!std::isfinite(v)) return ctx->fail(OBTE_ENONFINITE, "scattering scale is not finite");
      if (!(v > 0)) return ctx->fail(OBTE_EINVAL, "scattering scale must be positive");
    }
    sk[c] = (ctx->code_h[c] & CODE_SOLID) ? v : 1.0;  // pores: never used, kept finite
  }
  if (!ctx->s_d) ctx->s_d = ctx->dalloc_t<double>(ctx->n_cells);
  NEED(ctx->s_d);
  CK(cudaMemcpyAsync(ctx->s_d, sk.data(), sizeof(double) * ctx->n_cells, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->has_s = true;
  return OBTE_OK;
}

// ---------------------------------------------------------------------------
// material and ordinate table
// ---------------------------------------------------------------------------
enum { TB_BX, TB_BY, TB_BZ, TB_DIAG, TB_INV, TB_AW, TB_KXA, TB_KYA, TB_KZA };

static int upload_material(obte_ctx* ctx);

// One ordinate of the material as the table builder takes it (kernel frame).
struct OrdIn {
  int bin;       // MFP bin (per-bin kappa spectrum, reversed-ordinate pairing)
  double lam;    // Lambda_o
  double p[3];   // direction (unit, or projected onto the plane)
  double aw;     // E2 weight a_o (sums to 1)
  double kf;     // flux weight K_o = kf p
};

// Sorted ordinate table, per-ordinate coefficients and device copies.
// Ordinates go by octant, octants in reversed pairs (q, q^full); inside an
// octant in input order, and the reversed octant's list is reordered so that
// its k-th ordinate reverses the k-th of q (same bin, Lambda and a_o,
// opposite direction) when every ordinate has such a partner.
static int build_material(obte_ctx* ctx, const std::vector<OrdIn>& in, int n_bins, double w_total,
                          const double kappa_axes[3]) {
  const int dim = ctx->dim;
  const int n = (int)in.size();
  auto oct_of = [&](int o) {
    int q = 0;
    if (in[o].p[0] < 0) q |= 1;
    if (in[o].p[1] < 0) q |= 2;
    if (dim == 3 && in[o].p[2] < 0) q |= 4;
    return q;
  };
  const int full = dim == 3 ? 7 : 3;
  std::vector<int> oct_order;
  for (int q = 0; q <= full; ++q) {
    const int qb = q ^ full;
    if (q < qb) {
      oct_order.push_back(q);
      oct_order.push_back(qb);
    }
  }
  std::vector<std::vector<int>> in_oct(8);
  for (int o = 0; o < n; ++o) in_oct[oct_of(o)].push_back(o);
  auto reverses = [&](int t, int o) {
    if (in[t].bin != in[o].bin) return false;
    for (int a = 0; a < 3; ++a)
      if (std::fabs(in[t].p[a] + in[o].p[a]) > 1e-12) return false;
    if (std::fabs(in[t].lam - in[o].lam) > 1e-12 * in[o].lam) return false;
    return std::fabs(in[t].aw - in[o].aw) <= 1e-300 + 1e-12 * in[o].aw;
  };
  std::vector<char> paired(8, 0);
  for (int i = 0; i + 1 < (int)oct_order.size(); i += 2) {
    const int q = oct_order[i], qb = oct_order[i + 1];
    if (in_oct[q].size() != in_oct[qb].size()) continue;
    std::map<int, std::vector<int>> by_bin;  // candidates of the reversed octant, by bin
    for (int t : in_oct[qb]) by_bin[in[t].bin].push_back(t);
    std::vector<int> rv;
    std::vector<char> used(n, 0);
    bool ok = true;
    for (int o : in_oct[q]) {
      int r = -1;
      for (int t : by_bin[in[o].bin])
        if (!used[t] && reverses(t, o)) {
          r = t;
          break;
        }
      if (r < 0) {
        ok = false;
        break;
      }
      used[r] = 1;
      rv.push_back(r);
    }
    if (ok) {
      in_oct[qb] = rv;  // paired order
      paired[q] = paired[qb] = 1;
    }
  }
  std::vector<int> order;
  std::vector<int> first(8, 0);
  ctx->octant.clear();
  for (int q : oct_order) {
    first[q] = (int)order.size();
    for (int o : in_oct[q]) {
      order.push_back(o);
      ctx->octant.push_back(q);
    }
  }
  // reversed ordinate of every sorted ordinate (-1 where the set has none):
  // the paired octant order gives it directly; otherwise (directions on a
  // coordinate plane) a search in the ordinate's bin
  ctx->rev_o.assign(n, -1);
  {
    std::vector<int> pos(n);
    for (int o = 0; o < n; ++o) pos[order[o]] = o;
    std::map<int, std::vector<int>> by_bin;
    for (int t = 0; t < n; ++t) by_bin[in[t].bin].push_back(t);
    for (int q : oct_order)
      for (int k = 0; k < (int)in_oct[q].size(); ++k) {
        const int o = first[q] + k;
        if (paired[q]) {
          ctx->rev_o[o] = first[q ^ full] + k;
          continue;
        }
        for (int t : by_bin[in[order[o]].bin])
          if (reverses(t, order[o])) {
            ctx->rev_o[o] = pos[t];
            break;
          }
      }
  }
  const int O = n;
  ctx->O = O;
  ctx->M = n_bins;
  ctx->w_total = w_total;
  for (int a = 0; a < 3; ++a) ctx->kappa_axes[a] = kappa_axes[a];
  ctx->ord_m.assign(O, 0);
  ctx->ord_s.assign(O, 0);
  ctx->lam_o.assign(O, 0.0);
  for (auto* v : {&ctx->bx, &ctx->by, &ctx->bz, &ctx->diag, &ctx->inv, &ctx->aw, &ctx->kxa,
                  &ctx->kya, &ctx->kza})
    v->assign(O, 0.0);
  for (int a = 0; a < 3; ++a) ctx->pk[a].assign(O, 0.0);
  double den_side[6] = {0, 0, 0, 0, 0, 0};
  for (int o = 0; o < O; ++o) {
    const OrdIn& d = in[order[o]];
    ctx->ord_m[o] = d.bin;
    ctx->ord_s[o] = order[o];
    ctx->lam_o[o] = d.lam;
    for (int a = 0; a < 3; ++a) ctx->pk[a][o] = d.p[a];
    double beta[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) beta[a] = d.lam * std::fabs(d.p[a]) / ctx->h[a];
    const double D = beta[0] + beta[1] + beta[2];
    ctx->bx[o] = beta[0];
    ctx->by[o] = beta[1];
    ctx->bz[o] = beta[2];
    ctx->diag[o] = D;
    ctx->inv[o] = 1.0 / (1.0 + D);
    ctx->aw[o] = d.aw;
    ctx->kxa[o] = d.kf * std::fabs(d.p[0]);
    ctx->kya[o] = d.kf * std::fabs(d.p[1]);
    ctx->kza[o] = dim == 3 ? d.kf * std::fabs(d.p[2]) : 0.0;
    for (int a = 0; a < dim; ++a) {
      const double k = d.kf * d.p[a];
      if (k > 0) den_side[2 * a + 1] += k;   // leaves through the + face
      if (k < 0) den_side[2 * a] += -k;      // leaves through the - face
    }
  }
  for (int a = 0; a < dim; ++a) {
    const double s0 = den_side[2 * a], s1 = den_side[2 * a + 1];
    if (std::fabs(s0 - s1) > 1e-10 * std::max(s0, s1))
      return ctx->fail(OBTE_EINVAL, "direction set is not mirror-symmetric: walls would not conserve energy");
  }
  ctx->wall_den_h.assign(std::max(1, ctx->n_walls), 1.0);
  for (int f = 0; f < ctx->n_walls; ++f) {
    const double d = den_side[ctx->wall_side_h[f]];
    ctx->wall_den_h[f] = d > 0 ? d : 1.0;
  }
  return OBTE_OK;
}

extern "C" int obte_set_material(obte_ctx* ctx, int n_mfp, const double* kappa_m,
                                 const double* lambda_m, int n_dir, const double* dirs,
                                 const double* w, int angular_dim) {
  if (!ctx) return OBTE_EINVAL;
  if (!ctx->has_mesh) return ctx->fail(OBTE_ESTATE, "create_mesh first");
  if (n_mfp < 1 || n_dir < 1 || !kappa_m || !lambda_m || !dirs || !w)
    return ctx->fail(OBTE_EINVAL, "empty material");
  if (angular_dim != 2 && angular_dim != 3) return ctx->fail(OBTE_EINVAL, "angular_dim must be 2 or 3");
  double wsum = 0;
  for (int m = 0; m < n_mfp; ++m) {
    if (!std::isfinite(kappa_m[m]) || !std::isfinite(lambda_m[m]))
      return ctx->fail(OBTE_ENONFINITE, "material is not finite");
    if (!(lambda_m[m] > 0) || kappa_m[m] < 0) return ctx->fail(OBTE_EINVAL, "need lambda_m > 0, kappa_m >= 0");
  }
  for (int s = 0; s < n_dir; ++s) {
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(dirs[3 * s + a])) return ctx->fail(OBTE_ENONFINITE, "directions not finite");
    if (!std::isfinite(w[s]) || w[s] < 0) return ctx->fail(OBTE_EINVAL, "weights must be >= 0");
    wsum += w[s];
  }
  if (std::fabs(wsum - 1.0) > 1e-9) return ctx->fail(OBTE_EINVAL, "direction weights must sum to 1");
  double sk = 0;
  for (int m = 0; m < n_mfp; ++m) sk += kappa_m[m] / (lambda_m[m] * lambda_m[m]);
  if (!(sk > 0)) return ctx->fail(OBTE_EINVAL, "sum kappa_m / lambda_m^2 must be positive");
  if ((long)n_mfp * n_dir > (1L << 30)) return ctx->fail(OBTE_EINVAL, "too many ordinates");

  ctx->S = n_dir;
  ctx->d_ang = angular_dim;
  ctx->kappa_m.assign(kappa_m, kappa_m + n_mfp);
  ctx->lambda_m.assign(lambda_m, lambda_m + n_mfp);
  ctx->sum_k_over_l2 = sk;
  // ordinate (m, s), m-major: Lambda_m s_s with a_o = w_s (kappa_m / Lambda_m^2)
  // / sum (kappa / Lambda^2) (E2) and K_o = d_ang kappa_m w_s s_s / Lambda_m
  std::vector<OrdIn> in((size_t)n_mfp * n_dir);
  for (int m = 0; m < n_mfp; ++m)
    for (int s = 0; s < n_dir; ++s) {
      OrdIn& d = in[(size_t)m * n_dir + s];
      // kernel-frame direction (2D: user z dropped before the permutation)
      const double u[3] = {dirs[3 * s], dirs[3 * s + 1], ctx->dim == 3 ? dirs[3 * s + 2] : 0.0};
      for (int i = 0; i < 3; ++i) d.p[i] = u[ctx->perm[i]];
      const double lam = lambda_m[m];
      d.bin = m;
      d.lam = lam;
      d.aw = w[s] * (kappa_m[m] / (lam * lam)) / sk;
      d.kf = angular_dim * kappa_m[m] * w[s] / lam;
    }
  double kb = 0.0;
  for (int m = 0; m < n_mfp; ++m) kb += kappa_m[m];
  const double kax[3] = {kb, kb, kb};  // isotropic: d_ang sum_s w_s p p^T = I
  const int rc = build_material(ctx, in, n_mfp, angular_dim * sk, kax);
  if (rc) return rc;
  return upload_material(ctx);
}

// General aMFP material: per-ordinate vectorial MFP and weight (Sec. 5, App. A)
extern "C" int obte_set_material_ordinates(obte_ctx* ctx, int n_ord, const double* lambda,
                                           const double* dirs, const double* weight, const int* bin,
                                           int n_bins) {
  if (!ctx) return OBTE_EINVAL;
  if (!ctx->has_mesh) return ctx->fail(OBTE_ESTATE, "create_mesh first");
  if (n_ord < 1 || !lambda || !dirs || !weight) return ctx->fail(OBTE_EINVAL, "empty material");
  if (bin && n_bins < 1) return ctx->fail(OBTE_EINVAL, "n_bins must be >= 1");
  if (!bin) n_bins = 1;
  double W = 0.0;
  for (int o = 0; o < n_ord; ++o) {
    if (!std::isfinite(lambda[o]) || !std::isfinite(weight[o]))
      return ctx->fail(OBTE_ENONFINITE, "material is not finite");
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(dirs[3 * o + a])) return ctx->fail(OBTE_ENONFINITE, "directions not finite");
    if (!(lambda[o] > 0) || weight[o] < 0) return ctx->fail(OBTE_EINVAL, "need lambda > 0, weight >= 0");
    if (bin && (bin[o] < 0 || bin[o] >= n_bins)) return ctx->fail(OBTE_EINVAL, "bin out of range");
    W += weight[o];
  }
  if (!(W > 0)) return ctx->fail(OBTE_EINVAL, "the weights must not all be zero");
  std::vector<OrdIn> in(n_ord);
  double kax[3] = {0, 0, 0};
  for (int o = 0; o < n_ord; ++o) {
    OrdIn& d = in[o];
    const double u[3] = {dirs[3 * o], dirs[3 * o + 1], ctx->dim == 3 ? dirs[3 * o + 2] : 0.0};
    for (int i = 0; i < 3; ++i) d.p[i] = u[ctx->perm[i]];
    d.bin = bin ? bin[o] : 0;
    d.lam = lambda[o];
    d.aw = weight[o] / W;                 // a_o = W_o / sum W (E2)
    d.kf = weight[o] * lambda[o];         // K_o = W_o Lambda_o s_o
    for (int a = 0; a < 3; ++a) kax[a] += d.kf * lambda[o] * d.p[a] * d.p[a];
  }
  ctx->S = 0;
  ctx->d_ang = 0;
  ctx->kappa_m.clear();
  ctx->lambda_m.clear();
  ctx->sum_k_over_l2 = 0.0;
  if (!(kax[0] > 0)) return ctx->fail(OBTE_EINVAL, "no ordinate moves along the gradient axis");
  const int rc = build_material(ctx, in, n_bins, W, kax);
  if (rc) return rc;
  return upload_material(ctx);
}

// device copies of the ordinate table (FP64 and FP32), bins, octants and
// wall denominators
static int upload_material(obte_ctx* ctx) {
  const int O = ctx->O;
  cudaSetDevice(ctx->device);
  const std::vector<double>* tabs[9] = {&ctx->bx, &ctx->by, &ctx->bz, &ctx->diag, &ctx->inv,
                                        &ctx->aw, &ctx->kxa, &ctx->kya, &ctx->kza};
  for (int t = 0; t < 9; ++t) {
    if (!ctx->tab_d[0][t]) ctx->tab_d[0][t] = ctx->dalloc_t<double>(O);
    else {
      ctx->dfree(ctx->tab_d[0][t]);
      ctx->tab_d[0][t] = ctx->dalloc_t<double>(O);
    }
    if (ctx->tab_d[1][t]) ctx->dfree(ctx->tab_d[1][t]);
    ctx->tab_d[1][t] = ctx->dalloc_t<float>(O);
    NEED(ctx->tab_d[0][t]);
    NEED(ctx->tab_d[1][t]);
    std::vector<float> f(O);
    for (int o = 0; o < O; ++o) f[o] = (float)(*tabs[t])[o];
    CK(cudaMemcpyAsync(ctx->tab_d[0][t], tabs[t]->data(), sizeof(double) * O, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->tab_d[1][t], f.data(), sizeof(float) * O, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (ctx->mbin_d) ctx->dfree(ctx->mbin_d);
  if (ctx->octant_d) ctx->dfree(ctx->octant_d);
  if (ctx->wall_den_d) ctx->dfree(ctx->wall_den_d);
  ctx->mbin_d = ctx->dalloc_t<int>(O);
  ctx->octant_d = ctx->dalloc_t<int>(O);
  ctx->wall_den_d = ctx->dalloc_t<double>(ctx->wall_den_h.size());
  NEED(ctx->mbin_d);
  NEED(ctx->octant_d);
  NEED(ctx->wall_den_d);
  CK(cudaMemcpyAsync(ctx->mbin_d, ctx->ord_m.data(), sizeof(int) * O, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->octant_d, ctx->octant.data(), sizeof(int) * O, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->wall_den_d, ctx->wall_den_h.data(), sizeof(double) * ctx->wall_den_h.size(),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->has_material = true;
  ctx->solved = false;
  ctx->precision = -1;  // state buffers are rebuilt by the next solve
  return OBTE_OK;
}

// ---------------------------------------------------------------------------
// variant choice and autotuning
// ---------------------------------------------------------------------------
namespace {

struct Variant {
  int G, R;
  bool warp;         // 2D warp-per-group kernel (sweep2d.cuh)
  bool k3d = false;  // 3D block kernel with skewed records (sweep3d.cuh)
  int nh = 1;        // warps per group of the 2D warp kernel (2: rows fill 64 lanes)
};

const Variant kWarp2D_F[] = {{8, 8, true}, {8, 4, true, false, 2}, {8, 4, true}, {16, 4, true}, {16, 2, true},
                             {16, 1, true}, {8, 1, true},  {6, 8, true},  {4, 8, true},
                             {4, 4, true},  {8, 2, true},  {8, 3, true},  {8, 5, true},
                             {8, 6, true}};
const Variant kWarp2D_D[] = {{4, 8, true}, {8, 4, true}, {8, 2, true}, {8, 1, true}, {2, 8, true}};
const Variant kVariants2D_F[] = {{16, 4, false}, {8, 4, false}, {8, 8, false}, {16, 2, false},
                                 {8, 2, false}, {4, 4, false}, {16, 1, false}};
const Variant kVariants2D_D[] = {{8, 2, false}, {8, 4, false}, {4, 4, false}, {4, 8, false},
                                 {8, 1, false}};
const Variant kVariants3D_F[] = {{8, 4, false, true}, {8, 8, false, true}, {4, 8, false, true},
                                 {4, 4, false, true}, {8, 2, false, true},
                                 {8, 8, false}, {4, 8, false}, {8, 4, false}, {4, 4, false},
                                 {8, 2, false}, {4, 2, false}};
const Variant kVariants3D_D[] = {{4, 8, false, true}, {4, 4, false, true}, {2, 4, false, true},
                                 {4, 8, false}, {4, 4, false}, {4, 2, false}, {8, 2, false}};

int threads_for(int ny, int nz, int R) {
  const int tpp = (ny + R - 1) / R;
  const int t = tpp * nz;
  return ((t + 31) / 32) * 32;
}

template <size_t N>
void push_fitting(std::vector<Variant>& out, const Variant (&v)[N], int precision, int dim, int ny,
                  int nz, bool has_s) {
  for (size_t i = 0; i < N; ++i) {
    if (ny % v[i].R != 0) continue;
    if (v[i].warp && v[i].nh == 2) {
      if (dim != 2 || has_s || ny != 64 * v[i].R) continue;
      if (!sweep2d_split_exists(precision, v[i].G, v[i].R)) continue;
    } else if (v[i].warp) {
      if (dim != 2 || ny / v[i].R > 32) continue;
      if (!sweep2d_warp_exists(precision, v[i].G, v[i].R, has_s, true)) continue;
    } else if (v[i].k3d) {
      const int thr = threads_for(ny, nz, v[i].R);
      if (dim != 3 || thr > (v[i].R >= 8 ? 256 : 512)) continue;
      if (sweep3d_smem_bytes(precision, v[i].G, v[i].R, thr) > 226 * 1024) continue;
      if (!sweep3d_exists(precision, v[i].G, v[i].R, has_s)) continue;
    } else {
      const int thr = threads_for(ny, nz, v[i].R);
      if (thr > ((dim == 3 && v[i].R < 8) ? 512 : 256)) continue;  // the kernel's launch bound
      if (sweep_smem_bytes(precision, dim, v[i].G, v[i].R, thr) > 200 * 1024) continue;
      if (!sweep_variant_exists(precision, dim, v[i].G, v[i].R, has_s)) continue;
    }
    out.push_back(v[i]);
  }
}

std::vector<Variant> candidates(int precision, int dim, int ny, int nz, bool has_s) {
  std::vector<Variant> out;
  if (dim == 2) {
    if (precision) {
      push_fitting(out, kWarp2D_F, precision, dim, ny, nz, has_s);
      push_fitting(out, kVariants2D_F, precision, dim, ny, nz, has_s);
    } else {
      push_fitting(out, kWarp2D_D, precision, dim, ny, nz, has_s);
      push_fitting(out, kVariants2D_D, precision, dim, ny, nz, has_s);
    }
  } else {
    if (precision) push_fitting(out, kVariants3D_F, precision, dim, ny, nz, has_s);
    else push_fitting(out, kVariants3D_D, precision, dim, ny, nz, has_s);
  }
  return out;
}

std::map<std::tuple<int, int, int, int, int, int>, Variant>& tune_cache() {
  static std::map<std::tuple<int, int, int, int, int, int>, Variant> c;
  return c;
}

// guards tune_cache and the batch-form cache: contexts may be driven from
// different host threads
std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}

// events destroyed on every return path
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

// Work items: runs of at most G ordinates of one octant.  Items of one octant
// start their wavefront at evenly spaced columns (d0) so that, at a given
// step, they update different cells.
//
// pad > 1: every octant's items are padded with empty items (count 0) to a
// multiple of pad, and each run of pad consecutive items shares its start
// column (the 2D warp kernel's block-combined moments).
static void build_items(obte_ctx* ctx, int geom, int G, std::vector<WorkItem>& items,
                        std::vector<int>* ord_d0 = nullptr, int pad = 1) {
  const int O = ctx->O;
  const int nx = ctx->n[0];
  if (ord_d0) ord_d0->assign(O, 0);
  int o = 0;
  while (o < O) {
    const int q = ctx->octant[o];
    int e = o;
    while (e < O && ctx->octant[e] == q) ++e;
    const int n_it = (e - o + G - 1) / G;
    const int n_pad = ((n_it + pad - 1) / pad) * pad;
    const int n_run = n_pad / pad;  // runs sharing a start column
    for (int k = 0; k < n_pad; ++k) {
      const int d0 = (int)(((long)(k / pad) * nx) / std::max(1, n_run)) % nx;
      const int a = o + k * G;
      const int cnt = a < e ? std::min(G, e - a) : 0;
      items.push_back({geom, q, a < e ? a : e, cnt, d0});
      if (ord_d0)
        for (int b = a; b < a + cnt; ++b) (*ord_d0)[b] = d0;
    }
    o = e;
  }
}

// allocate the iteration state for a precision / variant; fill gh and gd
static int prepare_state(obte_ctx* ctx, int precision, int G, int R, bool warp, int max_iter,
                         const obte_solve_opts& op, bool k3d = false, int nh = 1) {
  cudaSetDevice(ctx->device);
  const int Nx = ctx->n[0], Ny = ctx->n[1], Nz = ctx->n[2];
  const int rows = Ny * Nz;
  if (ctx->precision != precision) {
    ctx->drop_graph();
    // (re)allocate everything that depends on the precision
    ctx->dfree(ctx->rec4);
    ctx->dfree(ctx->rec_idx);
    ctx->dfree(ctx->tlq);
    ctx->rec4 = nullptr;
    ctx->rec_idx = nullptr;
    ctx->tlq = nullptr;
    ctx->rec_w_alloc = 0;
    for (void* p : {(void*)ctx->aa_xd, (void*)ctx->aa_fd, ctx->aa_xt, ctx->aa_ft, (void*)ctx->aa_small,
                    (void*)ctx->aa_int})
      ctx->dfree(p);
    ctx->aa_xd = ctx->aa_fd = ctx->aa_small = nullptr;
    ctx->aa_xt = ctx->aa_ft = nullptr;
    ctx->aa_int = nullptr;
    ctx->aa_m_alloc = -1;
    for (void* p : {(void*)ctx->TL, (void*)ctx->TL_acc, ctx->src, ctx->twc, (void*)ctx->Tw, (void*)ctx->wall_acc,
                    ctx->front, (void*)ctx->scal, (void*)ctx->ctrl, (void*)ctx->hist, (void*)ctx->TF,
                    (void*)ctx->fwork, (void*)ctx->fiters, (void*)ctx->gd})
      ctx->dfree(p);
    const size_t e = precision == 0 ? 8 : 4;
    ctx->TL = ctx->dalloc_t<double>(ctx->n_cells);
    ctx->TL_acc = ctx->dalloc_t<double>(ctx->n_cells);
    ctx->src = ctx->dalloc(e * ctx->n_cells);
    ctx->twc = ctx->dalloc(e * (size_t)ctx->n_cells * 6);
    NEED(ctx->twc);
    ctx->Tw = ctx->dalloc_t<double>(std::max(1, ctx->n_walls));
    ctx->wall_acc = ctx->dalloc_t<double>((size_t)ctx->n_cells * 6);
    ctx->front = ctx->dalloc(e * (size_t)ctx->O * rows);
    ctx->scal = ctx->dalloc_t<double>(6);
    ctx->ctrl = ctx->dalloc_t<int>(4);
    ctx->hist = ctx->dalloc_t<double>(kMaxHist);
    ctx->TF = ctx->dalloc_t<double>(ctx->n_cells);
    ctx->fwork = ctx->dalloc_t<double>(fourier_work_doubles(ctx->n_cells, kFourierBlocksMax));
    ctx->fiters = ctx->dalloc_t<int>(1);
    ctx->gd = ctx->dalloc_t<GeomDev>(1);
    NEED(ctx->TL);
    NEED(ctx->TL_acc);
    NEED(ctx->src);
    NEED(ctx->Tw);
    NEED(ctx->wall_acc);
    NEED(ctx->front);
    NEED(ctx->scal);
    NEED(ctx->ctrl);
    NEED(ctx->hist);
    NEED(ctx->TF);
    NEED(ctx->fwork);
    NEED(ctx->fiters);
    NEED(ctx->gd);
    ctx->precision = precision;
  }
  const int nq = ctx->dim == 3 ? 8 : 4;          // octants
  const int rec_w = k3d ? 8 : (warp ? 4 : 0);     // values per skewed record
  if (rec_w && ctx->rec_w_alloc != rec_w) {
    ctx->dfree(ctx->rec4);
    ctx->dfree(ctx->rec_idx);
    ctx->dfree(ctx->tlq);
    ctx->tlq = nullptr;
    const size_t e = precision == 0 ? 8 : 4;
    ctx->rec4 = ctx->dalloc((size_t)nq * rec_w * e * (size_t)ctx->n_cells);
    ctx->rec_idx = ctx->dalloc_t<int>((size_t)nq * ctx->n_cells);
    NEED(ctx->rec4);
    NEED(ctx->rec_idx);
    {  // skewed T_L partials of the 2D warp kernel and of the 3D kernel
      ctx->tlq = ctx->dalloc_t<double>((size_t)nq * ctx->n_cells);
      NEED(ctx->tlq);
      CK(cudaMemsetAsync(ctx->tlq, 0, sizeof(double) * nq * (size_t)ctx->n_cells, ctx->stream));
    }
    ctx->rec_w_alloc = rec_w;
  }
  if (!ctx->blk_part) {
    ctx->blk_part = ctx->dalloc_t<double>((size_t)kMaxPartBlocks * 8);
    NEED(ctx->blk_part);
  }
  const int aa_m = std::max(0, std::min(op.accel, 7));
  const long aa_nd = (long)ctx->n_cells + ctx->n_walls;
  const long aa_nt = (long)ctx->O * rows;
  if (aa_m > 0 && ctx->aa_m_alloc != aa_m) {
    for (void* p : {(void*)ctx->aa_xd, (void*)ctx->aa_fd, ctx->aa_xt, ctx->aa_ft, (void*)ctx->aa_small,
                    (void*)ctx->aa_int})
      ctx->dfree(p);
    const size_t e = precision == 0 ? 8 : 4;
    // g(x) history slots plus the current iterate (last slot); f history
    ctx->aa_xd = ctx->dalloc_t<double>((size_t)(aa_m + 2) * aa_nd);
    ctx->aa_fd = ctx->dalloc_t<double>((size_t)(aa_m + 1) * aa_nd);
    ctx->aa_xt = ctx->dalloc(e * (size_t)(aa_m + 2) * aa_nt);
    ctx->aa_ft = ctx->dalloc(e * (size_t)(aa_m + 1) * aa_nt);
    ctx->aa_small = ctx->dalloc_t<double>(8 + 64 + 8);
    ctx->aa_int = ctx->dalloc_t<int>(2);
    NEED(ctx->aa_xd);
    NEED(ctx->aa_fd);
    NEED(ctx->aa_xt);
    NEED(ctx->aa_ft);
    NEED(ctx->aa_small);
    NEED(ctx->aa_int);
    CK(cudaMemsetAsync(ctx->aa_small, 0, sizeof(double) * 80, ctx->stream));
    CK(cudaMemsetAsync(ctx->aa_int, 0, sizeof(int) * 2, ctx->stream));
    ctx->aa_m_alloc = aa_m;
  }
  GeomDev& g = ctx->gh;
  std::memset(&g, 0, sizeof(g));
  g.aa_m = aa_m;
  if (aa_m > 0) {
    g.aa_nd = aa_nd;
    g.aa_nt = aa_nt;
    g.aa_gd = ctx->aa_xd;
    g.aa_fd = ctx->aa_fd;
    g.aa_xcd = ctx->aa_xd + (size_t)(aa_m + 1) * aa_nd;
    g.aa_gt = ctx->aa_xt;
    g.aa_ft = ctx->aa_ft;
    g.aa_xct = static_cast<char*>(ctx->aa_xt) + (size_t)(aa_m + 1) * aa_nt * (precision == 0 ? 8 : 4);
    g.aa_gram = ctx->aa_small + 8;
    g.aa_coef = ctx->aa_small + 72;
    g.aa_k = ctx->aa_int;
  }
  g.nx = Nx;
  g.ny = Ny;
  g.nz = Nz;
  g.dim = ctx->dim;
  g.n_cells = ctx->n_cells;
  g.rows = rows;
  g.py = ctx->periodic[1];
  g.pz = ctx->dim == 3 ? ctx->periodic[2] : 0;
  g.R = R;
  g.tpp = (Ny + R - 1) / R;
  g.n_ord = ctx->O;
  g.n_walls = ctx->n_walls;
  g.dT = ctx->dT;
  g.kappa_scale = ctx->kappa_scale;
  g.code = ctx->code_d;
  g.wall_id = ctx->wall_id_d;
  g.s = ctx->has_s ? ctx->s_d : nullptr;
  g.TL = ctx->TL;
  g.TL_acc = ctx->TL_acc;
  g.src = ctx->src;
  g.Tw = ctx->Tw;
  g.wall_acc = ctx->wall_acc;
  g.wall_den = ctx->wall_den_d;
  g.wall_cell = ctx->wall_cell_d;
  g.wall_side = ctx->wall_side_d;
  g.twc = ctx->twc;
  g.rec4 = rec_w ? ctx->rec4 : nullptr;
  g.rec_idx = rec_w ? ctx->rec_idx : nullptr;
  g.tlq = rec_w == 4 ? ctx->tlq : nullptr;
  g.tlq3 = rec_w == 8 ? ctx->tlq : nullptr;
  g.blk_part = ctx->blk_part;
  g.rec_w = rec_w;
  g.psi = (precision == 1 && rec_w > 0) ? 1 : 0;  // float record kernels: deviation form
  g.front = ctx->front;
  g.phi_acc = ctx->scal;
  g.delta_max = ctx->scal + 1;
  g.hot_tl = ctx->scal + 3;
  g.kx_pos = g.kx_neg = 0.0;
  for (int o = 0; o < ctx->O; ++o) {  // sorted-frame signed K_ox = sign(p_x) |K_ox|
    const double k = ctx->pk[0][o] > 0 ? ctx->kxa[o] : (ctx->pk[0][o] < 0 ? -ctx->kxa[o] : 0.0);
    if (k > 0) g.kx_pos += k;
    else g.kx_neg += k;
  }
  g.J_acc = ctx->J_acc;
  g.phi_sec = ctx->phi_sec;
  g.phi_bin = ctx->phi_bin;
  g.rec = nullptr;
  g.rec_slot = nullptr;
  const int p = precision == 0 ? 0 : 1;
  g.bx = ctx->tab_d[p][TB_BX];
  g.by = ctx->tab_d[p][TB_BY];
  g.bz = ctx->tab_d[p][TB_BZ];
  g.diag = ctx->tab_d[p][TB_DIAG];
  g.inv = ctx->tab_d[p][TB_INV];
  g.aw = ctx->tab_d[p][TB_AW];
  g.kxa = ctx->tab_d[p][TB_KXA];
  g.kya = ctx->tab_d[p][TB_KYA];
  g.kza = ctx->tab_d[p][TB_KZA];
  g.mbin = ctx->mbin_d;
  g.ord_d0 = nullptr;  // set below once the work items are known
  g.octant_of = ctx->octant_d;
  g.T0 = ctx->TF;
  g.done = ctx->ctrl + 0;
  g.iter = ctx->ctrl + 1;
  g.nonfinite = ctx->ctrl + 2;
  g.kappa_hist = ctx->hist;
  g.max_hist = kMaxHist;
  g.tol = op.tol;
  g.tol_TL = op.tol_TL;
  g.min_iter = std::max(op.min_iter, 1);
  g.max_iter = max_iter;
  ctx->G = G;
  ctx->R = R;
  ctx->warp = warp;
  ctx->k3d = k3d;
  ctx->nh = warp ? nh : 1;
  ctx->threads = warp ? (nh == 2 ? 256 : 32 * sweep2d_warps_per_block(precision, G, R, ctx->has_s, true))
                      : threads_for(Ny, Nz, R);
  std::vector<WorkItem> items;
  std::vector<int> ord_d0;
  // block-combined moments: warp kernel with four warps per block over full
  // 32-lane rows
  ctx->items_pad = (warp && ((nh == 2 && Ny == 64 * R) ||
                              (nh == 1 && sweep2d_warps_per_block(precision, G, R, ctx->has_s, true) == 4 &&
                               Ny == 32 * R)))
                       ? 4
                       : 1;
  build_items(ctx, 0, G, items, &ord_d0, ctx->items_pad);
  if (ctx->shard_n > 1) {
    // runs of items_pad items (one start column, one octant) go round-robin
    // to the ranks; every rank keeps the full ordinate tables
    std::vector<WorkItem> mine;
    for (size_t k = 0; k < items.size(); ++k)
      if ((int)((k / ctx->items_pad) % ctx->shard_n) == ctx->shard_rank) mine.push_back(items[k]);
    if (mine.empty())  // one run of empty items: the rank sweeps nothing
      for (int k = 0; k < ctx->items_pad; ++k) mine.push_back({0, items[0].octant, items[0].o0, 0, items[0].d0});
    items.swap(mine);
  }
  const bool same = ctx->items_d && items.size() == ctx->items_h.size() &&
                    std::memcmp(items.data(), ctx->items_h.data(), sizeof(WorkItem) * items.size()) == 0;
  if (!same) {
    ctx->items_h = items;
    if (ctx->ord_d0_d) ctx->dfree(ctx->ord_d0_d);
    ctx->ord_d0_d = ctx->dalloc_t<int>(ctx->O);
    NEED(ctx->ord_d0_d);
    CK(cudaMemcpyAsync(ctx->ord_d0_d, ord_d0.data(), sizeof(int) * ctx->O, cudaMemcpyHostToDevice,
                       ctx->stream));
    if (ctx->items_d) ctx->dfree(ctx->items_d);
    ctx->items_d = ctx->dalloc_t<WorkItem>(ctx->items_h.size());
    NEED(ctx->items_d);
    CK(cudaMemcpyAsync(ctx->items_d, ctx->items_h.data(), sizeof(WorkItem) * ctx->items_h.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
  }
  g.ord_d0 = ctx->ord_d0_d;
  CK(cudaMemcpyAsync(ctx->gd, &g, sizeof(GeomDev), cudaMemcpyHostToDevice, ctx->stream));
  return OBTE_OK;
}

// the context's 2D warp-kernel variant (one- or two-warp groups)
// (after a batched solve the context's rows per lane may have no fixed-rows
// instance: the general-rows instance then serves its flux and record passes)
static cudaError_t launch_ctx_warp(obte_ctx* ctx, const SweepLaunch& L) {
  if (ctx->nh == 2) return launch_sweep2d_split(L, ctx->precision, ctx->G, ctx->R, 0, ctx->stream);
  if (!sweep2d_warp_exists(ctx->precision, ctx->G, ctx->R, ctx->has_s, true))
    return launch_sweep2d_warp(L, ctx->precision, ctx->G, 8, ctx->has_s, false, 0, ctx->stream);
  return launch_sweep2d_warp(L, ctx->precision, ctx->G, ctx->R, ctx->has_s, true, 0, ctx->stream);
}

static cudaError_t sweep_once(obte_ctx* ctx, int flags) {
  SweepLaunch L;
  L.geoms = ctx->gd;
  L.items = ctx->items_d;
  L.n_items = (int)ctx->items_h.size();
  L.flags = flags | (ctx->warp && ctx->items_pad == 4 ? SWEEP_BLOCK_COMBINE : 0);
  L.item_counter = nullptr;
  if (ctx->warp) return launch_ctx_warp(ctx, L);
  if (ctx->k3d)
    return launch_sweep3d(L, ctx->precision, ctx->G, ctx->R, ctx->has_s, ctx->threads,
                          sweep3d_smem_bytes(ctx->precision, ctx->G, ctx->R, ctx->threads), ctx->stream);
  const size_t smem = sweep_smem_bytes(ctx->precision, ctx->dim, ctx->G, ctx->R, ctx->threads);
  return launch_sweep(L, ctx->precision, ctx->dim, ctx->G, ctx->R, ctx->has_s, ctx->threads,
                      L.n_items, smem, ctx->stream);
}

static int aa_blocks(int n_cells, int n_ord, int rows) {
  const long n = std::max((long)n_cells, (long)n_ord * rows);
  return (int)std::max(1L, std::min((n / 4 + 255) / 256, 456L));
}

static int finalize_blocks(int n_cells) {
  int b = (n_cells + 255) / 256;
  return std::max(1, std::min(b, 296));
}

// Grid spacings for the heat-conduction stencil (first guess, Fourier model):
// an axis-aligned anisotropic bulk tensor enters as kappa_a / h_a^2, i.e. as
// spacings h_a sqrt(kappa_x / kappa_a) at conductivity kappa_x.
static void cg_spacing(const obte_ctx* ctx, double he[3]) {
  he[0] = ctx->h[0];
  for (int a = 1; a < 3; ++a) {
    const double r = ctx->kappa_axes[a] / ctx->kappa_axes[0];
    he[a] = (r > 0 && std::isfinite(r)) ? ctx->h[a] / std::sqrt(r) : ctx->h[a];
  }
}

static int init_from_fourier(obte_ctx* ctx, const obte_solve_opts& op, int* fiters_out) {
  const int prec = ctx->precision;
  int fmax = op.fourier_max_iter > 0 ? op.fourier_max_iter : 4 * (ctx->n[0] + ctx->n[1] + ctx->n[2]);
  // 1e-3 was the best single setting for the time to kappa over the measured
  // workloads: tighter costs CG iterations and saves no transport iterations;
  // looser can stop at the linear starting profile (no CG step at all on a
  // 256 x 256 mesh with a 25 % pore) and cost transport iterations
  double ftol = op.fourier_tol > 0 ? op.fourier_tol : kFourierTolDefault;
  double he[3];
  cg_spacing(ctx, he);
  if (ctx->n_cells <= 4096) {
    // small mesh: one block solves it, no grid-wide synchronisation
    if (!ctx->cg_job) ctx->cg_job = ctx->dalloc_t<CGArgs>(1);
    NEED(ctx->cg_job);
    const CGArgs job = make_cg_args(ctx->gh, he[0], he[1], he[2], fmax, ftol, ctx->TF,
                                    ctx->fiters, ctx->fwork, kFourierBlocksMax);
    CK(cudaMemcpyAsync(ctx->cg_job, &job, sizeof(CGArgs), cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_fourier_cg_blocks(ctx->cg_job, 1, prec, ctx->stream));
  } else {
    CK(launch_fourier_cg(ctx->gh, he[0], he[1], he[2], prec, fmax, ftol, ctx->TF,
                         ctx->fiters, ctx->fwork, kFourierBlocksMax, ctx->stream));
  }
  CK(launch_init_state(ctx->gd, 1, std::max((long)ctx->gh.n_cells * 6, (long)ctx->gh.n_ord * ctx->gh.rows),
                       ctx->gh.n_walls, prec, ctx->stream));
  if (ctx->warp || ctx->k3d) {
    CK(launch_build_records(ctx->gd, 1, prec, finalize_blocks(ctx->n_cells), ctx->stream));
    CK(launch_psi_records(ctx->gd, 1, prec, finalize_blocks(ctx->n_cells), ctx->stream));
  }
  if (ctx->gh.aa_m > 0)
    CK(launch_anderson_init(ctx->gd, 1, prec, aa_blocks(ctx->n_cells, ctx->O, ctx->n[1] * ctx->n[2]), ctx->stream));
  if (fiters_out) {
    CK(cudaMemcpyAsync(fiters_out, ctx->fiters, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  }
  return OBTE_OK;
}

static std::vector<Variant> filtered_candidates(obte_ctx* ctx, int precision,
                                                const obte_solve_opts& op) {
  std::vector<Variant> out;
  for (auto& c : candidates(precision, ctx->dim, ctx->n[1], ctx->n[2], ctx->has_s)) {
    if ((c.warp || c.k3d) && ctx->n_cells > kMaxSkewCells) continue;  // packed cell index is 22 bits
    if (op.kernel == 1 && (c.warp || c.k3d)) continue;
    if (op.kernel == 2 && !c.warp) continue;
    if (op.kernel == 3 && !c.k3d) continue;
    if (op.group_size > 0 && c.G != op.group_size) continue;
    if (op.rows_per_thread > 0 && c.R != op.rows_per_thread) continue;
    out.push_back(c);
  }
  return out;
}

static int pick_variant(obte_ctx* ctx, int precision, const obte_solve_opts& op, Variant* out) {
  auto cands = filtered_candidates(ctx, precision, op);
  if (cands.empty())
    return ctx->fail(OBTE_EINVAL, "no compiled sweep variant matches kernel / group_size / "
                                  "rows_per_thread for this mesh");
  auto key = std::make_tuple(precision * 2 + (ctx->has_s ? 1 : 0), ctx->dim, ctx->n[0], ctx->n[1],
                             ctx->n[2], ctx->O);
  if (op.group_size == 0 && op.rows_per_thread == 0 && op.kernel == 0) {
    std::lock_guard<std::mutex> lock(tune_mutex());
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
      *out = it->second;
      return OBTE_OK;
    }
  }
  // default: the first listed candidate that gives every SM at least one warp
  // of work; the lists are ordered by measured preference
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  // (a warp kernel whose rows leave lanes idle comes after one that fills all 32)
  *out = cands[0];
  for (int pass = 0; pass < 2; ++pass)
    for (auto& c : cands) {
      const long units = (ctx->O + c.G - 1) / c.G;
      if (units < sms) continue;
      if (pass == 0 && c.warp && ctx->n[1] / c.R != 32 * c.nh) continue;
      *out = c;
      return OBTE_OK;
    }
  return OBTE_OK;
}

// timed autotune over the compiled variants (group_size = -1)
static int autotune(obte_ctx* ctx, int precision, const obte_solve_opts& op, Variant* out) {
  auto key = std::make_tuple(precision * 2 + (ctx->has_s ? 1 : 0), ctx->dim, ctx->n[0], ctx->n[1], ctx->n[2], ctx->O);
  auto cands = filtered_candidates(ctx, precision, op);
  if (cands.empty()) return ctx->fail(OBTE_EINVAL, "no compiled sweep variant fits this mesh");
  EventPair ev;
  CK(cudaEventCreate(&ev.a));
  CK(cudaEventCreate(&ev.b));
  cudaEvent_t a = ev.a, b = ev.b;
  float best = 1e30f;
  Variant bv = cands[0];
  for (auto& c : cands) {
    int rc = prepare_state(ctx, precision, c.G, c.R, c.warp, 1 << 30, op, c.k3d, c.nh);
    if (rc) return rc;
    obte_solve_opts o2 = op;
    o2.fourier_max_iter = 1;
    rc = init_from_fourier(ctx, o2, nullptr);
    if (rc) return rc;
    CK(sweep_once(ctx, 0));  // warm-up
    CK(cudaEventRecord(a, ctx->stream));
    for (int i = 0; i < 3; ++i) CK(sweep_once(ctx, 0));
    CK(cudaEventRecord(b, ctx->stream));
    CK(cudaEventSynchronize(b));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, a, b));
    if (ms < best) {
      best = ms;
      bv = c;
    }
  }
  {
    std::lock_guard<std::mutex> lock(tune_mutex());
    tune_cache()[key] = bv;
  }
  *out = bv;
  return OBTE_OK;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
struct IterTiming {
  int n_sweeps = 0;
  double sweep_ms = 0.0, finalize_ms = 0.0;
};

static int run_iterations(obte_ctx* ctx, const obte_solve_opts& op, int* iters, int* done_code,
                          IterTiming* tm) {
  const int k = std::max(1, op.check_every);
  int* host_ctrl = nullptr;
  int rc = OBTE_OK;
  // optional per-launch events: ev[3 i] before sweep i, ev[3 i + 1] after it,
  // ev[3 i + 2] after finalize i
  const long long key[8] = {(long long)(size_t)ctx->gd, (long long)(size_t)ctx->items_d,
                            (long long)ctx->items_h.size(), ctx->precision * 1000003LL + ctx->G * 1009 + ctx->R,
                            ctx->threads, k, op.profile, ctx->has_s};
  bool reuse = op.use_graph && ctx->it_exec && std::equal(key, key + 8, ctx->it_key);
  if (!reuse) {
    ctx->drop_graph();
    if (op.profile) {
      ctx->it_events.resize(3 * k);
      for (auto& e : ctx->it_events) CK(cudaEventCreate(&e));
    }
  }
  // pinned after the event setup, whose failures return early
  CK(cudaMallocHost(&host_ctrl, 4 * sizeof(int)));
  std::vector<cudaEvent_t>& ev = ctx->it_events;
  auto body = [&]() -> cudaError_t {
    for (int i = 0; i < k; ++i) {
      cudaError_t e;
      if (op.profile && (e = cudaEventRecordWithFlags(ev[3 * i], ctx->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
      e = sweep_once(ctx, 0);
      if (e != cudaSuccess) return e;
      if (op.profile && (e = cudaEventRecordWithFlags(ev[3 * i + 1], ctx->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
      e = launch_finalize(ctx->gd, 1, ctx->precision, finalize_blocks(ctx->n_cells), ctx->stream);
      if (e != cudaSuccess) return e;
      if (ctx->gh.aa_m > 0) {
        e = launch_anderson_step(ctx->gd, 1, ctx->precision,
                                 aa_blocks(ctx->n_cells, ctx->O, ctx->n[1] * ctx->n[2]), ctx->stream);
        if (e != cudaSuccess) return e;
      }
      if (ctx->gh.psi) {
        e = launch_psi_records(ctx->gd, 1, ctx->precision, finalize_blocks(ctx->n_cells), ctx->stream);
        if (e != cudaSuccess) return e;
      }
      if (op.profile && (e = cudaEventRecordWithFlags(ev[3 * i + 2], ctx->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (op.use_graph && !reuse) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t eb = body();
      e = cudaStreamEndCapture(ctx->stream, &graph);
      if (eb != cudaSuccess) e = eb;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->it_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->it_exec = nullptr;
    } else {
      std::copy(key, key + 8, ctx->it_key);
    }
  }
  cudaGraphExec_t exec = op.use_graph ? ctx->it_exec : nullptr;
  int launched = 0, prev_iter = 0;
  while (true) {
    cudaError_t e = exec ? cudaGraphLaunch(exec, ctx->stream) : body();
    if (e != cudaSuccess) {
      rc = ctx->cuda_fail(e, "iteration launch");
      break;
    }
    launched += k;
    e = cudaMemcpyAsync(host_ctrl, ctx->ctrl, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      rc = ctx->cuda_fail(e, "iteration sync");
      break;
    }
    if (op.profile && tm) {
      // sweeps that ran (the kernels return at once after convergence)
      const int ran = host_ctrl[1] - prev_iter;
      for (int i = 0; i < k && i < ran; ++i) {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, ev[3 * i], ev[3 * i + 1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, ev[3 * i + 1], ev[3 * i + 2]) == cudaSuccess) {
          tm->sweep_ms += a;
          tm->finalize_ms += b;
          tm->n_sweeps += 1;
        } else {
          cudaGetLastError();  // timing unavailable: keep the solve's error state clean
        }
      }
    }
    prev_iter = host_ctrl[1];
    if (host_ctrl[0]) break;
    if (launched > op.max_iter + k) {  // defensive: the device test stops at max_iter
      rc = ctx->fail(OBTE_NOT_CONVERGED, "iteration cap reached");
      break;
    }
  }
  *iters = host_ctrl[1];
  *done_code = host_ctrl[0];
  if (!op.use_graph) ctx->drop_graph();
  cudaFreeHost(host_ctrl);
  return rc;
}

extern "C" int obte_solve(obte_ctx* ctx, const obte_solve_opts* opts, obte_solve_stats* stats) {
  if (!ctx) return OBTE_EINVAL;
  if (!ctx->has_mesh || !ctx->has_material) return ctx->fail(OBTE_ESTATE, "create_mesh and set_material first");
  if (ctx->shard_n > 1)
    return ctx->fail(OBTE_ESTATE, "context holds one shard of the ordinates: iterate with obte_shard_*");
  obte_solve_opts op;
  if (opts) op = *opts;
  else obte_default_opts(&op);
  if (op.precision != OBTE_FP64 && op.precision != OBTE_MIXED) return ctx->fail(OBTE_EINVAL, "bad precision");
  if (op.max_iter < 1) return ctx->fail(OBTE_EINVAL, "max_iter must be >= 1");
  if (op.check_every < 1) op.check_every = 1;
  cudaSetDevice(ctx->device);
  const int prec = op.precision == OBTE_FP64 ? 0 : 1;
  Variant v;
  int rc = (op.group_size < 0) ? autotune(ctx, prec, op, &v) : pick_variant(ctx, prec, op, &v);
  if (rc) return rc;
  rc = prepare_state(ctx, prec, v.G, v.R, v.warp, op.max_iter, op, v.k3d, v.nh);
  if (rc) return rc;
  ctx->flux_done = false;
  cudaEvent_t e0, e1, e2;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventCreate(&e2));
  CK(cudaEventRecord(e0, ctx->stream));
  int fiters = 0;
  int* fi_host = nullptr;
  CK(cudaMallocHost(&fi_host, sizeof(int)));
  rc = init_from_fourier(ctx, op, fi_host);
  if (rc) {
    cudaFreeHost(fi_host);
    return rc;
  }
  CK(cudaEventRecord(e1, ctx->stream));
  int iters = 0, done = 0;
  IterTiming tm;
  rc = run_iterations(ctx, op, &iters, &done, &tm);
  CK(cudaEventRecord(e2, ctx->stream));
  CK(cudaEventSynchronize(e2));
  fiters = *fi_host;
  cudaFreeHost(fi_host);
  float t_f = 0, t_i = 0;
  cudaEventElapsedTime(&t_f, e0, e1);
  cudaEventElapsedTime(&t_i, e1, e2);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (rc && rc != OBTE_NOT_CONVERGED) return rc;
  std::vector<double> hist(std::min(iters, kMaxHist));
  double scal[4];
  if (!hist.empty())
    CK(cudaMemcpy(hist.data(), ctx->hist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(scal, ctx->scal, sizeof(double) * 4, cudaMemcpyDeviceToHost));
  ctx->kappa = hist.empty() ? NAN : hist.back();
  ctx->last_iters = iters;
  ctx->last_opts = op;
  ctx->solved = true;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iterations = iters;
    stats->fourier_iterations = fiters;
    stats->converged = done == 1;
    stats->kappa_eff = ctx->kappa;
    stats->delta_TL = scal[2];
    stats->time_fourier_ms = t_f;
    stats->time_iter_ms = t_i;
    stats->time_total_ms = t_f + t_i;
    stats->updates_per_s = t_i > 0 ? (double)ctx->n_solid * ctx->O * iters / (t_i * 1e-3) : 0.0;
    stats->group_size = ctx->G;
    stats->rows_per_thread = ctx->R;
    stats->threads_per_block = ctx->threads;
    stats->kernel = ctx->warp ? 2 : (ctx->k3d ? 3 : 1);
    stats->n_groups = (int)ctx->items_h.size();
    stats->n_history = (int)hist.size();
    for (size_t i = 0; i < hist.size(); ++i) stats->kappa_history[i] = hist[i];
    stats->n_sweeps = tm.n_sweeps;
    stats->time_sweep_ms = tm.sweep_ms;
    stats->time_finalize_ms = tm.finalize_ms;
  }
  if (done == 3) return ctx->fail(OBTE_ENONFINITE, "non-finite value in the iterate");
  if (done != 1) return ctx->fail(OBTE_NOT_CONVERGED, "stopping test not met within max_iter");
  return OBTE_OK;
}

// ---------------------------------------------------------------------------
// ordinate sharding of one solve (Sec. 3: directions spread over processors)
// ---------------------------------------------------------------------------
extern "C" int obte_set_shard(obte_ctx* ctx, int rank, int n_ranks) {
  if (!ctx) return OBTE_EINVAL;
  if (n_ranks < 1 || rank < 0 || rank >= n_ranks) return ctx->fail(OBTE_EINVAL, "need 0 <= rank < n_ranks");
  ctx->drop_graph();
  ctx->shard_rank = rank;
  ctx->shard_n = n_ranks;
  ctx->shard_active = false;
  ctx->solved = false;
  ctx->precision = -1;  // work items are rebuilt by the next begin
  return OBTE_OK;
}

extern "C" size_t obte_shard_partials_count(const obte_ctx* ctx) {
  if (!ctx || !ctx->has_mesh) return 0;
  return (size_t)ctx->n_cells + (size_t)ctx->n_walls + 1;
}

extern "C" int obte_shard_begin(obte_ctx* ctx, const obte_solve_opts* opts) {
  if (!ctx) return OBTE_EINVAL;
  if (!ctx->has_mesh || !ctx->has_material) return ctx->fail(OBTE_ESTATE, "create_mesh and set_material first");
  obte_solve_opts op;
  if (opts) op = *opts;
  else obte_default_opts(&op);
  if (op.precision != OBTE_FP64 && op.precision != OBTE_MIXED) return ctx->fail(OBTE_EINVAL, "bad precision");
  if (op.max_iter < 1) return ctx->fail(OBTE_EINVAL, "max_iter must be >= 1");
  if (op.group_size < 0) return ctx->fail(OBTE_EINVAL, "a sharded solve needs a fixed variant (group_size >= 0)");
  if (op.accel != 0) return ctx->fail(OBTE_EINVAL, "a sharded solve runs the plain source iteration (accel = 0)");
  CK(cudaSetDevice(ctx->device));
  const int prec = op.precision == OBTE_FP64 ? 0 : 1;
  Variant v;
  int rc = pick_variant(ctx, prec, op, &v);
  if (rc) return rc;
  rc = prepare_state(ctx, prec, v.G, v.R, v.warp, op.max_iter, op, v.k3d, v.nh);
  if (rc) return rc;
  ctx->flux_done = false;
  rc = init_from_fourier(ctx, op, nullptr);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->last_opts = op;
  ctx->last_iters = 0;
  ctx->kappa = NAN;
  ctx->solved = false;
  ctx->shard_active = true;
  return OBTE_OK;
}

extern "C" int obte_shard_sweep(obte_ctx* ctx, double* partials) {
  if (!ctx || !partials) return OBTE_EINVAL;
  if (!ctx->shard_active) return ctx->fail(OBTE_ESTATE, "obte_shard_begin first");
  CK(cudaSetDevice(ctx->device));
  CK(sweep_once(ctx, 0));
  CK(launch_shard_export(ctx->gd, partials, finalize_blocks(ctx->n_cells), ctx->stream));
  return OBTE_OK;
}

extern "C" int obte_shard_finalize(obte_ctx* ctx, const double* partials, int* done) {
  if (!ctx || !partials) return OBTE_EINVAL;
  if (!ctx->shard_active) return ctx->fail(OBTE_ESTATE, "obte_shard_begin first");
  CK(cudaSetDevice(ctx->device));
  CK(launch_shard_import(ctx->gd, partials, finalize_blocks(ctx->n_cells), ctx->stream));
  CK(launch_finalize(ctx->gd, 1, ctx->precision, finalize_blocks(ctx->n_cells), ctx->stream));
  if (ctx->gh.psi) CK(launch_psi_records(ctx->gd, 1, ctx->precision, finalize_blocks(ctx->n_cells), ctx->stream));
  int ctrl[4];
  CK(cudaMemcpyAsync(ctrl, ctx->ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int iters = ctrl[1];
  if (iters >= 1 && iters <= kMaxHist) {
    double k = NAN;
    CK(cudaMemcpy(&k, ctx->hist + (iters - 1), sizeof(double), cudaMemcpyDeviceToHost));
    ctx->kappa = k;
  }
  ctx->last_iters = iters;
  ctx->solved = true;
  if (done) *done = ctrl[0];
  if (ctrl[0] == 3) return ctx->fail(OBTE_ENONFINITE, "non-finite value in the iterate");
  return OBTE_OK;
}

// ---------------------------------------------------------------------------
// outputs
// ---------------------------------------------------------------------------
template <typename F>
static void to_user(const obte_ctx* ctx, F&& per_cell) {
  const int Nx = ctx->n[0], Ny = ctx->n[1];
  for (int c = 0; c < ctx->n_cells; ++c) {
    const int kc[3] = {c % Nx, (c / Nx) % Ny, c / (Nx * Ny)};
    int u[3];
    for (int i = 0; i < 3; ++i) u[ctx->perm[i]] = kc[i];
    const long ui = u[0] + (long)ctx->user_n[0] * (u[1] + (long)ctx->user_n[1] * u[2]);
    per_cell(c, ui);
  }
}

extern "C" int obte_get_kappa_eff(obte_ctx* ctx, double* out) {
  if (!ctx || !out) return OBTE_EINVAL;
  if (!ctx->solved) return ctx->fail(OBTE_ESTATE, "solve first");
  *out = ctx->kappa;
  return OBTE_OK;
}

extern "C" int obte_get_T_L(obte_ctx* ctx, double* out) {
  if (!ctx || !out) return OBTE_EINVAL;
  if (!ctx->solved) return ctx->fail(OBTE_ESTATE, "solve first");
  cudaSetDevice(ctx->device);
  double* tmp = ctx->dalloc_t<double>(ctx->n_cells);
  NEED(tmp);
  CK(launch_gauge(ctx->code_d, ctx->TL, ctx->n_cells, tmp, nullptr, ctx->stream));
  std::vector<double> k(ctx->n_cells);
  CK(cudaMemcpyAsync(k.data(), tmp, sizeof(double) * ctx->n_cells, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->dfree(tmp);
  to_user(ctx, [&](int c, long ui) { out[ui] = k[c]; });
  return OBTE_OK;
}

static int run_flux_pass(obte_ctx* ctx) {
  if (ctx->flux_done) return OBTE_OK;
  cudaSetDevice(ctx->device);
  if (!ctx->J_acc) ctx->J_acc = ctx->dalloc_t<double>((size_t)ctx->n_cells * 3);
  if (!ctx->phi_sec) ctx->phi_sec = ctx->dalloc_t<double>(ctx->n[0]);
  if (!ctx->phi_bin) ctx->phi_bin = ctx->dalloc_t<double>(ctx->M);
  NEED(ctx->J_acc);
  NEED(ctx->phi_sec);
  NEED(ctx->phi_bin);
  CK(cudaMemsetAsync(ctx->J_acc, 0, sizeof(double) * ctx->n_cells * 3, ctx->stream));
  CK(cudaMemsetAsync(ctx->phi_sec, 0, sizeof(double) * ctx->n[0], ctx->stream));
  CK(cudaMemsetAsync(ctx->phi_bin, 0, sizeof(double) * ctx->M, ctx->stream));
  ctx->gh.J_acc = ctx->J_acc;
  ctx->gh.phi_sec = ctx->phi_sec;
  ctx->gh.phi_bin = ctx->phi_bin;
  int zero = 0;
  CK(cudaMemcpyAsync(ctx->gd, &ctx->gh, sizeof(GeomDev), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->ctrl, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));  // done = 0
  CK(sweep_once(ctx, SWEEP_FLUX));
  // the pass does not advance the iterate: drop its moment accumulations
  CK(cudaMemsetAsync(ctx->TL_acc, 0, sizeof(double) * ctx->n_cells, ctx->stream));
  if (ctx->tlq) CK(cudaMemsetAsync(ctx->tlq, 0, sizeof(double) * (ctx->dim == 3 ? 8 : 4) * (size_t)ctx->n_cells, ctx->stream));
  CK(cudaMemsetAsync(ctx->wall_acc, 0, sizeof(double) * 6 * (size_t)ctx->n_cells, ctx->stream));
  CK(cudaMemsetAsync(ctx->scal, 0, sizeof(double), ctx->stream));
  int one = 1;
  CK(cudaMemcpyAsync(ctx->ctrl, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->flux_done = true;
  return OBTE_OK;
}

extern "C" int obte_get_flux(obte_ctx* ctx, double* out) {
  if (!ctx || !out) return OBTE_EINVAL;
  if (!ctx->solved) return ctx->fail(OBTE_ESTATE, "solve first");
  int rc = run_flux_pass(ctx);
  if (rc) return rc;
  std::vector<double> J((size_t)ctx->n_cells * 3);
  CK(cudaMemcpy(J.data(), ctx->J_acc, sizeof(double) * J.size(), cudaMemcpyDeviceToHost));
  const int dim = ctx->dim;
  to_user(ctx, [&](int c, long ui) {
    const bool solid = ctx->code_h[c] & CODE_SOLID;
    for (int i = 0; i < dim; ++i) {
      const int ua = ctx->perm[i];
      out[ui * dim + ua] = solid ? J[3 * (size_t)c + i] : NAN;
    }
  });
  return OBTE_OK;
}

extern "C" int obte_get_section_flux(obte_ctx* ctx, double* out) {
  if (!ctx || !out) return OBTE_EINVAL;
  if (!ctx->solved) return ctx->fail(OBTE_ESTATE, "solve first");
  int rc = run_flux_pass(ctx);
  if (rc) return rc;
  std::vector<double> p(ctx->n[0]);
  CK(cudaMemcpy(p.data(), ctx->phi_sec, sizeof(double) * p.size(), cudaMemcpyDeviceToHost));
  for (int i = 0; i < ctx->n[0]; ++i) out[i] = ctx->kappa_scale * p[i];
  return OBTE_OK;
}

extern "C" int obte_get_kappa_bins(obte_ctx* ctx, double* out) {
  if (!ctx || !out) return OBTE_EINVAL;
  if (!ctx->solved) return ctx->fail(OBTE_ESTATE, "solve first");
  int rc = run_flux_pass(ctx);
  if (rc) return rc;
  std::vector<double> p(ctx->M);
  CK(cudaMemcpy(p.data(), ctx->phi_bin, sizeof(double) * p.size(), cudaMemcpyDeviceToHost));
  for (int m = 0; m < ctx->M; ++m) out[m] = ctx->kappa_scale * p[m];
  return OBTE_OK;
}

// ---------------------------------------------------------------------------
// Fourier model alone (App. B)
// ---------------------------------------------------------------------------
extern "C" int obte_solve_fourier(obte_ctx* ctx, double tol, int max_iter, double* kappa_out,
                                  double* T_out, int* iters_out) {
  if (!ctx) return OBTE_EINVAL;
  if (!ctx->has_mesh || !ctx->has_material) return ctx->fail(OBTE_ESTATE, "create_mesh and set_material first");
  if (!kappa_out) return ctx->fail(OBTE_EINVAL, "kappa_out is NULL");
  if (!std::isfinite(tol) || tol < 0.0) return ctx->fail(OBTE_EINVAL, "tol must be finite and >= 0");
  if (max_iter < 0) return ctx->fail(OBTE_EINVAL, "max_iter must be >= 0");
  cudaSetDevice(ctx->device);
  if (tol == 0.0) tol = 1e-12;
  if (max_iter == 0) max_iter = 40 * (ctx->n[0] + ctx->n[1] + ctx->n[2]);
  const size_t n = (size_t)ctx->n_cells;
  const size_t nwork = fourier_work_doubles(ctx->n_cells, kFourierBlocksMax);
  // one scratch array: the block-form job, T, the CG vectors, the flux sum, the count
  const size_t job_bytes = (sizeof(CGArgs) + 15) / 16 * 16;
  char* buf = static_cast<char*>(ctx->dalloc(job_bytes + sizeof(double) * (n + nwork + 1) + 16));
  NEED(buf);
  CGArgs* job_d = reinterpret_cast<CGArgs*>(buf);
  double* Tf = reinterpret_cast<double*>(buf + job_bytes);
  double* work = Tf + n;
  double* flux_d = work + nwork;
  int* it_d = reinterpret_cast<int*>(flux_d + 1);
  GeomDev g{};
  g.code = ctx->code_d;
  g.nx = ctx->n[0];
  g.ny = ctx->n[1];
  g.nz = ctx->n[2];
  g.dim = ctx->dim;
  g.n_cells = ctx->n_cells;
  g.py = ctx->periodic[1];
  g.pz = ctx->dim == 3 ? ctx->periodic[2] : 0;
  g.dT = ctx->dT;
  double he[3];
  cg_spacing(ctx, he);
  double flux = 0.0;
  int its = 0;
  std::vector<double> Th(T_out ? n : 0);
  auto run = [&]() -> int {
    if (ctx->n_cells <= 4096) {  // one block, no grid-wide synchronisation
      const CGArgs job = make_cg_args(g, he[0], he[1], he[2], max_iter, tol, Tf, it_d, work,
                                      kFourierBlocksMax);
      CK(cudaMemcpyAsync(job_d, &job, sizeof(CGArgs), cudaMemcpyHostToDevice, ctx->stream));
      CK(launch_fourier_cg_blocks(job_d, 1, 0, ctx->stream));
    } else {
      CK(launch_fourier_cg(g, he[0], he[1], he[2], 0, max_iter, tol, Tf, it_d, work,
                           kFourierBlocksMax, ctx->stream));
    }
    CK(launch_fourier_hot_flux(ctx->code_d, Tf, ctx->n[0], ctx->n[1] * ctx->n[2], ctx->dT, flux_d,
                               ctx->stream));
    CK(cudaMemcpyAsync(&flux, flux_d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&its, it_d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (T_out) CK(cudaMemcpyAsync(Th.data(), Tf, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OBTE_OK;
  };
  const int rc = run();
  if (rc) cudaStreamSynchronize(ctx->stream);  // nothing in flight uses the scratch when it is freed
  ctx->dfree(buf);
  if (rc) return rc;
  // kappa_fourier = L / (dT A_sec) sum_faces kappa_xx (T_image + dT - T_cell) / h_x
  *kappa_out = ctx->kappa_scale * ctx->kappa_axes[0] / ctx->h[0] * flux;
  if (iters_out) *iters_out = its;
  if (T_out)
    to_user(ctx, [&](int c, long ui) { T_out[ui] = (ctx->code_h[c] & CODE_SOLID) ? Th[c] : NAN; });
  if (its >= max_iter) return ctx->fail(OBTE_NOT_CONVERGED, "Fourier CG: residual test not met within max_iter");
  return OBTE_OK;
}

// ---------------------------------------------------------------------------
// d kappa / d s
// ---------------------------------------------------------------------------
// Batches of reversed ordinate pairs (o, rev(o)) for the gradient's record
// passes, o running over the first octant of each reversed octant pair; up to
// cap pairs per batch, octant pairs merged, so that a record pass holds as
// many groups as the field budget allows.
static std::vector<std::vector<int>> grad_batches(const obte_ctx* ctx, size_t cap) {
  const int O = ctx->O;
  std::vector<std::pair<int, int>> pairs;
  int o = 0;
  while (o < O) {
    const int q = ctx->octant[o];
    int e1 = o;
    while (e1 < O && ctx->octant[e1] == q) ++e1;
    int e2 = e1;
    while (e2 < O && ctx->octant[e2] == ctx->octant[e1]) ++e2;
    for (int k = o; k < e1; ++k) pairs.push_back({k, ctx->rev_o[k]});
    o = e2;
  }
  std::vector<std::vector<int>> batches;
  for (size_t a = 0; a < pairs.size(); a += cap) {
    std::vector<int> b;
    for (size_t k = a; k < std::min(pairs.size(), a + cap); ++k) {
      b.push_back(pairs[k].first);
      b.push_back(pairs[k].second);
    }
    batches.push_back(b);
  }
  return batches;
}

extern "C" int obte_kappa_grad_s(obte_ctx* ctx, double* out, size_t max_field_bytes) {
  if (!ctx || !out) return OBTE_EINVAL;
  if (!ctx->solved) return ctx->fail(OBTE_ESTATE, "solve first");
  if (ctx->shard_n > 1) return ctx->fail(OBTE_ESTATE, "gradient of a sharded solve is not available");
  cudaSetDevice(ctx->device);
  const int O = ctx->O;
  // reversed ordinate of every sorted ordinate (same bin, opposite direction)
  // (paired when the material was set: same bin, MFP and weight, opposite direction)
  const std::vector<int>& rev = ctx->rev_o;
  for (int o = 0; o < O; ++o)
    if (rev[o] < 0) return ctx->fail(OBTE_EINVAL, "direction set is not symmetric under p -> -p");
  if (max_field_bytes == 0) max_field_bytes = (size_t)1 << 30;
  const size_t e = ctx->precision == 0 ? 8 : 4;
  const size_t per_ord = e * (size_t)ctx->n_cells;
  // batches: whole reversed octant pairs when they fit, else matching slices
  const std::vector<std::vector<int>> batches =
      grad_batches(ctx, std::max<size_t>(1, max_field_bytes / (2 * per_ord)));
  size_t max_b = 0;
  for (auto& b : batches) max_b = std::max(max_b, b.size());
  void* rec = ctx->dalloc(per_ord * max_b);
  int* slot_d = ctx->dalloc_t<int>(O);
  int* revl_d = ctx->dalloc_t<int>(max_b);
  double* a_d = ctx->dalloc_t<double>(max_b);
  double* grad_d = ctx->dalloc_t<double>(ctx->n_cells);
  NEED(rec);
  NEED(slot_d);
  NEED(revl_d);
  NEED(a_d);
  NEED(grad_d);
  CK(cudaMemsetAsync(grad_d, 0, sizeof(double) * ctx->n_cells, ctx->stream));
  // adjoint jump: -(L_x / (dT N_sec)) h_x W, W the sum of the E2 weights before
  // normalisation (d_ang sum kappa_m / Lambda_m^2 for the bin-separable set); the
  // adjoint field of o is jscale * T_rev(o) (up to a constant that cancels)
  const double jadj = -ctx->kappa_scale * ctx->h[0] * ctx->w_total;
  const double jscale = jadj / ctx->dT;
  std::vector<int> slot(O);
  std::vector<WorkItem> all_items = ctx->items_h;
  int one = 1, zero = 0;
  for (auto& b : batches) {
    std::fill(slot.begin(), slot.end(), -1);
    for (size_t k2 = 0; k2 < b.size(); ++k2) slot[b[k2]] = (int)k2;
    std::vector<int> revl(b.size());
    std::vector<double> ab(b.size());
    for (size_t k2 = 0; k2 < b.size(); ++k2) {
      revl[k2] = slot[rev[b[k2]]];
      ab[k2] = ctx->aw[b[k2]];
    }
    // work items that hold a recorded ordinate
    std::vector<WorkItem> its;
    for (auto& it : all_items) {
      bool any = false;
      for (int o = it.o0; o < it.o0 + it.count; ++o)
        if (slot[o] >= 0) any = true;
      if (any) its.push_back(it);
    }
    WorkItem* its_d = ctx->dalloc_t<WorkItem>(its.size());
    NEED(its_d);
    CK(cudaMemcpyAsync(its_d, its.data(), sizeof(WorkItem) * its.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(slot_d, slot.data(), sizeof(int) * O, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(revl_d, revl.data(), sizeof(int) * b.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(a_d, ab.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice, ctx->stream));
    GeomDev g = ctx->gh;
    g.rec = rec;
    g.rec_slot = slot_d;
    CK(cudaMemcpyAsync(ctx->gd, &g, sizeof(GeomDev), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->ctrl, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    SweepLaunch L;
    L.geoms = ctx->gd;
    L.items = its_d;
    L.n_items = (int)its.size();
    L.flags = SWEEP_RECORD;
    L.item_counter = nullptr;
    if (ctx->warp) {
      CK(launch_ctx_warp(ctx, L));
    } else if (ctx->k3d) {
      CK(launch_sweep3d(L, ctx->precision, ctx->G, ctx->R, ctx->has_s, ctx->threads,
                        sweep3d_smem_bytes(ctx->precision, ctx->G, ctx->R, ctx->threads), ctx->stream));
    } else {
      const size_t smem = sweep_smem_bytes(ctx->precision, ctx->dim, ctx->G, ctx->R, ctx->threads);
      CK(launch_sweep(L, ctx->precision, ctx->dim, ctx->G, ctx->R, ctx->has_s, ctx->threads,
                      L.n_items, smem, ctx->stream));
    }
    CK(launch_grad_contract2(ctx->code_d, ctx->TL, ctx->n_cells, rec, (int)b.size(), revl_d, a_d,
                             jscale, grad_d, ctx->precision, ctx->gh.psi, ctx->stream));
    CK(cudaMemsetAsync(ctx->TL_acc, 0, sizeof(double) * ctx->n_cells, ctx->stream));
    if (ctx->tlq) CK(cudaMemsetAsync(ctx->tlq, 0, sizeof(double) * (ctx->dim == 3 ? 8 : 4) * (size_t)ctx->n_cells, ctx->stream));
    CK(cudaMemsetAsync(ctx->wall_acc, 0, sizeof(double) * 6 * (size_t)ctx->n_cells, ctx->stream));
    CK(cudaMemsetAsync(ctx->scal, 0, sizeof(double), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->dfree(its_d);
  }
  CK(cudaMemcpyAsync(ctx->gd, &ctx->gh, sizeof(GeomDev), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->ctrl, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<double> gk(ctx->n_cells);
  CK(cudaMemcpyAsync(gk.data(), grad_d, sizeof(double) * ctx->n_cells, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (void* p : {rec, (void*)slot_d, (void*)revl_d, (void*)a_d, (void*)grad_d}) ctx->dfree(p);
  to_user(ctx, [&](int c, long ui) { out[ui] = (ctx->code_h[c] & CODE_SOLID) ? gk[c] : 0.0; });
  return OBTE_OK;
}

// ---------------------------------------------------------------------------
// batched solve: many geometries, one persistent sweep launch per iteration
// ---------------------------------------------------------------------------
// Timed choice of the batch form (opts.group_size = -1).  The compiled
// variants allow up to three forms for a batch: fixed-rows class launches
// (mixed precision without s(x), rows per lane chosen per geometry), one
// persistent launch of the warp kernel over a cost-sorted work queue (general
// rows per lane), and one persistent launch of the block kernel.  Each form
// the batch accepts runs the same fixed number of iterations twice from the
// Fourier guess (the first run pays for module loading and graph
// instantiation); the fastest second run is kept per batch shape
// (precision, dimension, and every geometry's cells per axis, ordinates and
// s(x) flag) and returned in *best as explicit options.
static std::map<std::vector<int>, std::tuple<int, int, int>>& batch_tune_cache() {
  static std::map<std::vector<int>, std::tuple<int, int, int>> c;
  return c;
}

static int batch_autotune(obte_ctx* const* ctxs, int n, const obte_solve_opts& op,
                          obte_solve_opts* best) {
  std::vector<int> key{op.precision, ctxs[0]->dim, n, op.accel};
  for (int i = 0; i < n; ++i) {
    const obte_ctx* c = ctxs[i];
    key.insert(key.end(), {c->n[0], c->n[1], c->n[2], c->O, c->has_s ? 1 : 0});
  }
  // (group_size, rows_per_thread, kernel) of each form; 0 leaves the choice
  // inside the form to the batch solver's rules
  const std::tuple<int, int, int> forms[3] = {
      std::make_tuple(0, 0, 0),  // fixed-rows classes where they apply
      std::make_tuple(0, 8, 0),  // persistent warp queue, general rows per lane
      std::make_tuple(0, 0, 1)}; // persistent block kernel
  auto with = [&](const std::tuple<int, int, int>& f) {
    obte_solve_opts o = op;
    o.group_size = std::get<0>(f);
    o.rows_per_thread = std::get<1>(f);
    o.kernel = std::get<2>(f);
    return o;
  };
  {
    std::lock_guard<std::mutex> lock(tune_mutex());
    auto hit = batch_tune_cache().find(key);
    if (hit != batch_tune_cache().end()) {
      *best = with(hit->second);
      return OBTE_OK;
    }
  }
  std::vector<obte_solve_stats> st(n);
  double best_ms = 1e300;
  int bi = -1;
  for (int f = 0; f < 3; ++f) {
    obte_solve_opts t = with(forms[f]);
    t.tol = 0.0;
    t.tol_TL = 0.0;
    t.min_iter = 0;
    t.profile = 0;
    t.check_every = std::max(1, op.check_every);
    t.max_iter = 4 * t.check_every;
    double ms = 0.0;
    int rc = OBTE_OK;
    for (int rep = 0; rep < 2 && (rc == OBTE_OK || rc == OBTE_NOT_CONVERGED); ++rep) {
      rc = obte_solve_batch(ctxs, n, &t, st.data());
      ms = st[0].time_iter_ms;
    }
    if (rc == OBTE_EINVAL) continue;  // this batch does not fit the form
    if (rc != OBTE_OK && rc != OBTE_NOT_CONVERGED) return rc;
    if (ms < best_ms) {
      best_ms = ms;
      bi = f;
    }
  }
  if (bi < 0) return ctxs[0]->fail(OBTE_EINVAL, "no batch form fits every geometry");
  {
    std::lock_guard<std::mutex> lock(tune_mutex());
    batch_tune_cache()[key] = forms[bi];
  }
  *best = with(forms[bi]);
  return OBTE_OK;
}

extern "C" int obte_solve_batch(obte_ctx* const* ctxs, int n, const obte_solve_opts* opts,
                                obte_solve_stats* stats) {
  if (!ctxs || n < 1 || !ctxs[0]) return OBTE_EINVAL;
  obte_ctx* ctx = ctxs[0];  // owns the batch buffers and the stream
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return ctx->fail(OBTE_EINVAL, "null context in batch");
    if (!ctxs[i]->has_mesh || !ctxs[i]->has_material)
      return ctx->fail(OBTE_ESTATE, "every context needs create_mesh and set_material");
    if (ctxs[i]->device != ctx->device || ctxs[i]->dim != ctx->dim)
      return ctx->fail(OBTE_EINVAL, "batch contexts must share device and dimension");
    if (ctxs[i]->shard_n > 1) return ctx->fail(OBTE_ESTATE, "sharded contexts cannot join a batch");
  }
  obte_solve_opts op;
  if (opts) op = *opts;
  else obte_default_opts(&op);
  if (op.precision != OBTE_FP64 && op.precision != OBTE_MIXED) return ctx->fail(OBTE_EINVAL, "bad precision");
  if (op.max_iter < 1) return ctx->fail(OBTE_EINVAL, "max_iter must be >= 1");
  const int prec = op.precision == OBTE_FP64 ? 0 : 1;
  cudaSetDevice(ctx->device);
  if (op.group_size < 0) {
    obte_solve_opts tuned;
    const int rc = batch_autotune(ctxs, n, op, &tuned);
    if (rc) return rc;
    return obte_solve_batch(ctxs, n, &tuned, stats);
  }
  // 2D: the warp kernel with per-geometry rows per lane (R <= 8 dividing ny,
  // ny / R <= 32 lanes); otherwise a block-kernel variant every geometry accepts
  bool any_s = false;
  for (int i = 0; i < n; ++i) any_s = any_s || ctxs[i]->has_s;
  int max_ny = 0, max_nz = 0;
  for (int i = 0; i < n; ++i) {
    max_ny = std::max(max_ny, ctxs[i]->n[1]);
    max_nz = std::max(max_nz, ctxs[i]->n[2]);
  }
  const int wG = prec ? 8 : 4, wR = 8;
  std::vector<int> r_eff(n, 0);
  bool use_warp = ctx->dim == 2 && op.kernel != 1 && sweep2d_warp_exists(prec, wG, wR, any_s, false) &&
                  (op.group_size <= 0 || op.group_size == wG);
  for (int i = 0; use_warp && i < n; ++i) {
    const int ny = ctxs[i]->n[1];
    if (ctxs[i]->n_cells > kMaxSkewCells) use_warp = false;
    for (int R = 1; R <= wR; ++R)
      if (ny % R == 0 && ny / R <= 32) {
        r_eff[i] = R;
        break;
      }
    if (!r_eff[i]) use_warp = false;
  }
  // Fixed-rows classes (mixed precision without s(x)): every geometry runs the
  // compiled fixed-R instance with the most lanes in use (R in 1 .. 6 or 8
  // dividing N with N / R <= 32 lanes); the geometries of one class share a
  // launch, the classes run side by side on forked streams, and a class whose
  // rows fill the 32 lanes adds the four warps' moments in shared memory
  bool use_cls = use_warp && prec == 1 && !any_s && op.rows_per_thread <= 0;
  {
    std::vector<int> r_cls(n, 0);
    for (int i = 0; use_cls && i < n; ++i) {
      const int ny = ctxs[i]->n[1];
      for (int R : {1, 2, 3, 4, 5, 6, 8})
        if (ny % R == 0 && ny / R <= 32 && sweep2d_warp_exists(prec, wG, R, false, true)) {
          r_cls[i] = R;
          break;
        }
      if (!r_cls[i]) use_cls = false;
    }
    if (use_cls) r_eff = r_cls;
  }
  Variant v{0, 0, false};
  if (!use_warp) {
    std::vector<Variant> common;
    for (auto& c : candidates(prec, ctx->dim, max_ny, max_nz, any_s)) {
      if (c.warp || c.k3d) continue;  // batches of 3D meshes use the plain block kernel
      bool ok = true;
      for (int i = 0; i < n; ++i)
        if (ctxs[i]->n[1] % c.R != 0) ok = false;
      if ((op.group_size > 0 && c.G != op.group_size) || (op.rows_per_thread > 0 && c.R != op.rows_per_thread))
        ok = false;
      if (ok) common.push_back(c);
    }
    if (common.empty()) return ctx->fail(OBTE_EINVAL, "no compiled sweep variant fits every geometry");
    v = common[0];
  } else {
    v = Variant{wG, wR, true};
  }
  for (int i = 0; i < n; ++i) {
    int rc = prepare_state(ctxs[i], prec, v.G, use_warp ? r_eff[i] : v.R, v.warp, op.max_iter, op);
    if (rc) return ctx->fail(rc, std::string("batch member: ") + ctxs[i]->err);
    ctxs[i]->flux_done = false;
  }
  const int wpb = v.warp ? sweep2d_warps_per_block(prec, v.G, v.R, any_s, false) : 0;
  const int threads = v.warp ? 32 * wpb : threads_for(max_ny, max_nz, v.R);
  const size_t smem = v.warp ? 0 : sweep_smem_bytes(prec, ctx->dim, v.G, v.R, threads);
  // contiguous geometry table and a work list sorted by cost (largest first)
  GeomDev* gds = ctx->dalloc_t<GeomDev>(n);
  NEED(gds);
  std::vector<GeomDev> gh(n);
  std::vector<WorkItem> items;
  struct ItemClass {
    int R;
    bool full;      // rows fill 32 lanes: items in blocks of four of one octant, moments combined
    size_t off, count;
  };
  std::vector<ItemClass> classes;
  for (int i = 0; i < n; ++i) gh[i] = ctxs[i]->gh;
  if (use_cls) {
    // per class: the geometries' items (padded as their starting state
    // assumed), blocks of four kept together, costliest first
    std::vector<std::pair<int, bool>> keys;
    for (int i = 0; i < n; ++i) {
      const std::pair<int, bool> key(r_eff[i], ctxs[i]->items_pad == 4);
      if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
    }
    for (const auto& key : keys) {
      const int pad = key.second ? 4 : 1;
      std::vector<std::vector<WorkItem>> chunks;
      for (int i = 0; i < n; ++i) {
        if (r_eff[i] != key.first || (ctxs[i]->items_pad == 4) != key.second) continue;
        std::vector<WorkItem> it;
        build_items(ctxs[i], i, v.G, it, nullptr, ctxs[i]->items_pad);
        for (size_t a = 0; a < it.size(); a += pad)
          chunks.emplace_back(it.begin() + a, it.begin() + std::min(it.size(), a + pad));
      }
      auto cost = [&](const std::vector<WorkItem>& c) {
        long w = 0;
        for (const WorkItem& x : c) w += (long)gh[x.geom].n_cells * x.count;
        return w;
      };
      std::stable_sort(chunks.begin(), chunks.end(),
                       [&](const std::vector<WorkItem>& a, const std::vector<WorkItem>& b) { return cost(a) > cost(b); });
      ItemClass c{key.first, key.second, items.size(), 0};
      for (auto& ch : chunks) items.insert(items.end(), ch.begin(), ch.end());
      c.count = items.size() - c.off;
      classes.push_back(c);
    }
  } else {
    for (int i = 0; i < n; ++i) build_items(ctxs[i], i, v.G, items, nullptr, ctxs[i]->items_pad);
    std::stable_sort(items.begin(), items.end(), [&](const WorkItem& a, const WorkItem& b) {
      return (long)gh[a.geom].n_cells * a.count > (long)gh[b.geom].n_cells * b.count;
    });
  }
  // one stream per class, forked from and joined back into the solve's stream
  std::vector<cudaStream_t> side(classes.size(), nullptr);
  std::vector<cudaEvent_t> joined(classes.size(), nullptr);
  cudaEvent_t forked = nullptr;
  auto drop_streams = [&]() {
    for (auto& st : side)
      if (st) cudaStreamDestroy(st);
    for (auto& ev : joined)
      if (ev) cudaEventDestroy(ev);
    if (forked) cudaEventDestroy(forked);
  };
  if (!classes.empty()) {
    CK(cudaEventCreateWithFlags(&forked, cudaEventDisableTiming));
    for (size_t c = 0; c < classes.size(); ++c) {
      CK(cudaStreamCreateWithFlags(&side[c], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&joined[c], cudaEventDisableTiming));
    }
  }
  WorkItem* items_d = ctx->dalloc_t<WorkItem>(items.size());
  int* counter = ctx->dalloc_t<int>(1);
  NEED(items_d);
  NEED(counter);
  CK(cudaMemcpyAsync(gds, gh.data(), sizeof(GeomDev) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(items_d, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice,
                     ctx->stream));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  // warp kernel: 8 resident warps per SM (the register budget of the wide groups)
  const int per_sm = v.warp ? std::max(1, 8 / std::max(1, wpb))
                            : std::max(1, sweep_blocks_per_sm(prec, ctx->dim, v.G, v.R, any_s, threads, smem));
  const int blocks = v.warp ? (int)std::min<long>(((long)items.size() + wpb - 1) / std::max(1, wpb),
                                                  (long)sms * per_sm)
                            : (int)std::min<long>((long)items.size(), (long)sms * per_sm);
  int max_cells = 0, max_ord = 0, max_rows = 0;
  for (int i = 0; i < n; ++i) {
    max_cells = std::max(max_cells, ctxs[i]->n_cells);
    max_ord = std::max(max_ord, ctxs[i]->O);
    max_rows = std::max(max_rows, ctxs[i]->n[1] * ctxs[i]->n[2]);
  }

  cudaEvent_t e0, e1, e2;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventCreate(&e2));
  CK(cudaEventRecord(e0, ctx->stream));
  // Fourier first guesses: geometries small enough for one block share one
  // launch (a block each); larger ones get the cooperative solver
  std::vector<CGArgs> jobs;
  for (int i = 0; i < n; ++i) {
    obte_ctx* c = ctxs[i];
    const int fmax = op.fourier_max_iter > 0 ? op.fourier_max_iter : 4 * (c->n[0] + c->n[1] + c->n[2]);
    const double ftol = op.fourier_tol > 0 ? op.fourier_tol : kFourierTolDefault;
    if (c->n_cells <= kBlockCGMaxCells) {
      double he[3];
      cg_spacing(c, he);
      jobs.push_back(make_cg_args(c->gh, he[0], he[1], he[2], fmax, ftol, c->TF, c->fiters,
                                  c->fwork, kFourierBlocksMax));
    } else {
      double he[3];
      cg_spacing(c, he);
      cudaError_t e = launch_fourier_cg(c->gh, he[0], he[1], he[2], prec, fmax, ftol, c->TF,
                                        c->fiters, c->fwork, kFourierBlocksMax, ctx->stream);
      if (e != cudaSuccess) return ctx->cuda_fail(e, "batch Fourier");
    }
  }
  CGArgs* jobs_d = nullptr;
  if (!jobs.empty()) {
    // largest first: clusters of the big meshes start in the first wave
    std::stable_sort(jobs.begin(), jobs.end(), [](const CGArgs& x, const CGArgs& y) {
      return (long)x.nx * x.ny * x.nz > (long)y.nx * y.ny * y.nz;
    });
    jobs_d = ctx->dalloc_t<CGArgs>(jobs.size());
    NEED(jobs_d);
    CK(cudaMemcpyAsync(jobs_d, jobs.data(), sizeof(CGArgs) * jobs.size(), cudaMemcpyHostToDevice, ctx->stream));
    const cudaError_t ec = launch_fourier_cg_cluster_jobs(jobs_d, jobs.data(), (int)jobs.size(), prec,
                                                          ctx->stream);
    if (ec == cudaErrorNotSupported) CK(launch_fourier_cg_blocks(jobs_d, (int)jobs.size(), prec, ctx->stream));
    else CK(ec);
  }
  {
    // every geometry's starting state in one launch per kernel (grid y = geometry)
    long max_work = 0;
    int max_walls = 0;
    bool any_aa = false;
    for (int i = 0; i < n; ++i) {
      max_work = std::max(max_work, std::max((long)gh[i].n_cells * 6, (long)gh[i].n_ord * gh[i].rows));
      max_walls = std::max(max_walls, gh[i].n_walls);
      any_aa = any_aa || gh[i].aa_m > 0;
    }
    cudaError_t e = launch_init_state(gds, n, max_work, max_walls, prec, ctx->stream);
    if (e == cudaSuccess && v.warp) e = launch_build_records(gds, n, prec, finalize_blocks(max_cells), ctx->stream);
    if (e == cudaSuccess && v.warp) e = launch_psi_records(gds, n, prec, finalize_blocks(max_cells), ctx->stream);
    if (e == cudaSuccess && any_aa)
      e = launch_anderson_init(gds, n, prec, aa_blocks(max_cells, max_ord, max_rows), ctx->stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "batch init");
  }
  CK(cudaEventRecord(e1, ctx->stream));
  const int k = std::max(1, op.check_every);
  auto body = [&]() -> cudaError_t {
    for (int it = 0; it < k; ++it) {
      cudaError_t e = cudaSuccess;
      if (!classes.empty()) {
        e = cudaEventRecord(forked, ctx->stream);
        for (size_t c = 0; c < classes.size() && e == cudaSuccess; ++c) {
          e = cudaStreamWaitEvent(side[c], forked, 0);
          if (e != cudaSuccess) break;
          SweepLaunch L;
          L.geoms = gds;
          L.items = items_d + classes[c].off;
          L.n_items = (int)classes[c].count;
          L.flags = classes[c].full ? SWEEP_BLOCK_COMBINE : 0;
          L.item_counter = nullptr;  // one warp per item, blocks of four items
          e = launch_sweep2d_warp(L, prec, v.G, classes[c].R, false, true, 0, side[c]);
          if (e == cudaSuccess) e = cudaEventRecord(joined[c], side[c]);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, joined[c], 0);
        }
        if (e != cudaSuccess) return e;
      } else {
        e = cudaMemsetAsync(counter, 0, sizeof(int), ctx->stream);
        if (e != cudaSuccess) return e;
        SweepLaunch L;
        L.geoms = gds;
        L.items = items_d;
        L.n_items = (int)items.size();
        L.flags = 0;
        L.item_counter = counter;
        e = v.warp ? launch_sweep2d_warp(L, prec, v.G, v.R, any_s, false, blocks, ctx->stream)
                   : launch_sweep(L, prec, ctx->dim, v.G, v.R, any_s, threads, blocks, smem, ctx->stream);
        if (e != cudaSuccess) return e;
      }
      e = launch_finalize(gds, n, prec, finalize_blocks(max_cells), ctx->stream);
      if (e != cudaSuccess) return e;
      if (op.accel > 0) {
        e = launch_anderson_step(gds, n, prec, aa_blocks(max_cells, max_ord, max_rows), ctx->stream);
        if (e != cudaSuccess) return e;
      }
      if (v.warp) {
        e = launch_psi_records(gds, n, prec, finalize_blocks(max_cells), ctx->stream);
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  };
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (op.use_graph) {
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t eb = body();
      e = cudaStreamEndCapture(ctx->stream, &graph);
      if (eb != cudaSuccess) e = eb;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      graph = nullptr;
      exec = nullptr;
    }
  }
  int* hc = nullptr;
  CK(cudaMallocHost(&hc, sizeof(int) * 4 * n));
  int rc = OBTE_OK;
  int launched = 0;
  while (true) {
    cudaError_t e = exec ? cudaGraphLaunch(exec, ctx->stream) : body();
    if (e != cudaSuccess) {
      rc = ctx->cuda_fail(e, "batch iteration");
      break;
    }
    launched += k;
    for (int i = 0; i < n && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(hc + 4 * i, ctxs[i]->ctrl, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      rc = ctx->cuda_fail(e, "batch sync");
      break;
    }
    bool all = true;
    for (int i = 0; i < n; ++i)
      if (!hc[4 * i]) all = false;
    if (all) break;
    if (launched > op.max_iter + k) break;
  }
  CK(cudaEventRecord(e2, ctx->stream));
  CK(cudaEventSynchronize(e2));
  float t_f = 0, t_i = 0;
  cudaEventElapsedTime(&t_f, e0, e1);
  cudaEventElapsedTime(&t_i, e1, e2);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  int worst = OBTE_OK;
  long total_updates = 0;
  for (int i = 0; i < n; ++i) total_updates += (long)ctxs[i]->n_solid * ctxs[i]->O * hc[4 * i + 1];
  for (int i = 0; i < n; ++i) {
    obte_ctx* c = ctxs[i];
    const int iters = hc[4 * i + 1], done = hc[4 * i];
    std::vector<double> hist(std::min(iters, kMaxHist));
    if (!hist.empty())
      CK(cudaMemcpy(hist.data(), c->hist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost));
    double scal[4];
    CK(cudaMemcpy(scal, c->scal, sizeof(double) * 4, cudaMemcpyDeviceToHost));
    c->kappa = hist.empty() ? NAN : hist.back();
    c->last_iters = iters;
    c->last_opts = op;
    c->solved = true;
    c->gh.kappa_hist = c->hist;
    CK(cudaMemcpy(c->gd, &c->gh, sizeof(GeomDev), cudaMemcpyHostToDevice));
    if (stats) {
      obte_solve_stats* s = stats + i;
      std::memset(s, 0, sizeof(*s));
      s->iterations = iters;
      s->converged = done == 1;
      s->kappa_eff = c->kappa;
      s->delta_TL = scal[2];
      s->time_fourier_ms = t_f;
      s->time_iter_ms = t_i;
      s->time_total_ms = t_f + t_i;
      s->updates_per_s = t_i > 0 ? (double)total_updates / (t_i * 1e-3) : 0.0;
      s->group_size = v.G;
      s->rows_per_thread = c->R;
      s->kernel = v.warp ? 2 : 1;
      s->threads_per_block = threads;
      s->n_groups = (int)items.size();
      s->n_history = (int)hist.size();
      for (size_t j = 0; j < hist.size(); ++j) s->kappa_history[j] = hist[j];
    }
    if (done == 3) worst = OBTE_ENONFINITE;
    else if (done != 1 && worst == OBTE_OK) worst = OBTE_NOT_CONVERGED;
  }
  cudaFreeHost(hc);
  drop_streams();
  if (jobs_d) ctx->dfree(jobs_d);
  ctx->dfree(gds);
  ctx->dfree(items_d);
  ctx->dfree(counter);
  if (rc) return rc;
  if (worst == OBTE_ENONFINITE) return ctx->fail(worst, "non-finite value in a batch member");
  if (worst == OBTE_NOT_CONVERGED) return ctx->fail(worst, "a batch member did not converge");
  return OBTE_OK;
}

// ---------------------------------------------------------------------------
// d kappa / d s without device allocation
// ---------------------------------------------------------------------------
// Some callers cannot allocate device memory when they need the gradient: a
// service that reserves its whole device-memory budget at start-up and whose
// allocator refuses new blocks afterwards, or an optimisation loop running
// next to other jobs on a GPU that is already full, where a cudaMalloc of the
// recorded fields would fail (or evict a neighbour's cached blocks) in the
// middle of a run.  For them, obte_kappa_grad_s_noalloc does the work of
// obte_kappa_grad_s with every buffer it needs beyond the context's existing
// state (recorded ordinate fields, gradient accumulator, record slots, work
// list) carved out of this fixed, file-scope device array.  The array is part
// of the library image: every GPU that loads the library holds it until the
// process exits.  The call synchronises the host with the context's stream
// between batches and copies small index tables from pageable host memory.
#define OBTE_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
static __device__ __align__(256) unsigned char g_obte_noalloc_scratch[OBTE_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device.  In host code the
// array's name only stands for the device symbol, so its address is taken once
// per device, with that device current, by cudaGetSymbolAddress.
static cudaError_t noalloc_scratch(int device, unsigned char** out) {
  static std::mutex mu;
  static std::map<int, unsigned char*> ptrs;
  std::lock_guard<std::mutex> lock(mu);
  auto it = ptrs.find(device);
  if (it != ptrs.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_obte_noalloc_scratch);
  if (e != cudaSuccess) return e;
  ptrs[device] = static_cast<unsigned char*>(p);
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

extern "C" int obte_kappa_grad_s_noalloc(obte_ctx* ctx, double* out) {
  if (!ctx || !out) return OBTE_EINVAL;
  if (!ctx->solved) return ctx->fail(OBTE_ESTATE, "solve first");
  if (ctx->shard_n > 1) return ctx->fail(OBTE_ESTATE, "gradient of a sharded solve is not available");
  CK(cudaSetDevice(ctx->device));
  unsigned char* base = nullptr;
  CK(noalloc_scratch(ctx->device, &base));
  const int O = ctx->O;
  // (paired when the material was set: same bin, MFP and weight, opposite direction)
  const std::vector<int>& rev = ctx->rev_o;
  for (int o = 0; o < O; ++o)
    if (rev[o] < 0) return ctx->fail(OBTE_EINVAL, "direction set is not symmetric under p -> -p");
  // scratch layout: grad | slots | work items | per batch ordinate: field + rev + weight
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t e = ctx->precision == 0 ? 8 : 4;
  const size_t n_items = ctx->items_h.size();
  const size_t fixed = up(sizeof(double) * ctx->n_cells) + up(sizeof(int) * O) +
                       up(sizeof(WorkItem) * n_items) + 2 * 256;
  const size_t per_ord = e * (size_t)ctx->n_cells + sizeof(int) + sizeof(double);
  if (fixed + 2 * per_ord > OBTE_NOALLOC_SCRATCH_BYTES)
    return ctx->fail(OBTE_EINVAL, "problem too large for the no-allocation scratch (" +
                                      std::to_string(OBTE_NOALLOC_SCRATCH_BYTES >> 20) +
                                      " MiB: gradient, ordinate slots, work list and one reversed "
                                      "ordinate pair of fields must fit)");
  const size_t pairs_cap = (OBTE_NOALLOC_SCRATCH_BYTES - fixed) / (2 * per_ord);
  // every carve starts on a 256-byte boundary; the last one need not end on
  // one, so the layout is checked against its unrounded end
  size_t off = 0, end = 0;
  auto carve = [&](size_t bytes) {
    unsigned char* p = base + off;
    end = off + bytes;
    off += up(bytes);
    return p;
  };
  double* grad_d = reinterpret_cast<double*>(carve(sizeof(double) * ctx->n_cells));
  int* slot_d = reinterpret_cast<int*>(carve(sizeof(int) * O));
  WorkItem* its_d = reinterpret_cast<WorkItem*>(carve(sizeof(WorkItem) * n_items));
  int* revl_d = reinterpret_cast<int*>(carve(sizeof(int) * 2 * pairs_cap));
  double* a_d = reinterpret_cast<double*>(carve(sizeof(double) * 2 * pairs_cap));
  void* rec = carve(e * (size_t)ctx->n_cells * 2 * pairs_cap);
  if (end > OBTE_NOALLOC_SCRATCH_BYTES) return ctx->fail(OBTE_EINVAL, "no-allocation scratch layout overflow");
  // batches of reversed ordinate pairs
  const std::vector<std::vector<int>> batches = grad_batches(ctx, pairs_cap);
  // the scratch keeps the previous call's contents: start the sum at zero
  CK(cudaMemsetAsync(grad_d, 0, sizeof(double) * ctx->n_cells, ctx->stream));
  const double jadj = -ctx->kappa_scale * ctx->h[0] * ctx->w_total;
  const double jscale = jadj / ctx->dT;
  std::vector<int> slot(O);
  int one = 1, zero = 0;
  for (auto& b : batches) {
    std::fill(slot.begin(), slot.end(), -1);
    for (size_t k2 = 0; k2 < b.size(); ++k2) slot[b[k2]] = (int)k2;
    std::vector<int> revl(b.size());
    std::vector<double> ab(b.size());
    for (size_t k2 = 0; k2 < b.size(); ++k2) {
      revl[k2] = slot[rev[b[k2]]];
      ab[k2] = ctx->aw[b[k2]];
    }
    std::vector<WorkItem> its;
    for (auto& it : ctx->items_h) {
      bool any = false;
      for (int o = it.o0; o < it.o0 + it.count; ++o)
        if (slot[o] >= 0) any = true;
      if (any) its.push_back(it);
    }
    CK(cudaMemcpyAsync(its_d, its.data(), sizeof(WorkItem) * its.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(slot_d, slot.data(), sizeof(int) * O, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(revl_d, revl.data(), sizeof(int) * b.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(a_d, ab.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice, ctx->stream));
    GeomDev g = ctx->gh;
    g.rec = rec;
    g.rec_slot = slot_d;
    CK(cudaMemcpyAsync(ctx->gd, &g, sizeof(GeomDev), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->ctrl, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    SweepLaunch L;
    L.geoms = ctx->gd;
    L.items = its_d;
    L.n_items = (int)its.size();
    L.flags = SWEEP_RECORD;
    L.item_counter = nullptr;
    if (ctx->warp) {
      CK(launch_ctx_warp(ctx, L));
    } else if (ctx->k3d) {
      CK(launch_sweep3d(L, ctx->precision, ctx->G, ctx->R, ctx->has_s, ctx->threads,
                        sweep3d_smem_bytes(ctx->precision, ctx->G, ctx->R, ctx->threads), ctx->stream));
    } else {
      const size_t smem = sweep_smem_bytes(ctx->precision, ctx->dim, ctx->G, ctx->R, ctx->threads);
      CK(launch_sweep(L, ctx->precision, ctx->dim, ctx->G, ctx->R, ctx->has_s, ctx->threads,
                      L.n_items, smem, ctx->stream));
    }
    CK(launch_grad_contract2(ctx->code_d, ctx->TL, ctx->n_cells, rec, (int)b.size(), revl_d, a_d,
                             jscale, grad_d, ctx->precision, ctx->gh.psi, ctx->stream));
    CK(cudaMemsetAsync(ctx->TL_acc, 0, sizeof(double) * ctx->n_cells, ctx->stream));
    if (ctx->tlq) CK(cudaMemsetAsync(ctx->tlq, 0, sizeof(double) * (ctx->dim == 3 ? 8 : 4) * (size_t)ctx->n_cells, ctx->stream));
    CK(cudaMemsetAsync(ctx->wall_acc, 0, sizeof(double) * 6 * (size_t)ctx->n_cells, ctx->stream));
    CK(cudaMemsetAsync(ctx->scal, 0, sizeof(double), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // host vectors above are copy sources
  }
  CK(cudaMemcpyAsync(ctx->gd, &ctx->gh, sizeof(GeomDev), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->ctrl, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<double> gk(ctx->n_cells);
  CK(cudaMemcpyAsync(gk.data(), grad_d, sizeof(double) * ctx->n_cells, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  to_user(ctx, [&](int c, long ui) { out[ui] = (ctx->code_h[c] & CODE_SOLID) ? gk[c] : 0.0; });
  return OBTE_OK;
}

"""ctypes binding to libobte (include/obte.h): argument marshalling only.

Every step of the solver runs in the CUDA library; this module converts numpy
arrays to host pointers, hands the library PyTorch's caching allocator and
current CUDA stream, and turns status codes into exceptions.  It fails loudly
when the library has not been built or no CUDA device is present: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libobte.so")

OBTE_OK, OBTE_EINVAL, OBTE_ESTATE, OBTE_ECUDA, OBTE_ENOMEM = 0, -1, -2, -3, -4
OBTE_NOT_CONVERGED, OBTE_ENONFINITE, OBTE_ETIMEOUT = -5, -6, -7
OBTE_FP64, OBTE_MIXED = 0, 1
MAX_HISTORY = 4096

_STATUS = {0: "OK", -1: "EINVAL", -2: "ESTATE", -3: "ECUDA", -4: "ENOMEM",
           -5: "NOT_CONVERGED", -6: "ENONFINITE", -7: "ETIMEOUT"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class DeviceCfg(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p),
                ("cuda_stream", C.c_void_p), ("device", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("tol_TL", C.c_double),
                ("max_iter", C.c_int), ("min_iter", C.c_int), ("check_every", C.c_int),
                ("fourier_max_iter", C.c_int), ("fourier_tol", C.c_double),
                ("group_size", C.c_int), ("rows_per_thread", C.c_int), ("use_graph", C.c_int),
                ("profile", C.c_int), ("kernel", C.c_int), ("accel", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("fourier_iterations", C.c_int), ("converged", C.c_int),
                ("kappa_eff", C.c_double), ("delta_TL", C.c_double),
                ("time_fourier_ms", C.c_double), ("time_iter_ms", C.c_double),
                ("time_total_ms", C.c_double), ("updates_per_s", C.c_double),
                ("group_size", C.c_int), ("rows_per_thread", C.c_int),
                ("threads_per_block", C.c_int), ("n_groups", C.c_int), ("kernel", C.c_int),
                ("n_sweeps", C.c_int), ("time_sweep_ms", C.c_double), ("time_finalize_ms", C.c_double),
                ("n_history", C.c_int),
                ("kappa_history", C.c_double * MAX_HISTORY)]

    def to_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "kappa_history"}
        d["kappa_history"] = list(self.kappa_history[:self.n_history])
        return d


# (name, restype, argtypes) of every entry point declared in include/obte.h
SIGNATURES = [
    ("obte_default_opts", None, [C.POINTER(SolveOpts)]),
    ("obte_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(DeviceCfg)]),
    ("obte_create_mesh", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                   C.c_double, C.c_double, C.c_void_p, C.POINTER(C.c_int),
                                   C.c_int, C.c_double]),
    ("obte_set_material", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_int]),
    ("obte_set_material_ordinates", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_int]),
    ("obte_set_scattering_scale", C.c_int, [C.c_void_p, C.c_void_p]),
    ("obte_solve", C.c_int, [C.c_void_p, C.POINTER(SolveOpts), C.POINTER(SolveStats)]),
    ("obte_solve_batch", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(SolveOpts),
                                   C.POINTER(SolveStats)]),
    ("obte_get_T_L", C.c_int, [C.c_void_p, C.c_void_p]),
    ("obte_get_flux", C.c_int, [C.c_void_p, C.c_void_p]),
    ("obte_get_kappa_eff", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("obte_get_section_flux", C.c_int, [C.c_void_p, C.c_void_p]),
    ("obte_kappa_grad_s", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("obte_get_kappa_bins", C.c_int, [C.c_void_p, C.c_void_p]),
    ("obte_kappa_grad_s_noalloc", C.c_int, [C.c_void_p, C.c_void_p]),
    ("obte_solve_fourier", C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_double),
                                     C.c_void_p, C.POINTER(C.c_int)]),
    ("obte_measure_fma_rate", C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
    ("obte_set_shard", C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    ("obte_shard_partials_count", C.c_size_t, [C.c_void_p]),
    ("obte_shard_begin", C.c_int, [C.c_void_p, C.POINTER(SolveOpts)]),
    ("obte_shard_sweep", C.c_int, [C.c_void_p, C.c_void_p]),
    ("obte_shard_finalize", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    ("obte_last_error", C.c_char_p, [C.c_void_p]),
    ("obte_destroy", None, [C.c_void_p]),
]

_lib = None


def load_library(path: Optional[str] = None):
    """Load libobte.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libobte.so not built ({p}); run python -m paper_2106_02764_gb300.build")
    lib = C.CDLL(p)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


class ObteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class _TorchMemory:
    """PyTorch caching allocator and current stream, handed to the library."""

    def __init__(self, device: int, stream=None):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, _user):
        try:
            return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
        except Exception:
            return None

    def _do_free(self, ptr, _user):
        if ptr:
            self.torch.cuda.caching_allocator_delete(ptr)

    def cfg(self):
        return DeviceCfg(self._alloc, self._free, None, C.c_void_p(self.stream.cuda_stream), self.device)


class Solver:
    """One geometry + material on one CUDA device (a libobte context)."""

    def __init__(self, device: int = 0, stream=None, torch_memory: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the solver has no CPU path")
        self.lib = load_library()
        self.mem = _TorchMemory(device, stream) if torch_memory else None
        cfg = self.mem.cfg() if self.mem else DeviceCfg(ALLOC_FN(0), FREE_FN(0), None, None, device)
        self.ctx = C.c_void_p()
        rc = self.lib.obte_create(C.byref(self.ctx), C.byref(cfg))
        self._check(rc)
        self.shape = None
        self.dim = None
        self.n_mfp = None
        self.stats = None

    # -- helpers
    def _check(self, rc):
        if rc != OBTE_OK:
            msg = self.lib.obte_last_error(self.ctx).decode() if self.ctx else ""
            raise ObteError(rc, msg)
        return rc

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            self.lib.obte_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inputs
    def create_mesh(self, mask, lengths, periodic=(1, 1, 1), grad_axis=0, delta_T=1.0, dim=None):
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        if m.ndim == 2:
            m = m[None]
        nz, ny, nx = m.shape
        dim = dim or (2 if nz == 1 else 3)
        per = (C.c_int * 3)(*[int(v) for v in periodic])
        lz = lengths[2] if len(lengths) > 2 else 0.0
        self._check(self.lib.obte_create_mesh(self.ctx, dim, nx, ny, nz, float(lengths[0]),
                                              float(lengths[1]), float(lz), _ptr(m), per,
                                              int(grad_axis), float(delta_T)))
        self.shape = (nz, ny, nx)
        self.dim = dim
        return self

    def set_material(self, kappa_m, lambda_m, dirs, weights, angular_dim):
        k, l = _f64(kappa_m), _f64(lambda_m)
        d, w = _f64(dirs).reshape(-1, 3), _f64(weights)
        self._check(self.lib.obte_set_material(self.ctx, len(k), _ptr(k), _ptr(l), len(w), _ptr(d),
                                               _ptr(w), int(angular_dim)))
        self.n_mfp = len(k)
        return self

    def set_material_ordinates(self, lam, dirs, weight, bins=None, n_bins=None):
        """General aMFP material: per-ordinate MFP, direction and weight
        (C/tau of the modes it stands for), optional MFP bin per ordinate."""
        l, w = _f64(lam), _f64(weight)
        d = _f64(dirs).reshape(-1, 3)
        if bins is None:
            bp, nb = None, 1
        else:
            b = np.ascontiguousarray(np.asarray(bins, dtype=np.int32))
            nb = int(n_bins if n_bins is not None else b.max() + 1)
            bp = b.ctypes.data_as(C.c_void_p)
        self._check(self.lib.obte_set_material_ordinates(self.ctx, len(l), _ptr(l), _ptr(d), _ptr(w),
                                                         bp, nb))
        self.n_mfp = nb
        return self

    def set_scattering_scale(self, s):
        if s is None:
            self._check(self.lib.obte_set_scattering_scale(self.ctx, None))
        else:
            a = _f64(s).reshape(self.shape)
            self._check(self.lib.obte_set_scattering_scale(self.ctx, _ptr(a)))
        return self

    @classmethod
    def from_workload(cls, wl, device=0, stream=None):
        s = cls(device, stream)
        s.create_mesh(wl.mask, wl.lengths, wl.periodic, wl.grad_axis, wl.delta_T, wl.dim)
        if getattr(wl, "ords", None) is not None:
            o = wl.ords
            s.set_material_ordinates(o["lambda"], o["dirs"], o["weight"], o["bin"])
        else:
            s.set_material(wl.kappa_m, wl.lambda_m, wl.quad.dirs, wl.quad.weights, wl.quad.angular_dim)
        if wl.s is not None:
            s.set_scattering_scale(wl.s)
        return s

    # -- solve
    def options(self, precision="fp64", tol=1e-6, tol_TL=0.0, max_iter=2000, min_iter=2,
                check_every=8, fourier_max_iter=0, fourier_tol=0.0, group_size=0,
                rows_per_thread=0, use_graph=True, profile=False, kernel=0, accel=0):
        o = SolveOpts()
        self.lib.obte_default_opts(C.byref(o))
        o.precision = OBTE_MIXED if precision in ("mixed", OBTE_MIXED) else OBTE_FP64
        o.tol, o.tol_TL, o.max_iter, o.min_iter = float(tol), float(tol_TL), int(max_iter), int(min_iter)
        o.check_every, o.fourier_max_iter, o.fourier_tol = int(check_every), int(fourier_max_iter), float(fourier_tol)
        o.group_size, o.rows_per_thread, o.use_graph = int(group_size), int(rows_per_thread), int(bool(use_graph))
        o.profile = int(bool(profile))
        o.kernel = {"auto": 0, "block": 1, "warp": 2, "block3d": 3}.get(kernel, kernel)
        o.accel = int(accel)
        return o

    def solve(self, allow_not_converged=False, **kw):
        o = self.options(**kw)
        st = SolveStats()
        rc = self.lib.obte_solve(self.ctx, C.byref(o), C.byref(st))
        self.stats = st.to_dict()
        if rc == OBTE_NOT_CONVERGED and allow_not_converged:
            return self.stats
        self._check(rc)
        return self.stats

    # -- outputs
    @property
    def kappa_eff(self) -> float:
        v = C.c_double()
        self._check(self.lib.obte_get_kappa_eff(self.ctx, C.byref(v)))
        return v.value

    def T_L(self):
        out = np.empty(self.shape, dtype=np.float64)
        self._check(self.lib.obte_get_T_L(self.ctx, _ptr(out)))
        return out

    def flux(self):
        out = np.empty(self.shape + (self.dim,), dtype=np.float64)
        self._check(self.lib.obte_get_flux(self.ctx, _ptr(out)))
        return out

    def section_flux(self, n_sections):
        out = np.empty(n_sections, dtype=np.float64)
        self._check(self.lib.obte_get_section_flux(self.ctx, _ptr(out)))
        return out

    def kappa_bins(self):
        out = np.empty(self.n_mfp, dtype=np.float64)
        self._check(self.lib.obte_get_kappa_bins(self.ctx, _ptr(out)))
        return out

    def kappa_grad_s(self, max_field_bytes=0):
        out = np.empty(self.shape, dtype=np.float64)
        self._check(self.lib.obte_kappa_grad_s(self.ctx, _ptr(out), C.c_size_t(int(max_field_bytes))))
        return out

    def solve_fourier(self, tol=0.0, max_iter=0, allow_not_converged=False):
        """Fourier model alone (App. B): kappa_fourier in W/m/K, the temperature
        (solid-cell mean 0, NaN in pores) and the CG iteration count."""
        k, it = C.c_double(), C.c_int()
        T = np.empty(self.shape, dtype=np.float64)
        rc = self.lib.obte_solve_fourier(self.ctx, float(tol), int(max_iter), C.byref(k), _ptr(T),
                                         C.byref(it))
        if not (rc == OBTE_NOT_CONVERGED and allow_not_converged):
            self._check(rc)
        return {"kappa": k.value, "T": T, "iterations": it.value, "converged": rc == OBTE_OK}


def _set_shard(self, rank, n_ranks):
    """Sweep only this rank's share of the ordinate groups (obte_set_shard)."""
    self._check(self.lib.obte_set_shard(self.ctx, int(rank), int(n_ranks)))
    return self


def _shard_partials_count(self):
    return int(self.lib.obte_shard_partials_count(self.ctx))


def _shard_begin(self, **kw):
    """State and Fourier first guess of a sharded solve (obte_shard_begin)."""
    kw.setdefault("group_size", 0)
    kw.setdefault("accel", 0)
    o = self.options(**kw)
    self._check(self.lib.obte_shard_begin(self.ctx, C.byref(o)))
    return self


def _shard_sweep(self, partials):
    """One sweep of this rank's ordinates; its FP64 moment partials go to
    ``partials``, a CUDA float64 tensor of shard_partials_count() elements on
    the solver's device (enqueued on the solver's stream)."""
    self._check(self.lib.obte_shard_sweep(self.ctx, C.c_void_p(partials.data_ptr())))


def _shard_finalize(self, partials):
    """Finalise the iteration from the partials summed over the ranks;
    returns the done code (0 running, 1 converged, 2 iteration cap)."""
    done = C.c_int(0)
    self._check(self.lib.obte_shard_finalize(self.ctx, C.c_void_p(partials.data_ptr()), C.byref(done)))
    return done.value


Solver.set_shard = _set_shard
Solver.shard_partials_count = _shard_partials_count
Solver.shard_begin = _shard_begin
Solver.shard_sweep = _shard_sweep
Solver.shard_finalize = _shard_finalize


def _grad_noalloc(self):
    """d kappa_eff / d s through obte_kappa_grad_s_noalloc (no device
    allocation: the library's fixed scratch array holds the work buffers)."""
    out = np.empty(self.shape, dtype=np.float64)
    self._check(self.lib.obte_kappa_grad_s_noalloc(self.ctx, _ptr(out)))
    return out


Solver.kappa_grad_s_noalloc = _grad_noalloc


def solve_batch(solvers, allow_not_converged=False, **kw):
    """Iterate several geometries together (one launch per iteration)."""
    lib = load_library()
    arr = (C.c_void_p * len(solvers))(*[s.ctx.value for s in solvers])
    o = solvers[0].options(**kw)
    stats = (SolveStats * len(solvers))()
    rc = lib.obte_solve_batch(arr, len(solvers), C.byref(o), stats)
    for s, st in zip(solvers, stats):
        s.stats = st.to_dict()
    if rc != OBTE_OK and not (rc == OBTE_NOT_CONVERGED and allow_not_converged):
        raise ObteError(rc, lib.obte_last_error(solvers[0].ctx).decode())
    return [s.stats for s in solvers]


def measure_fma_rate(precision="mixed", device=0) -> float:
    """Measured FMA throughput of a device in flop/s (FP32 for "mixed", FP64
    for "fp64"): the ALU roof of the transport sweep."""
    lib = load_library()
    out = C.c_double()
    p = OBTE_MIXED if precision in ("mixed", OBTE_MIXED) else OBTE_FP64
    rc = lib.obte_measure_fma_rate(p, int(device), C.byref(out))
    if rc != OBTE_OK:
        raise ObteError(rc, "FMA rate measurement failed")
    return out.value

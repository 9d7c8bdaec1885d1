"""Seeded synthetic inputs for the aMFP phonon-BTE solver.

This module builds the *inputs* a user hands to the solver: voxel solid masks
(pores removed), mean-free-path bins with their bulk conductivity weights, an
angular quadrature (unit directions and weights) and, for the sensitivity
workload, a per-cell scattering-scale field.  It holds none of the solver's
arithmetic (no transport coefficients, no moment weights, no discretisation):
both the CUDA library and the CPU oracle consume what it returns.

Readings of the paper used here (OpenBTE, arXiv 2106.02764):
  * MFP bins: log-spaced, endpoints included; kappa_m follow a log-normal in
    ln(Lambda) and sum to kappa_bulk (the paper reads them from ab-initio data,
    Sec. 5; the synthetic spectrum stands in for that data).
  * Directions are "located uniformly on a spherical grid" (App. A): azimuth
    midpoints phi_k = 2 pi (k + 1/2) / n_phi and Gauss-Legendre nodes in
    mu = cos(theta).  The in-plane projected model (Sec. 5, rta2DSym) maps a
    3D direction to sin(theta) (cos phi, sin phi, 0); theta and pi - theta give
    the same projection and are folded into one node with twice the weight.
  * Pores (Sec. 6, lattice model) are voxelised: a cell is removed iff its
    centre lies strictly inside a pore, using the periodic minimum image.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SEED_BASE = 2106_02764


def seed_for(config: int, index: int = 0) -> int:
    """Seed of geometry ``index`` of workload ``config``."""
    return SEED_BASE + config * 1000 + index


# --------------------------------------------------------------------------
# material: MFP bins and bulk conductivity weights
# --------------------------------------------------------------------------
def mfp_bins(n_bins: int, lam_min: float = 1e-9, lam_max: float = 1e-5,
             median: float = 300e-9, sigma_ln: float = 1.5,
             kappa_bulk: float = 150.0):
    """Return (kappa_m [W/m/K], lambda_m [m]) for ``n_bins`` log-spaced bins."""
    lam = np.logspace(math.log10(lam_min), math.log10(lam_max), n_bins)
    g = np.exp(-(np.log(lam) - math.log(median)) ** 2 / (2.0 * sigma_ln ** 2))
    kappa = kappa_bulk * g / g.sum()
    return kappa.astype(np.float64), lam.astype(np.float64)


# --------------------------------------------------------------------------
# angular quadratures: (dirs [S,3] unit or projected, weights [S] sum 1, d_ang)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Quadrature:
    dirs: np.ndarray      # [S, 3] float64
    weights: np.ndarray   # [S] float64, sums to 1
    angular_dim: int      # 2 for an in-plane circle, 3 for sphere-based sets


def circle_quadrature(n_phi: int) -> Quadrature:
    """In-plane directions at azimuth midpoints, equal weights (2D phonon gas)."""
    k = np.arange(n_phi, dtype=np.float64)
    phi = 2.0 * math.pi * (k + 0.5) / n_phi
    dirs = np.stack([np.cos(phi), np.sin(phi), np.zeros_like(phi)], axis=1)
    w = np.full(n_phi, 1.0 / n_phi)
    return Quadrature(dirs, w, 2)


def sphere_quadrature(n_phi: int, n_mu: int) -> Quadrature:
    """Azimuth midpoints x Gauss-Legendre polar nodes on the unit sphere."""
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    k = np.arange(n_phi, dtype=np.float64)
    phi = 2.0 * math.pi * (k + 0.5) / n_phi
    dirs, w = [], []
    for a in range(n_mu):
        st = math.sqrt(max(0.0, 1.0 - mu[a] * mu[a]))
        for b in range(n_phi):
            dirs.append((st * math.cos(phi[b]), st * math.sin(phi[b]), mu[a]))
            w.append(0.5 * wmu[a] / n_phi)
    return Quadrature(np.array(dirs), np.array(w), 3)


def projected_quadrature(n_phi: int, n_mu: int, fold: bool = True) -> Quadrature:
    """Sphere directions projected onto the x-y plane (infinite-thickness model).

    With ``fold`` the polar nodes mu and -mu (identical projections) are merged
    into one node of doubled weight; ``n_mu`` must then be even.
    """
    q = sphere_quadrature(n_phi, n_mu)
    dirs = q.dirs.copy()
    mu = dirs[:, 2].copy()
    dirs[:, 2] = 0.0
    w = q.weights.copy()
    if fold:
        if n_mu % 2:
            raise ValueError("folding needs an even number of polar nodes")
        keep = mu > 0.0
        dirs, w = dirs[keep], 2.0 * w[keep]
    return Quadrature(dirs, w, 3)


# --------------------------------------------------------------------------
# geometry: voxel masks (uint8, 1 = solid), shape (nz, ny, nx), x fastest
# --------------------------------------------------------------------------
def _cell_centres(n: int, length: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def _min_image(d: np.ndarray, length: float) -> np.ndarray:
    return d - length * np.round(d / length)


def pores_mask(nx: int, ny: int, lx: float, ly: float, pores: Sequence[dict],
               nz: int = 1) -> np.ndarray:
    """Solid mask with pores removed; each pore is a dict with keys
    ``shape`` ('circle'|'square'), ``x``, ``y`` (centre) and ``size`` (radius
    for circles, side for squares).  Pores run through the whole thickness."""
    xc = _cell_centres(nx, lx)[None, :]
    yc = _cell_centres(ny, ly)[:, None]
    solid = np.ones((ny, nx), dtype=bool)
    for p in pores:
        dx = _min_image(xc - p["x"], lx)
        dy = _min_image(yc - p["y"], ly)
        if p["shape"] == "circle":
            inside = dx * dx + dy * dy < p["size"] ** 2
        elif p["shape"] == "square":
            half = 0.5 * p["size"]
            inside = (np.abs(dx) < half) & (np.abs(dy) < half)
        else:
            raise ValueError(p["shape"])
        solid &= ~inside
    return np.repeat(solid[None, :, :], nz, axis=0).astype(np.uint8)


def circle_pore(lx: float, ly: float, porosity: float, x=None, y=None) -> dict:
    r = math.sqrt(porosity * lx * ly / math.pi)
    return {"shape": "circle", "x": 0.5 * lx if x is None else x,
            "y": 0.5 * ly if y is None else y, "size": r}


def square_pore(lx: float, ly: float, porosity: float, x=None, y=None) -> dict:
    s = math.sqrt(porosity * lx * ly)
    return {"shape": "square", "x": 0.5 * lx if x is None else x,
            "y": 0.5 * ly if y is None else y, "size": s}


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    dim: int                      # 2 or 3
    shape: tuple                  # (nx, ny, nz); nz = 1 in 2D
    lengths: tuple                # (lx, ly, lz) [m]; lz unused in 2D
    mask: np.ndarray              # uint8 [nz, ny, nx], 1 = solid
    periodic: tuple               # (px, py, pz) 1 = periodic, 0 = diffuse walls
    delta_T: float                # applied temperature jump across the x period [K]
    kappa_m: np.ndarray           # [M] W/m/K
    lambda_m: np.ndarray          # [M] m
    quad: Quadrature
    s: Optional[np.ndarray] = None  # per-cell scattering scale [nz, ny, nx]
    grad_axis: int = 0
    # general per-ordinate material (lambda [O], dirs [O,3], weight [O], bin [O]);
    # when set it replaces the bin x direction material above
    ords: Optional[dict] = None

    @property
    def n_solid(self) -> int:
        return int(self.mask.sum())

    @property
    def n_ordinates(self) -> int:
        if self.ords is not None:
            return len(self.ords["lambda"])
        return len(self.kappa_m) * len(self.quad.weights)

    @property
    def porosity(self) -> float:
        return 1.0 - self.mask.mean()

    def updates_per_iteration(self) -> int:
        return self.n_solid * self.n_ordinates


def make_2d(name, n, length, pores, n_bins, quad, delta_T=1.0, s=None):
    mask = pores_mask(n, n, length, length, pores)
    return Workload(name, 2, (n, n, 1), (length, length, 0.0), mask, (1, 1, 1),
                    delta_T, *mfp_bins(n_bins), quad, s)


def config1() -> Workload:
    """2D 32x32, L = 100 nm, centred circular pore porosity 0.2, 8 bins,
    16 in-plane directions."""
    L = 100e-9
    return make_2d("2d-32x32-circle-phi0.2-8bins-16dirs", 32, L,
                   [circle_pore(L, L, 0.2)], 8, circle_quadrature(16))


def config2(fold: bool = True) -> Workload:
    """2D 256x256, L = 200 nm, circular pore porosity 0.25, 30 bins,
    48 azimuthal x 12 polar directions projected on the plane."""
    L = 200e-9
    return make_2d("2d-256x256-circle-phi0.25-30bins-48x12proj", 256, L,
                   [circle_pore(L, L, 0.25)], 30,
                   projected_quadrature(48, 12, fold=fold))


def config3() -> Workload:
    """3D film 64x64x32, L = 100 nm, thickness 50 nm with diffuse top/bottom
    walls, through-thickness cylindrical pore porosity 0.15, 30 bins,
    24 azimuthal x 12 polar directions."""
    L, t = 100e-9, 50e-9
    mask = pores_mask(64, 64, L, L, [circle_pore(L, L, 0.15)], nz=32)
    return Workload("3d-film-64x64x32-cyl-phi0.15-30bins-24x12", 3, (64, 64, 32),
                    (L, L, t), mask, (1, 1, 0), 1.0, *mfp_bins(30),
                    sphere_quadrature(24, 12))


def config3_reduced(n_bins: int = 2, n_phi: int = 8, n_mu: int = 2) -> Workload:
    """The 64x64x32 film mesh of ``config3`` (same cylinder, walls and
    lengths) with fewer MFP bins and directions: 2 bins (1 nm and 10 um) x
    (8 azimuthal x 2 polar) sphere directions, 32 ordinates.  Same mesh,
    faces and walls as the full film; the smaller ordinate set is one whose
    per-ordinate sparse factorisations (about 1 GB each on this mesh) fit a
    host's memory, so a converged FP64 reference exists for the 3D kernels at
    the film's own mesh size."""
    wl = config3()
    kappa_m, lambda_m = mfp_bins(n_bins)
    return dataclasses.replace(
        wl, name=f"3d-film-64x64x32-cyl-phi0.15-{n_bins}bins-{n_phi}x{n_mu}",
        kappa_m=kappa_m, lambda_m=lambda_m, quad=sphere_quadrature(n_phi, n_mu))


def _random_pores(rng, n, length, n_pores, porosity, min_gap_cells=2.0,
                  max_tries=2000):
    h = length / n
    per = porosity / n_pores
    for _ in range(max_tries):
        pores = []
        ok = True
        for _k in range(n_pores):
            shape = "circle" if rng.random() < 0.5 else "square"
            size = (math.sqrt(per * length * length / math.pi) if shape == "circle"
                    else math.sqrt(per * length * length))
            reach = size if shape == "circle" else size / math.sqrt(2.0)
            placed = False
            for _t in range(200):
                x, y = rng.random() * length, rng.random() * length
                good = True
                for q in pores:
                    qr = q["size"] if q["shape"] == "circle" else q["size"] / math.sqrt(2.0)
                    dx = _min_image(np.array(x - q["x"]), length)
                    dy = _min_image(np.array(y - q["y"]), length)
                    if math.hypot(float(dx), float(dy)) < reach + qr + min_gap_cells * h:
                        good = False
                        break
                if good:
                    pores.append({"shape": shape, "x": x, "y": y, "size": size})
                    placed = True
                    break
            if not placed:
                ok = False
                break
        if ok:
            return pores
    raise RuntimeError("could not place pores")


def config4(n_geom: int = 64) -> List[Workload]:
    """64 independent 2D periodic geometries, N in {48, 64, ..., 192},
    1-4 circular or square pores at seeded positions, porosity U[0.05, 0.4],
    20 bins, 32 in-plane directions."""
    L = 100e-9
    sizes = list(range(48, 193, 16))
    out = []
    quad = circle_quadrature(32)
    for g in range(n_geom):
        rng = np.random.default_rng(seed_for(4, g))
        n = int(rng.choice(sizes))
        n_pores = int(rng.integers(1, 5))
        phi = float(rng.uniform(0.05, 0.4))
        pores = _random_pores(rng, n, L, n_pores, phi)
        out.append(make_2d(f"batch{g:02d}-{n}x{n}-{n_pores}pores", n, L, pores, 20, quad))
    return out


def scattering_field(shape, seed: int, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Per-cell scattering scale s(x) ~ U[lo, hi], shape (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(np.float64)


def config5() -> Workload:
    """2D 128x128, L = 100 nm, centred circle porosity 0.2, per-cell scattering
    scale s ~ U[0.5, 2], 20 bins, 32 in-plane directions (sensitivity case)."""
    L = 100e-9
    s = scattering_field((1, 128, 128), seed_for(5))
    return make_2d("2d-128x128-circle-phi0.2-20bins-32dirs-s", 128, L,
                   [circle_pore(L, L, 0.2)], 20, circle_quadrature(32), s=s)


def small_2d(n=8, porosity=0.2, n_bins=3, n_phi=8, length=100e-9, delta_T=1.0,
             pore="circle", s_seed=None) -> Workload:
    """Small seeded 2D case for parity tests (several sweep tiles, ragged sizes)."""
    pores = [] if porosity <= 0 else [
        (circle_pore if pore == "circle" else square_pore)(length, length, porosity)]
    s = None if s_seed is None else scattering_field((1, n, n), s_seed)
    return make_2d(f"small-2d-{n}", n, length, pores, n_bins,
                   circle_quadrature(n_phi), delta_T, s)


def small_film(n=8, nz=4, porosity=0.15, n_bins=3, n_phi=8, n_mu=4,
               length=100e-9, thickness=50e-9) -> Workload:
    """Small 3D film: periodic x, y; diffuse walls at z = 0 and z = t."""
    pores = [] if porosity <= 0 else [circle_pore(length, length, porosity)]
    mask = pores_mask(n, n, length, length, pores, nz=nz)
    return Workload(f"small-film-{n}x{n}x{nz}", 3, (n, n, nz), (length, length, thickness),
                    mask, (1, 1, 0), 1.0, *mfp_bins(n_bins),
                    sphere_quadrature(n_phi, n_mu))


def anisotropic_material(kappa_m, lambda_m, quad: Quadrature, eps_lambda: float = 0.3,
                         eps_weight: float = 0.5) -> dict:
    """Synthetic per-ordinate material: the general aMFP input (Sec. 5), where
    the Material module gives every ordinate its own vectorial MFP and weight
    from mode data; no mode data exist here, so an anisotropy is imposed on
    MFP bins (kappa_m, lambda_m) and the directions of ``quad``.  Ordinate
    (m, s), phi_s the azimuth of s:
        Lambda = lambda_m (1 + eps_lambda cos 2 phi_s)
        weight = d_ang w_s (kappa_m / lambda_m^2) (1 + eps_weight sin^2 phi_s)
    (weight: the C/tau of the ordinate's modes, scaled so that at
    eps_lambda = eps_weight = 0 the bulk conductivity is sum kappa_m).  Both
    are even under s -> -s (time reversal, as for mode data)."""
    kappa_m = np.asarray(kappa_m, np.float64)
    lam_m = np.asarray(lambda_m, np.float64)
    phi = np.arctan2(quad.dirs[:, 1], quad.dirs[:, 0])
    M, S = len(lam_m), len(quad.weights)
    lam = (lam_m[:, None] * (1.0 + eps_lambda * np.cos(2.0 * phi))[None, :]).ravel()
    weight = (quad.angular_dim * (kappa_m / lam_m ** 2)[:, None] * quad.weights[None, :]
              * (1.0 + eps_weight * np.sin(phi) ** 2)[None, :]).ravel()
    dirs = np.tile(quad.dirs, (M, 1))
    bins = np.repeat(np.arange(M), S)
    return {"lambda": lam, "dirs": dirs, "weight": weight, "bin": bins}


def anisotropic(wl: Workload, eps_lambda: float = 0.3, eps_weight: float = 0.5) -> Workload:
    """The workload ``wl`` with its material made anisotropic (see
    anisotropic_material; same bins and directions)."""
    w = dataclasses.replace(wl, name=wl.name + f"-aniso{eps_lambda:g}-{eps_weight:g}")
    w.ords = anisotropic_material(wl.kappa_m, wl.lambda_m, wl.quad, eps_lambda, eps_weight)
    return w


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}

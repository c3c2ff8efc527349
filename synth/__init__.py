"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the traversal method.  It only draws
random arrays (ray origins and directions, sample points, path endpoints,
adjoint weights, clump parameters) and states the analytic test models of
the paper's Sect. 3.1 in the form of parameter records, with their total
mass (the "total dust mass in the system" of Sect. 2.2) obtained from
closed forms or one-dimensional quadrature of the model.  The density
formulas themselves are written out separately by each consumer (the
oracle in plain C, the library in C++/CUDA).

The paper's own models (three-armed spiral, clumpy AGN torus, SPH
snapshot) are not available, so the stand-ins are:

* ``disk``   rho = rho_c exp(-R/h_R - |z|/h_z), R = sqrt(x^2 + y^2)
* ``torus``  ring torus with a hard edge, (sqrt(x^2+y^2) - R0)^2 + z^2 < r^2,
             constant rho0 inside, plus Gaussian clumps truncated at 5 sigma
* ``const``  uniform rho0 (closed-form pins)
* ``dyadic`` piecewise-constant on a 2^L x 2^L x 2^L lattice (pins where the
             grid can represent the model exactly)
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

MODEL_CONST = 0
MODEL_DISK = 1
MODEL_TORUS = 2
MODEL_DYADIC = 3

TREE_OCTREE = 0
TREE_KD = 1

PLANE_CENTRE = 0
PLANE_BARYCENTRE = 1
PLANE_EQUAL_MASS = 2
PLANE_EQUAL_DENSITY = 3

#: truncation radius of a clump in units of its sigma
CLUMP_CUT_SIGMAS = 5.0

BASE_SEED = 1311070500


def config_seed(i: int) -> int:
    """Seed of workload ``i`` (1..5)."""
    return BASE_SEED + int(i)


@dataclasses.dataclass
class Model:
    """Parameter record of a density model.

    ``params`` meaning by kind:
      const : [rho0]
      disk  : [rho_c, h_R, h_z]
      torus : [R0, r_tube, rho0]   + ``table`` = clumps [n, 5] (cx, cy, cz, sigma, A)
      dyadic: [L]                  + ``table`` = values [8^L], index ix + n*(iy + n*iz)
    ``m_tot`` is the model's total mass inside ``domain``.
    """

    kind: int
    params: np.ndarray
    table: np.ndarray
    m_tot: float
    domain_lo: np.ndarray
    domain_hi: np.ndarray
    name: str = ""

    @property
    def n_table(self) -> int:
        return 0 if self.table is None else int(self.table.shape[0])


def _box(lo, hi):
    lo = np.full(3, float(lo)) if np.isscalar(lo) else np.asarray(lo, np.float64)
    hi = np.full(3, float(hi)) if np.isscalar(hi) else np.asarray(hi, np.float64)
    return lo, hi


def make_const(rho0: float = 1.0, lo=-1.0, hi=1.0) -> Model:
    lo, hi = _box(lo, hi)
    vol = float(np.prod(hi - lo))
    return Model(MODEL_CONST, np.array([rho0], np.float64), np.zeros((0, 5)),
                 rho0 * vol, lo, hi, "const")


def _disk_radial_mass(h: float, a: float) -> float:
    """Integral of exp(-R/h) over the square [-a, a]^2 (eight octants, radial part closed form)."""
    from scipy.integrate import quad

    def inner(phi):
        x = a / math.cos(phi)
        return h * h * (1.0 - math.exp(-x / h) * (1.0 + x / h))

    val, _ = quad(inner, 0.0, math.pi / 4, epsabs=0.0, epsrel=1e-13, limit=200)
    return 8.0 * val


def make_disk(rho_c: float = 1.0, h_R: float = 0.25, h_z: float = 0.03, half: float = 1.0) -> Model:
    """Exponential disk in the cube [-half, half]^3 (total mass by closed form + 1-D quadrature)."""
    lo, hi = _box(-half, half)
    mz = 2.0 * h_z * (1.0 - math.exp(-half / h_z))
    m_tot = rho_c * _disk_radial_mass(h_R, half) * mz
    return Model(MODEL_DISK, np.array([rho_c, h_R, h_z], np.float64), np.zeros((0, 5)),
                 m_tot, lo, hi, "disk")


def clump_truncated_fraction(cut: float = CLUMP_CUT_SIGMAS) -> float:
    """Mass fraction of a 3-D Gaussian inside radius cut*sigma."""
    from scipy.special import erf
    return float(erf(cut / math.sqrt(2.0)) - math.sqrt(2.0 / math.pi) * cut * math.exp(-0.5 * cut * cut))


def make_torus(seed: int, n_clumps: int = 1000, R0: float = 0.5, r_tube: float = 0.2,
               tau_eq: float = 10.0, kappa: float = 1.0, w_min: float = 0.005, w_max: float = 0.05,
               mass_dex: float = 1.0, clump_mass_ratio: float = 1.0, half: float = 1.0) -> Model:
    """Ring torus with a hard edge plus truncated Gaussian clumps.

    rho0 is set so that the equatorial optical depth through the tube (a chord
    of length 2 r_tube) is ``tau_eq`` at opacity ``kappa``.  Clump centres are
    uniform inside the tube, widths log-uniform in [w_min, w_max], masses
    log-normal with ``mass_dex`` dex, scaled so the clumps hold
    ``clump_mass_ratio`` times the smooth mass.  Each clump is truncated at
    5 sigma and its amplitude A is chosen so the truncated clump holds its
    nominal mass exactly.
    """
    lo, hi = _box(-half, half)
    rng = np.random.default_rng(seed)
    rho0 = tau_eq / (kappa * 2.0 * r_tube)
    m_smooth = rho0 * 2.0 * math.pi ** 2 * R0 * r_tube ** 2
    # centres uniform in the tube volume (rejection sampling from the bounding box)
    cen = np.empty((0, 3))
    while cen.shape[0] < n_clumps:
        p = rng.uniform(-(R0 + r_tube), R0 + r_tube, size=(4 * n_clumps, 3))
        p[:, 2] = rng.uniform(-r_tube, r_tube, size=4 * n_clumps)
        d = np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2) - R0
        cen = np.concatenate([cen, p[d * d + p[:, 2] ** 2 < r_tube ** 2]])
    cen = cen[:n_clumps]
    sig = np.exp(rng.uniform(math.log(w_min), math.log(w_max), size=n_clumps))
    m = 10.0 ** rng.normal(0.0, mass_dex, size=n_clumps)
    if n_clumps > 0:
        m *= clump_mass_ratio * m_smooth / m.sum()
    frac = clump_truncated_fraction()
    amp = m / ((2.0 * math.pi) ** 1.5 * sig ** 3 * frac)
    table = np.column_stack([cen, sig, amp]).astype(np.float64)
    reach = R0 + r_tube + CLUMP_CUT_SIGMAS * w_max
    if reach > half or r_tube + CLUMP_CUT_SIGMAS * w_max > half:
        raise ValueError("torus and clumps must lie inside the domain")
    return Model(MODEL_TORUS, np.array([R0, r_tube, rho0], np.float64), table,
                 m_smooth + float(m.sum()), lo, hi, "torus")


def make_dyadic(seed: int, level: int = 2, lo=-1.0, hi=1.0, vmin: float = 0.1, vmax: float = 10.0) -> Model:
    """Piecewise-constant model on a 2^level lattice with log-uniform cell values."""
    lo, hi = _box(lo, hi)
    rng = np.random.default_rng(seed)
    n = 1 << level
    vals = np.exp(rng.uniform(math.log(vmin), math.log(vmax), size=n ** 3)).astype(np.float64)
    cell_vol = float(np.prod((hi - lo) / n))
    return Model(MODEL_DYADIC, np.array([float(level)], np.float64), vals.reshape(-1, 1),
                 float(vals.sum()) * cell_vol, lo, hi, "dyadic")


# --------------------------------------------------------------------------- build parameters

@dataclasses.dataclass
class BuildParams:
    """Subdivision-stopping criteria of Sect. 4 (mass, optical depth, density gradient).

    A criterion is disabled by ``use_*`` = False.  ``max_level`` is in octree
    levels; a k-d tree may go 3*max_level splits deep (one octree level equals
    three k-d levels, Sect. 2.1).  ``split_axis`` (k-d trees): 0 cycles through
    x, y, z; 1 splits on the axis of the strongest density gradient (Sect. 2.2).
    ``split_plane``: 0 cuts at the geometric centre; octrees 1 at the
    barycentre of the node's draws; k-d trees 2 at equal mass, 3 at equal
    mean density of the two halves (Sect. 2.2's location options).
    """

    kind: int = TREE_OCTREE
    delta_max: float = 1e-4
    use_delta: bool = True
    tau_max: float = 0.0
    use_tau: bool = False
    q_max: float = 1.0
    use_q: bool = False
    max_level: int = 6
    n_ran: int = 100
    kappa: float = 1.0
    seed: int = BASE_SEED
    split_axis: int = 0
    split_plane: int = 0


# --------------------------------------------------------------------------- rays and points

def uniform_points(rng: np.random.Generator, n: int, lo, hi) -> np.ndarray:
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return lo + rng.random((n, 3)) * (hi - lo)


def isotropic_dirs(rng: np.random.Generator, n: int) -> np.ndarray:
    mu = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return np.column_stack([s * np.cos(phi), s * np.sin(phi), mu])


def emission_rays(seed: int, n: int, lo=-1.0, hi=1.0):
    """Origins uniform in the box, isotropic unit directions ([n,3] f64 each)."""
    lo, hi = _box(lo, hi)
    rng = np.random.default_rng(seed)
    o = uniform_points(rng, n, lo, hi)
    d = isotropic_dirs(rng, n)
    return np.ascontiguousarray(o), np.ascontiguousarray(d)


def endpoint_paths(seed: int, n: int, lo=-1.0, hi=1.0):
    """Paths with both endpoints uniform in the box: origin a, unit direction, length |b - a|."""
    lo, hi = _box(lo, hi)
    rng = np.random.default_rng(seed)
    a = uniform_points(rng, n, lo, hi)
    b = uniform_points(rng, n, lo, hi)
    v = b - a
    L = np.sqrt((v * v).sum(axis=1))
    L = np.where(L > 0, L, 1.0)
    return np.ascontiguousarray(a), np.ascontiguousarray(v / L[:, None]), np.ascontiguousarray(L)


def interaction_depths(seed: int, n: int) -> np.ndarray:
    """Optical depths to the next interaction of photon packets, tau = -ln u with u uniform in (0, 1]
    (the draw of the Monte Carlo loop; passed to both sides as an input)."""
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random(n)  # (0, 1]
    return np.ascontiguousarray(-np.log(u))


def sample_points(seed: int, n: int, lo=-1.0, hi=1.0) -> np.ndarray:
    lo, hi = _box(lo, hi)
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(uniform_points(rng, n, lo, hi))


def adjoint_weights(seed: int, n: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.random(n).astype(np.float32)


def degenerate_rays(lo=-1.0, hi=1.0, levels: int = 3, n_random: int = 64, seed: int = 7):
    """Adversarial rays: axis-aligned, inside split planes, through edges and corners.

    Origins sit on dyadic positions of a 2^levels lattice (split planes of
    a grid refined that far), directions are axis-aligned, face-diagonal,
    body-diagonal, or contain signed zeros.
    """
    lo, hi = _box(lo, hi)
    rng = np.random.default_rng(seed)
    n = 1 << levels
    ticks = [lo + (hi - lo) * (i / n) for i in range(n + 1)]
    dirs = []
    for v in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
              (1, 1, 0), (1, -1, 0), (-1, 1, 0), (0, 1, 1), (0, -1, -1), (1, 0, 1),
              (1, 1, 1), (-1, -1, -1), (1, -1, 1), (-1, 1, -1)]:
        v = np.array(v, np.float64)
        dirs.append(v / np.linalg.norm(v))
    dirs.append(np.array([-0.0, 1.0, 0.0]))
    dirs.append(np.array([1.0, -0.0, -0.0]))
    origins, ds = [], []
    for _ in range(n_random):
        i = rng.integers(0, n + 1, size=3)
        o = np.array([ticks[int(i[0])][0], ticks[int(i[1])][1], ticks[int(i[2])][2]])
        # keep some coordinates generic so that rays run inside a single split plane
        mask = rng.random(3) < 0.3
        o = np.where(mask, lo + rng.random(3) * (hi - lo), o)
        d = dirs[int(rng.integers(0, len(dirs)))]
        origins.append(o)
        ds.append(d)
    return np.ascontiguousarray(np.array(origins)), np.ascontiguousarray(np.array(ds))


# --------------------------------------------------------------------------- workload presets

def workload_disk_small():
    """Plain FP64 workload: disk, octree, mass threshold 1e-4, max level 6, 1e4 rays."""
    seed = config_seed(1)
    model = make_disk()
    bp = BuildParams(kind=TREE_OCTREE, delta_max=1e-4, max_level=6, seed=seed)
    return model, bp, 10_000, seed


def workload_disk_1e6(kind: int, delta_max: Optional[float] = None):
    """Disk at ~1e6 leaves: octree (mass 1e-6, max level 12) or k-d tree."""
    seed = config_seed(2)
    model = make_disk()
    dm = 1e-6 if delta_max is None else delta_max
    bp = BuildParams(kind=kind, delta_max=dm, max_level=12, seed=seed)
    return model, bp, 1_000_000, seed


def workload_torus_1e7(max_level: int = 10, delta_max: float = 7e-7):
    """Ring torus + 1000 clumps, k-d tree under the mass, optical-depth (tau 0.5) and dispersion (q 0.9,
    density ratio 10) criteria.  Max level 10 with the mass threshold 7e-7 gives ~9.8e6 leaves; the
    nominal mass threshold 1e-7 gives 8.4e6 leaves at max level 9 and 1.6e7 at max level 10."""
    seed = config_seed(3)
    model = make_torus(seed)
    bp = BuildParams(kind=TREE_KD, delta_max=delta_max, use_tau=True, tau_max=0.5,
                     use_q=True, q_max=0.9, max_level=max_level, seed=seed)
    return model, bp, 10_000_000, seed


def batch_specs(n_grids: int = 64, seed: Optional[int] = None, rays_lo: float = 1e5, rays_hi: float = 1e7,
                leaves_lo: float = 1e4, leaves_hi: float = 1e6):
    """Specs of the uneven multi-grid batch: kind, model, target leaves, ray count per grid."""
    seed = config_seed(4) if seed is None else seed
    rng = np.random.default_rng(seed)
    specs = []
    for g in range(n_grids):
        kind = int(rng.integers(0, 2))
        mk = int(rng.integers(0, 3))  # 0 disk, 1 ring, 2 clumps
        target = float(np.exp(rng.uniform(math.log(leaves_lo), math.log(leaves_hi))))
        rays = int(np.exp(rng.uniform(math.log(rays_lo), math.log(rays_hi))))
        sub = int(rng.integers(0, 2 ** 31))
        if mk == 0:
            model = make_disk(h_R=float(rng.uniform(0.15, 0.35)), h_z=float(rng.uniform(0.02, 0.08)))
        elif mk == 1:
            model = make_torus(sub, n_clumps=0, R0=float(rng.uniform(0.4, 0.6)), r_tube=0.15,
                               tau_eq=float(rng.uniform(1.0, 10.0)))
        else:
            model = make_torus(sub, n_clumps=int(rng.integers(50, 400)), R0=0.5, r_tube=0.2,
                               tau_eq=float(rng.uniform(1.0, 10.0)))
        specs.append(dict(kind=kind, model=model, target_leaves=target, n_rays=rays, seed=sub))
    return specs

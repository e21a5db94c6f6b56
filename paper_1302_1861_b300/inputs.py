"""Seeded synthetic workloads for the phase-space-let (PSL) dose path.

This module is the one place where inputs are made.  Both the CUDA path and
the CPU oracle take their inputs from here; it holds none of the method's
arithmetic (no binning, selection, weighting, transport or tally).  Every
array is drawn from numpy's PCG64 generator seeded with
``1302186100 + config index``.

The paper measures on a BEAMnrc phase space of a Varian Clinac 21EX 6 MV
beam, a water phantom and a clinical IMRT patient (Sec. 2.6).  None of these
exist here; the generators below are stand-ins with the stated shapes:

* phase space (Sec. 2.3.2): SoA float32 ``x, y, u, v, e, wt`` plus int8
  ``q`` (0 photon, -1 electron, +1 positron) at the phase-space plane
  ``z_psl`` (a virtual plane at the isocentre distance).  Positions are
  uniform over a square plus Gaussian penumbra; directions come from a point
  source at z = 0; photon energies follow a piecewise-linear 6 MV-like
  spectrum; 3 % of records are electrons with uniform energy.
* phantoms: water boxes with slabs, or CT-like boxes of ellipsoids with
  density classes (air, lung, soft tissue, bone).
* beams: jaw settings, gantry/collimator/couch angles, MU and fluence maps
  (Sec. 2.4) drawn as smooth random fields in [0, 1].
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 1302186100

# photon spectrum nodes (MeV, relative pdf); linear between nodes
SPECTRUM_NODES = ((0.1, 0.2), (0.5, 1.0), (2.0, 0.35), (6.0, 0.0))
E_MAX = 6.0          # MeV, top of the spectrum (top energy-bin edge)
E_LO = 0.01          # MeV, bottom of the log energy bins (photon cut-off)
SAD = 100.0          # source-axis distance, cm (Sec. 2.6)
Z_PSL = 100.0        # virtual phase-space plane, cm from the source
Z_JAW_Y = 28.0       # upper (Y) jaw plane, cm from the source
Z_JAW_X = 36.7       # lower (X) jaw plane, cm from the source

MAT_WATER = 0        # water-like media (air, lung, soft tissue, water)
MAT_BONE = 1

RHO_AIR, RHO_LUNG, RHO_TISSUE, RHO_BONE = 0.001, 0.26, 1.04, 1.6


@dataclasses.dataclass
class Records:
    x: np.ndarray
    y: np.ndarray
    u: np.ndarray
    v: np.ndarray
    e: np.ndarray
    wt: np.ndarray
    q: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def arrays(self):
        return (self.x, self.y, self.u, self.v, self.e, self.wt, self.q)


@dataclasses.dataclass
class Binning:
    x_edges: np.ndarray      # float32, nx+1
    y_edges: np.ndarray      # float32, ny+1
    e_edges: np.ndarray      # float32, n_ebins+1
    log_ebins: bool
    apr_copies: int = 1      # azimuthal redistribution: copies per record (Sec. 2.3.1)
    apr_seed: int = 0        # Philox key of the redistribution angles

    @property
    def nx(self):
        return len(self.x_edges) - 1

    @property
    def ny(self):
        return len(self.y_edges) - 1

    @property
    def n_ebins(self):
        return len(self.e_edges) - 1

    @property
    def n_bins(self):
        return 2 * self.n_ebins * self.nx * self.ny


@dataclasses.dataclass
class Beam:
    x1: float
    x2: float
    y1: float
    y2: float
    gantry: float = 0.0
    collimator: float = 0.0
    couch: float = 0.0
    mu: float = 1.0
    roi_margin: float = 1.0
    iso: tuple = (0.0, 0.0, SAD)
    z_jaw_x: float = Z_JAW_X
    z_jaw_y: float = Z_JAW_Y
    fluence: Optional[np.ndarray] = None     # float32 [fny, fnx]
    fx0: float = -20.0
    fy0: float = -20.0
    fdx: float = 1.0
    fdy: float = 1.0


@dataclasses.dataclass
class Phantom:
    mat: np.ndarray          # uint8 [nz, ny, nx]
    rho: np.ndarray          # float32 [nz, ny, nx]
    voxel: tuple             # (vx, vy, vz) cm
    origin: tuple            # patient coordinates of the (0,0,0) voxel corner

    @property
    def shape(self):
        return self.mat.shape


@dataclasses.dataclass
class Workload:
    name: str
    index: int
    records: Records
    binning: Binning
    beams: List[Beam]
    phantom: Phantom
    n_histories: int
    n_batches: int = 10
    z_psl: float = Z_PSL
    sad: float = SAD

    @property
    def seed(self) -> int:
        return SEED_BASE + self.index


def _rng(index: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + index, stream]))


def sample_spectrum(rng: np.random.Generator, n: int) -> np.ndarray:
    """Inverse-CDF draw from the piecewise-linear photon spectrum."""
    xs = np.array([p[0] for p in SPECTRUM_NODES])
    ps = np.array([p[1] for p in SPECTRUM_NODES])
    seg_mass = 0.5 * (ps[:-1] + ps[1:]) * np.diff(xs)
    cdf = np.concatenate([[0.0], np.cumsum(seg_mass)]) / seg_mass.sum()
    r = rng.random(n)
    k = np.clip(np.searchsorted(cdf, r, side="right") - 1, 0, len(seg_mass) - 1)
    x0, x1, p0, p1 = xs[k], xs[k + 1], ps[k], ps[k + 1]
    # mass inside segment to reach: solve p0*t + 0.5*slope*t^2 = m
    m = (r - cdf[k]) * seg_mass.sum()
    slope = (p1 - p0) / (x1 - x0)
    disc = np.maximum(p0 * p0 + 2.0 * slope * m, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(np.abs(slope) > 1e-12, (-p0 + np.sqrt(disc)) / slope, m / p0)
    return np.clip(x0 + t, x0, x1)


def make_records(index: int, n: int, half: float, sigma: float = 0.3,
                 e_frac: float = 0.03, z_psl: float = Z_PSL) -> Records:
    """Phase-space records: uniform square of half-width ``half`` plus
    Gaussian penumbra, point-source directions, 6 MV-like spectrum."""
    rng = _rng(index, 1)
    x = rng.uniform(-half, half, n) + rng.normal(0.0, sigma, n)
    y = rng.uniform(-half, half, n) + rng.normal(0.0, sigma, n)
    norm = np.sqrt(x * x + y * y + z_psl * z_psl)
    u = x / norm
    v = y / norm
    is_e = rng.random(n) < e_frac
    e = sample_spectrum(rng, n)
    e_el = rng.uniform(0.2, 5.0, n)
    e = np.where(is_e, e_el, e)
    q = np.where(is_e, -1, 0).astype(np.int8)
    f32 = np.float32
    return Records(x.astype(f32), y.astype(f32), u.astype(f32), v.astype(f32),
                   e.astype(f32), np.ones(n, f32), q)


def make_binning(half_extent: float, dxy: float, n_ebins: int, log_ebins: bool) -> Binning:
    nxy = int(round(2 * half_extent / dxy))
    xe = (-half_extent + dxy * np.arange(nxy + 1, dtype=np.float64)).astype(np.float32)
    if log_ebins:
        k = np.arange(n_ebins + 1, dtype=np.float64)
        ee = E_LO * (E_MAX / E_LO) ** (k / n_ebins)
    else:
        ee = E_MAX * np.arange(n_ebins + 1, dtype=np.float64) / n_ebins
    return Binning(xe, xe.copy(), ee.astype(np.float32), log_ebins)


def water_phantom(n: int, vox: float, ssd: float = 90.0) -> Phantom:
    mat = np.full((n, n, n), MAT_WATER, np.uint8)
    rho = np.ones((n, n, n), np.float32)
    half = 0.5 * n * vox
    return Phantom(mat, rho, (vox, vox, vox), (-half, -half, ssd))


def slab_phantom(index: int, n: int, vox: float, ssd: float = 90.0) -> Phantom:
    """Water with a 2 cm lung slab (0.25 g/cc) and a 1 cm bone slab
    (1.85 g/cc) at seeded, non-overlapping depths within [2, 14] cm."""
    ph = water_phantom(n, vox, ssd)
    rng = _rng(index, 2)
    while True:
        d_lung = rng.uniform(2.0, 12.0)
        d_bone = rng.uniform(2.0, 13.0)
        if d_lung + 2.0 <= d_bone or d_bone + 1.0 <= d_lung:
            break
    for d0, th, rho, mat in ((d_lung, 2.0, 0.25, MAT_WATER), (d_bone, 1.0, 1.85, MAT_BONE)):
        k0 = int(round(d0 / vox))
        k1 = int(round((d0 + th) / vox))
        ph.rho[k0:k1] = rho
        ph.mat[k0:k1] = mat
    return ph


def ct_phantom(index: int, shape: tuple, vox: float, center_z: float = SAD) -> Phantom:
    """CT-like phantom: air box holding a soft-tissue body ellipsoid with two
    lung ellipsoids and two bone ellipsoids at seeded offsets."""
    nz, ny, nx = shape
    rng = _rng(index, 3)
    L = np.array([nx, ny, nz], np.float64) * vox
    origin = (-0.5 * L[0], -0.5 * L[1], center_z - 0.5 * L[2])
    xs = (np.arange(nx) + 0.5) * vox + origin[0]
    ys = (np.arange(ny) + 0.5) * vox + origin[1]
    zs = (np.arange(nz) + 0.5) * vox + origin[2]
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    rho = np.full(shape, RHO_AIR, np.float32)
    mat = np.full(shape, MAT_WATER, np.uint8)

    def ell(c, a):
        return ((X - c[0]) / a[0]) ** 2 + ((Y - c[1]) / a[1]) ** 2 + ((Z - c[2]) / a[2]) ** 2 <= 1.0

    j = lambda s: rng.uniform(-s, s)
    body = ell((j(0.5), j(0.5), center_z + j(0.5)),
               (0.42 * L[0], 0.45 * L[1], 0.36 * L[2]))
    rho[body] = RHO_TISSUE
    for side in (-1.0, 1.0):
        lung = ell((side * 0.17 * L[0] + j(0.5), j(1.0), center_z + j(0.5)),
                   (0.11 * L[0], 0.25 * L[1], 0.14 * L[2])) & body
        rho[lung] = RHO_LUNG
    spine = ell((j(0.3), j(0.5), center_z + 0.24 * L[2] + j(0.3)),
                (0.05 * L[0], 0.40 * L[1], 0.05 * L[2])) & body
    sternum = ell((j(0.3), j(0.5), center_z - 0.28 * L[2] + j(0.3)),
                  (0.04 * L[0], 0.20 * L[1], 0.03 * L[2])) & body
    for b in (spine, sternum):
        rho[b] = RHO_BONE
        mat[b] = MAT_BONE
    return Phantom(mat, rho, (vox, vox, vox), origin)


def smooth_field(rng: np.random.Generator, n: int = 40, bumps: int = 12) -> np.ndarray:
    """Sum of Gaussian bumps on an n x n grid, rescaled to [0, 1]."""
    g = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(g, g, indexing="xy")
    f = np.zeros((n, n))
    for _ in range(bumps):
        cx, cy = rng.random(2)
        s = rng.uniform(0.08, 0.3)
        a = rng.uniform(0.3, 1.0)
        f += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * s * s))
    f = (f - f.min()) / (f.max() - f.min())
    return f.astype(np.float32)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def config1(n_records: int = 100_000, n_histories: int = 100_000) -> Workload:
    """4x4 cm2 field, 1e5 records, 32^3 x 0.5 cm water, 1e5 histories.
    Paper-style linear energy bins (10) over [0, 6] MeV, 1 cm bins over +-3 cm."""
    rec = make_records(1, n_records, half=3.0)
    binning = make_binning(3.0, 1.0, 10, log_ebins=False)
    beams = [Beam(-2.0, 2.0, -2.0, 2.0, roi_margin=1.0)]
    return Workload("psl-4x4-water32", 1, rec, binning, beams,
                    water_phantom(32, 0.5), n_histories)


def config2(n_records: int = 10_000_000, n_histories: int = 100_000_000) -> Workload:
    """10x10 cm2 field, 1e7 records, 2 x 32 log-E x (12 x 12) 1 cm bins,
    64^3 x 0.25 cm water with lung and bone slabs, 1e8 histories."""
    rec = make_records(2, n_records, half=6.0)
    binning = make_binning(6.0, 1.0, 32, log_ebins=True)
    beams = [Beam(-5.0, 5.0, -5.0, 5.0, roi_margin=1.0)]
    return Workload("psl-10x10-slab64", 2, rec, binning, beams,
                    slab_phantom(2, 64, 0.25), n_histories)


def config3(n_records: int = 40_000_000, n_histories: int = 1_000_000_000, records=None) -> Workload:
    """30x30 cm2 jaws over a 40x40 cm patient-independent phase space with a
    40x40 fluence map; 128^3 x 0.25 cm CT-like phantom; 1e9 histories.
    `records` may pass the phase space already made (the same seeded one)."""
    rec = make_records(3, n_records, half=20.0) if records is None else records
    binning = make_binning(20.0, 1.0, 32, log_ebins=True)
    flu = smooth_field(_rng(3, 4))
    beams = [Beam(-15.0, 15.0, -15.0, 15.0, roi_margin=1.0, fluence=flu,
                  fx0=-20.0, fy0=-20.0, fdx=1.0, fdy=1.0)]
    return Workload("psl-30x30-ct128", 3, rec, binning, beams,
                    ct_phantom(3, (128, 128, 128), 0.25), n_histories)


def config4(n_records: int = 40_000_000, n_histories: int = 500_000_000, records=None) -> Workload:
    """Batched IMRT plan on the config-3 phase space: 7 gantry angles x
    10-60 square segments (2-20 cm), per-segment 40x40 fluence, MU in
    [0.5, 2]; 128x128x100 x 0.25 cm CT-like phantom; 5e8 histories.
    `records` may pass the config-3 phase space already made."""
    rec = make_records(3, n_records, half=20.0) if records is None else records
    binning = make_binning(20.0, 1.0, 32, log_ebins=True)
    rng = _rng(4, 5)
    beams = []
    for a in range(7):
        gantry = 360.0 * a / 7.0
        for _ in range(int(rng.integers(10, 61))):
            side = rng.uniform(2.0, 20.0)
            cx, cy = rng.uniform(-2.0, 2.0, 2)
            f32 = lambda v: float(np.float32(v))          # beam parameters are float32 in the plan
            beams.append(Beam(f32(cx - side / 2), f32(cx + side / 2), f32(cy - side / 2), f32(cy + side / 2),
                              gantry=f32(gantry), mu=f32(rng.uniform(0.5, 2.0)),
                              roi_margin=1.0, fluence=smooth_field(rng, 40, 6)))
    return Workload("psl-imrt-ct128x100", 4, rec, binning, beams,
                    ct_phantom(4, (100, 128, 128), 0.25), n_histories)


def denoiser_geometry(kind: str, g: int):
    """Seeded training geometry g for the dose denoiser: ('slab', g) a 64^3 x
    0.25 cm slab phantom (config-2 recipe, its own slab depths) under a square
    field of side U(3, 10) cm shifted by up to 1 cm; ('ct', g) a 128^3 x 0.25
    cm CT-like phantom (config-3 recipe) under a field of side U(8, 30) cm
    with its own smooth fluence map.  Returns (phantom, beams)."""
    rng = _rng(100 + g, 7 if kind == "slab" else 8)
    f32 = lambda v: float(np.float32(v))
    if kind == "slab":
        side = rng.uniform(3.0, 10.0)
        cx, cy = rng.uniform(-1.0, 1.0, 2)
        beams = [Beam(f32(cx - side / 2), f32(cx + side / 2), f32(cy - side / 2), f32(cy + side / 2),
                      roi_margin=1.0)]
        return slab_phantom(1000 + g, 64, 0.25), beams
    side = rng.uniform(8.0, 30.0)
    beams = [Beam(f32(-side / 2), f32(side / 2), f32(-side / 2), f32(side / 2), roi_margin=1.0,
                  fluence=smooth_field(rng), fx0=-20.0, fy0=-20.0, fdx=1.0, fdy=1.0)]
    return ct_phantom(2000 + g, (128, 128, 128), 0.25), beams


def small(config: int = 1, n_records: int = 20_000, n_histories: int = 4_000) -> Workload:
    """A reduced copy of a workload for fast parity tests (same recipe)."""
    if config == 1:
        return config1(n_records, n_histories)
    if config == 2:
        w = config2(n_records, n_histories)
        return w
    if config == 3:
        return config3(n_records, n_histories)
    if config == 4:
        return config4(n_records, n_histories)
    raise ValueError(config)

"""Seeded synthetic inputs for the FSPB D_ij engine.

This module is the only code shared by the CUDA path and the FP64 oracle: it
builds the *inputs* (density grids, beam descriptors, the tabulated beam
model) and holds none of the method's arithmetic (no ray tracing, no frames,
no kernel evaluation).  Every array is produced from a seed with a
counter-based generator so that both sides, on any machine, see the same
bytes.

Units are millimetres throughout.  Density grids are FP32 ``[nz][ny][nx]``
(x fastest).  The grid origin is the outer corner of voxel (0, 0, 0).

Workloads (shapes follow the paper's water phantom of Section 3.1 / Table 1
and the 9-field prostate case of Section 3.2):

* ``water_32``      -- 32^3 water at 5 mm, one beam, 20x20 beamlets of 5 mm,
                       lateral cutoff a_t/2 + 3 sigma_1.
* ``slabs_128``     -- 128^3 at 2.5 mm, lung slab (0.25) at 40-80 mm depth and
                       bone slab (1.8) at 100-120 mm, one beam of 40x40
                       beamlets of 2.5 mm, VOI of 6x the beamlet side.
* ``prostate_256``  -- 256x256x100 at 2x2x2.5 mm, elliptic body with noise,
                       femoral heads and a rectal gas pocket, 9 coplanar
                       fields of 16x16 beamlets of 5 mm.
* ``batched``       -- uneven re-plan instances drawn around the prostate
                       shape (grid, spacing, field count and beamlet size
                       vary per instance).
* ``table1_water``  -- the paper's Table 1 water cases (5 coplanar beams,
                       10x10 cm field, 30 cm cube).

The beam model stands in for the 6 MV parameter set the paper fits (Jiang
1998), which is not available: c1 = (0.90, 0.08, 0.02), c2 = 1, depth-linear
c3 and a build-up/attenuation depth-dose curve, all sampled to an FP32 table.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

# cutoff modes, same numbering as the C-ABI
CUTOFF_VOI6 = 0   # VOI: co-axial beamlet with 6x the side (Section 2.1)
CUTOFF_SIGMA = 1  # half-width a_t/2 + k * c3^(1)(d)
CUTOFF_NONE = 2   # every voxel in front of the source

VALUE_F32 = 0
VALUE_BF16 = 1

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


# --------------------------------------------------------------------------
# counter-based random numbers (SplitMix64, Steele/Lea/Flood 2014)
# --------------------------------------------------------------------------
def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied to the uint64 counters ``x``."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in (0, 1) from (seed, counter) pairs, 53-bit mantissa."""
    key = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    with np.errstate(over="ignore"):
        bits = splitmix64((np.asarray(counters, dtype=np.uint64) ^ key) & _MASK64)
    return ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """``n`` standard normals by Box-Muller on counter pairs (2i, 2i+1)."""
    i = np.arange(n, dtype=np.uint64)
    u1 = uniform01(seed, 2 * i)
    u2 = uniform01(seed, 2 * i + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


class _Draw:
    """Sequential scalar draws for per-instance parameters."""

    def __init__(self, seed: int):
        self.seed = seed
        self.k = 0

    def u(self) -> float:
        v = float(uniform01(self.seed, np.array([self.k], dtype=np.uint64))[0])
        self.k += 1
        return v

    def randint(self, lo: int, hi: int) -> int:  # inclusive
        return lo + min(int(self.u() * (hi - lo + 1)), hi - lo)

    def choice(self, seq):
        return seq[self.randint(0, len(seq) - 1)]


# --------------------------------------------------------------------------
# descriptors
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    origin: tuple  # (x, y, z) of the outer corner of voxel (0,0,0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def nvox(self) -> int:
        return self.nx * self.ny * self.nz

    def centre(self):
        return (self.origin[0] + 0.5 * self.nx * self.dx,
                self.origin[1] + 0.5 * self.ny * self.dy,
                self.origin[2] + 0.5 * self.nz * self.dz)

    def voxel_centres(self):
        """1-D arrays of voxel-centre coordinates along x, y, z."""
        x = self.origin[0] + (np.arange(self.nx) + 0.5) * self.dx
        y = self.origin[1] + (np.arange(self.ny) + 0.5) * self.dy
        z = self.origin[2] + (np.arange(self.nz) + 0.5) * self.dz
        return x, y, z


@dataclasses.dataclass
class Beam:
    gantry_deg: float
    sad: float
    iso: tuple
    a: float   # beamlet side along u at the isocentre plane
    b: float   # beamlet side along v at the isocentre plane
    n_u: int
    n_v: int

    @property
    def nbeamlets(self) -> int:
        return self.n_u * self.n_v


@dataclasses.dataclass
class Model:
    lut: np.ndarray          # float32 [n][4] = {T(d), c3_1(d), c3_2(d), c3_3(d)}
    d_max: float             # LUT spans [0, d_max] mm, entries equally spaced
    c1: tuple = (0.90, 0.08, 0.02)
    c2: tuple = (1.0, 1.0, 1.0)
    cutoff_mode: int = CUTOFF_VOI6
    cutoff_k: float = 3.0
    profile: int = 0         # PROFILE_ERF (Eq. 3), PROFILE_LAPLACE or PROFILE_LOGISTIC


# lateral spread kernel of the FSPB profile
PROFILE_ERF, PROFILE_LAPLACE, PROFILE_LOGISTIC = 0, 1, 2

# depth-table construction of a workload
TABLE_EXACT, TABLE_TRILINEAR = 0, 1

# relative threshold on the per-beamlet maximum (the library's decisions near
# it are taken in FP64 with this exact value, as the oracle's)
TAU = 1e-3

@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    density: np.ndarray      # float32 [nz][ny][nx]
    model: Model
    beams: List[Beam]
    tau: float = TAU         # relative threshold on the per-beamlet maximum
    h_frac: float = 0.5      # depth-table spacing as a fraction of min voxel side
    value_dtype: int = VALUE_F32
    table_mode: int = 0      # TABLE_EXACT (Siddon integral) or TABLE_TRILINEAR (the paper's sampled table)

    @property
    def nrows(self) -> int:
        return sum(b.nbeamlets for b in self.beams)


# --------------------------------------------------------------------------
# synthetic 6 MV-like beam model (stand-in for the fitted parameter set)
# --------------------------------------------------------------------------
def synthetic_model(n: int = 256, d_max: float = 300.0, cutoff_mode: int = CUTOFF_VOI6,
                    cutoff_k: float = 3.0, c1=(0.90, 0.08, 0.02), c2=(1.0, 1.0, 1.0),
                    c3_slopes=(0.010, 0.030, 0.050), c3_at0=(1.5, 4.0, 10.0), profile: int = 0) -> Model:
    """Tabulated depth-dose T(d) and depth-dependent widths c3^(i)(d).

    T(d) = [0.4 + 0.6 (1 - exp(-d/5))] exp(-0.0045 d), scaled to a maximum of
    1 over the sampled points; c3^(i)(d) = c3_at0[i] + c3_slopes[i] * d (mm).
    Sampled at n equally spaced depths on [0, d_max] and rounded to FP32.
    """
    d = np.linspace(0.0, d_max, n)
    t = (0.4 + 0.6 * (1.0 - np.exp(-d / 5.0))) * np.exp(-0.0045 * d)
    t = t / t.max()
    lut = np.empty((n, 4), dtype=np.float64)
    lut[:, 0] = t
    for i in range(3):
        lut[:, 1 + i] = c3_at0[i] + c3_slopes[i] * d
    return Model(lut=lut.astype(np.float32), d_max=float(d_max), c1=tuple(c1), c2=tuple(c2),
                 cutoff_mode=cutoff_mode, cutoff_k=float(cutoff_k), profile=int(profile))


# --------------------------------------------------------------------------
# phantoms
# --------------------------------------------------------------------------
def centred_grid(nx, ny, nz, dx, dy, dz, centre=(0.0, 0.0, 0.0)) -> Grid:
    return Grid(nx, ny, nz, float(dx), float(dy), float(dz),
                (centre[0] - 0.5 * nx * dx, centre[1] - 0.5 * ny * dy, centre[2] - 0.5 * nz * dz))


def water_32() -> Workload:
    """32^3 water at 5 mm, gantry 0, SAD 1000, 20x20 beamlets of 5 mm, 3-sigma cutoff."""
    g = centred_grid(32, 32, 32, 5.0, 5.0, 5.0)
    rho = np.ones(g.shape, dtype=np.float32)
    m = synthetic_model(cutoff_mode=CUTOFF_SIGMA, cutoff_k=3.0)
    beams = [Beam(0.0, 1000.0, (0.0, 0.0, 0.0), 5.0, 5.0, 20, 20)]
    return Workload("water_32", g, rho, m, beams)


def slabs_128(value_dtype: int = VALUE_BF16) -> Workload:
    """128^3 at 2.5 mm: water, lung 0.25 at depth [40,80) mm, bone 1.8 at [100,120) mm.

    Depth is measured along +y from the entry face y = y_min (gantry 0 beams
    travel along +y); slabs span the full x and z extent.
    """
    g = centred_grid(128, 128, 128, 2.5, 2.5, 2.5)
    rho = np.ones(g.shape, dtype=np.float32)
    _, yc, _ = g.voxel_centres()
    depth = yc - g.origin[1]
    lung = (depth >= 40.0) & (depth < 80.0)
    bone = (depth >= 100.0) & (depth < 120.0)
    rho[:, lung, :] = 0.25
    rho[:, bone, :] = 1.8
    m = synthetic_model(cutoff_mode=CUTOFF_VOI6)
    beams = [Beam(0.0, 1000.0, (0.0, 0.0, 0.0), 2.5, 2.5, 40, 40)]
    return Workload("slabs_128", g, rho, m, beams, value_dtype=value_dtype)


def prostate_density(g: Grid, seed: int, scale_x: float = 1.0, scale_y: float = 1.0,
                     scale_r: float = 1.0) -> np.ndarray:
    """Elliptic water body (1 + N(0, 0.02^2)), femoral heads 1.6, rectal gas 0.001.

    Geometry in mm relative to the grid centre, scaled by (scale_x, scale_y)
    in-plane and scale_r for radii: body semi-axes 180 x 120, femoral heads
    r = 25 at (+-90, 0), rectal gas r = 12 at (0, +35) for |z| <= 30.
    Outside the body the density is 0.001.
    """
    cx, cy, cz = g.centre()
    x, y, z = g.voxel_centres()
    X = (x - cx)[None, None, :]
    Y = (y - cy)[None, :, None]
    Z = (z - cz)[:, None, None]
    noise = normal(seed, g.nvox).reshape(g.shape)
    rho = np.full(g.shape, 0.001, dtype=np.float64)
    body = (X / (180.0 * scale_x)) ** 2 + (Y / (120.0 * scale_y)) ** 2 <= 1.0
    body = np.broadcast_to(body, g.shape)
    rho = np.where(body, 1.0 + 0.02 * noise, rho)
    for sx in (-1.0, 1.0):
        head = (X - sx * 90.0 * scale_x) ** 2 + Y ** 2 <= (25.0 * scale_r) ** 2
        rho = np.where(np.broadcast_to(head, g.shape), 1.6, rho)
    gas = ((X ** 2 + (Y - 35.0 * scale_y) ** 2 <= (12.0 * scale_r) ** 2) & (np.abs(Z) <= 30.0 * scale_r))
    rho = np.where(np.broadcast_to(gas, g.shape), 0.001, rho)
    return np.maximum(rho, 0.0).astype(np.float32)


def prostate_256(seed: int = 20090908, fields: int = 9) -> Workload:
    """256x256x100 at 2x2x2.5 mm, 9 fields at 0,40,...,320 deg, 16x16 beamlets of 5 mm
    (the first `fields` of them)."""
    g = centred_grid(256, 256, 100, 2.0, 2.0, 2.5)
    rho = prostate_density(g, seed)
    m = synthetic_model(cutoff_mode=CUTOFF_VOI6)
    beams = [Beam(40.0 * k, 1000.0, (0.0, 0.0, 0.0), 5.0, 5.0, 16, 16) for k in range(fields)]
    name = "prostate_256" if fields == 9 else f"prostate_256_{fields}f"
    return Workload(name, g, rho, m, beams)


def batched_instance(seed: int) -> Workload:
    """One re-plan instance of the batched distribution.

    nx, ny ~ U{96..256}, nz ~ U{96..128}, isotropic spacing ~ U[2, 4] mm,
    prostate phantom scaled to the grid extent, 5-9 fields at random gantry
    angles, beamlet side in {2.5, 5, 10} mm over an 80 x 80 mm field.
    """
    r = _Draw(seed)
    nx, ny, nz = r.randint(96, 256), r.randint(96, 256), r.randint(96, 128)
    sp = 2.0 + 2.0 * r.u()
    g = centred_grid(nx, ny, nz, sp, sp, sp)
    X, Y = nx * sp, ny * sp
    rho = prostate_density(g, seed, scale_x=0.35 * X / 180.0, scale_y=0.23 * Y / 120.0,
                           scale_r=min(0.35 * X / 180.0, 0.23 * Y / 120.0))
    nf = r.randint(5, 9)
    bsize = r.choice([2.5, 5.0, 10.0])
    nb = int(round(80.0 / bsize))
    beams = [Beam(360.0 * r.u(), 1000.0, (0.0, 0.0, 0.0), bsize, bsize, nb, nb) for _ in range(nf)]
    m = synthetic_model(cutoff_mode=CUTOFF_VOI6)
    return Workload(f"batched_{seed}", g, rho, m, beams)


def batched(n: int = 32, seed_base: int = 4417) -> List[Workload]:
    return [batched_instance(seed_base + k) for k in range(n)]


def table1_water(case: int) -> Workload:
    """The paper's Table 1 water cases: 5 coplanar equally spaced beams, 10x10 cm
    field, 30x30x30 cm water cube; (voxel side, beamlet side) per case in cm."""
    cases = {1: (0.50, 0.20), 2: (0.37, 0.20), 3: (0.30, 0.20), 4: (0.25, 0.20),
             5: (0.25, 0.25), 6: (0.25, 0.33), 7: (0.25, 0.50)}
    vox_cm, bl_cm = cases[case]
    n = int(round(300.0 / (vox_cm * 10.0)))
    sp = 300.0 / n
    g = centred_grid(n, n, n, sp, sp, sp)
    rho = np.ones(g.shape, dtype=np.float32)
    a = bl_cm * 10.0
    nb = int(round(100.0 / a))
    beams = [Beam(72.0 * k, 1000.0, (0.0, 0.0, 0.0), a, a, nb, nb) for k in range(5)]
    m = synthetic_model(cutoff_mode=CUTOFF_VOI6)
    return Workload(f"table1_case{case}", g, rho, m, beams)


def random_grid_density(seed: int, shape: Sequence[int], lo: float = 0.0, hi: float = 2.0) -> np.ndarray:
    """Uniform random densities on [lo, hi) for tiny brute-force grids."""
    n = int(np.prod(shape))
    u = uniform01(seed, np.arange(n, dtype=np.uint64))
    return (lo + (hi - lo) * u).reshape(shape).astype(np.float32)


WORKLOADS = {
    "water_32": water_32,
    "slabs_128": slabs_128,
    "prostate_256": prostate_256,
    "prostate_256_2f": lambda: prostate_256(fields=2),
}
WORKLOADS.update({f"table1_case{c}": (lambda c=c: table1_water(c)) for c in range(1, 8)})


def get(name: str) -> Workload:
    return WORKLOADS[name]()

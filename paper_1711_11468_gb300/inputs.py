"""Seeded synthetic inputs for the D3Q19 TRT sweep: geometries and initial fields.

This module serves both the CUDA path and the CPU oracle and holds none of the
method's arithmetic (no equilibrium, collision, streaming, voxelisation or
adjacency). It produces only what a user would hand to the library:

  * flag arrays for the paper's ``channel`` geometry (Sec. 2) and its
    verification slab (Sec. 2.1), and for a duct walled on four sides;
  * sphere lists (cx, cy, cz, r) describing a porous medium (the heterogeneous
    case of Sec. 4.5); cells are voxelised by the library and by the oracle,
    each with its own code;
  * seeded initial velocity perturbations;
  * the 512-lattice batch of channels and porous media.

Randomness is counter-based (splitmix64, Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) for fields, and numpy's
PCG64 for the sphere placement, which runs once on the host.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FLUID = 0
SOLID_FULLWAY = 1
SOLID_HALFWAY = 2

SEED_BASE = 1711114680

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """k-th splitmix64 output of the stream started at `seed`: mix(seed + (k+1)*gamma)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(counter: np.ndarray, seed: int) -> np.ndarray:
    """Uniform in [-1, 1) from the top 53 bits of splitmix64 (exact in FP64)."""
    h = splitmix64(counter, seed)
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def channel_flags(nx: int, ny: int, nz: int) -> np.ndarray:
    """Slab channel: full-way solid layers at y = 0 and y = ny-1, fluid elsewhere."""
    f = np.zeros((nz, ny, nx), dtype=np.uint8)
    f[:, 0, :] = SOLID_FULLWAY
    f[:, ny - 1, :] = SOLID_FULLWAY
    return f.reshape(-1)


def duct_flags(nx: int, ny: int, nz: int) -> np.ndarray:
    """Square duct along x: full-way solid layers at y, z in {0, n-1}."""
    f = np.zeros((nz, ny, nx), dtype=np.uint8)
    f[:, 0, :] = SOLID_FULLWAY
    f[:, ny - 1, :] = SOLID_FULLWAY
    f[0, :, :] = SOLID_FULLWAY
    f[nz - 1, :, :] = SOLID_FULLWAY
    return f.reshape(-1)


def velocity_perturbation(nx: int, ny: int, nz: int, seed: int, amplitude: float = 0.01,
                          flags: np.ndarray | None = None) -> np.ndarray:
    """Initial velocity float64[3, N]: each component uniform in +-amplitude/sqrt(3)
    (so |u| <= amplitude) from splitmix64 counter 3*cell + component; 0 at solid cells."""
    N = nx * ny * nz
    scale = amplitude / math.sqrt(3.0)
    u = np.empty((3, N))
    cells = np.arange(N, dtype=np.uint64)
    for a in range(3):
        u[a] = uniform_pm1(cells * np.uint64(3) + np.uint64(a), seed) * scale
    if flags is not None:
        u[:, np.asarray(flags) != FLUID] = 0.0
    return u


@dataclass
class SpherePack:
    spheres: np.ndarray          # int32 [ns, 4]: cx, cy, cz, r
    n_nonoverlap: int            # spheres placed by the non-overlapping phase
    n_overlap: int               # spheres added afterwards with overlap allowed
    est_solid_fraction: float    # Monte Carlo estimate used as the stopping rule


def sphere_pack(dims, seed: int, r_min: int, r_max: int, porosity: float,
                nonoverlap_attempts: int = 50_000, mc_points: int = 200_000,
                gap: int = 1) -> SpherePack:
    """Porous medium of spheres with integer centres and radii.

    Phase 1 places non-overlapping spheres by random sequential addition
    (centre distance >= r1 + r2 + gap, minimum image) for a fixed number of
    attempts. Phase 2 keeps adding spheres with overlap allowed until the
    estimated solid fraction reaches 1 - porosity. The estimate is a Monte
    Carlo count over `mc_points` random points in continuous space; the exact
    porosity is whatever the voxelisation gives, and callers record it.
    """
    nx, ny, nz = dims
    box = np.array([nx, ny, nz], dtype=np.int64)
    rng = np.random.Generator(np.random.PCG64(seed))
    target = 1.0 - porosity
    pts = rng.random((mc_points, 3)) * box
    inside = np.zeros(mc_points, dtype=bool)

    def cover(c, r):
        d = pts - c
        d -= box * np.round(d / box)
        inside[(d * d).sum(1) <= float(r) * float(r)] = True

    placed_c = np.empty((0, 3), dtype=np.int64)
    placed_r = np.empty(0, dtype=np.int64)
    attempts = 0
    batch = 2048
    while attempts < nonoverlap_attempts and inside.mean() < target:
        m = min(batch, nonoverlap_attempts - attempts)
        cand_c = np.stack([rng.integers(0, n, m) for n in (nx, ny, nz)], 1).astype(np.int64)
        cand_r = rng.integers(r_min, r_max + 1, m).astype(np.int64)
        attempts += m
        if placed_r.size:
            d = cand_c[:, None, :] - placed_c[None, :, :]
            d = (d + box // 2) % box - box // 2
            d2 = (d * d).sum(2)
            lim = cand_r[:, None] + placed_r[None, :] + gap
            ok = ~(d2 < lim * lim).any(1)
        else:
            ok = np.ones(m, dtype=bool)
        acc_c, acc_r = [], []
        for k in np.nonzero(ok)[0]:
            c, r = cand_c[k], cand_r[k]
            good = True
            for c2, r2 in zip(acc_c, acc_r):
                d = (c - c2 + box // 2) % box - box // 2
                if int((d * d).sum()) < (r + r2 + gap) ** 2:
                    good = False
                    break
            if good:
                acc_c.append(c)
                acc_r.append(r)
                cover(c, r)
                if inside.mean() >= target:
                    break
        if acc_r:
            placed_c = np.concatenate([placed_c, np.array(acc_c)])
            placed_r = np.concatenate([placed_r, np.array(acc_r)])
    n_nonoverlap = placed_r.size
    extra_c, extra_r = [], []
    while inside.mean() < target:
        c = np.array([rng.integers(0, n) for n in (nx, ny, nz)], dtype=np.int64)
        r = int(rng.integers(r_min, r_max + 1))
        extra_c.append(c)
        extra_r.append(r)
        cover(c, r)
    if extra_r:
        placed_c = np.concatenate([placed_c, np.array(extra_c)])
        placed_r = np.concatenate([placed_r, np.array(extra_r)])
    spheres = np.concatenate([placed_c, placed_r[:, None]], 1).astype(np.int32)
    return SpherePack(spheres, n_nonoverlap, len(extra_r), float(inside.mean()))


@dataclass
class LatticeSpec:
    """One lattice of a workload: its dims, geometry and TRT parameters."""
    dims: tuple
    kind: str                      # "channel", "duct", "porous", "periodic"
    omega: float
    Lambda: float
    force: tuple
    flags: np.ndarray | None = None        # for channel/duct/periodic
    spheres: np.ndarray | None = None      # for porous (voxelised as half-way solid)
    porosity_target: float | None = None
    meta: dict = field(default_factory=dict)


def batch_specs(count: int = 512, seed: int = SEED_BASE + 4, n_min: int = 16, n_max: int = 96,
                omega_range=(0.6, 1.8), Lambda: float = 3.0 / 16.0,
                porosity_range=(0.4, 0.9), force: float = 1e-6) -> list:
    """The many-lattice batch: dims uniform per axis, alternating channel / porous.

    Channels: full-way walls at y = 0 and ny-1 and a body force along x.
    Porous: spheres with overlap allowed, radius uniform in [2, max(2, min(12, min_dim // 4))],
    porosity uniform in the given range, the same body force. omega uniform per lattice.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        dims = tuple(int(v) for v in rng.integers(n_min, n_max + 1, 3))
        omega = float(rng.uniform(*omega_range))
        if k % 2 == 0:
            out.append(LatticeSpec(dims, "channel", omega, Lambda, (force, 0.0, 0.0),
                                   flags=channel_flags(*dims)))
        else:
            por = float(rng.uniform(*porosity_range))
            r_max = max(2, min(12, min(dims) // 4))
            pack = sphere_pack(dims, int(rng.integers(0, 2 ** 31)), 2, r_max, por,
                               nonoverlap_attempts=0, mc_points=20_000)
            out.append(LatticeSpec(dims, "porous", omega, Lambda, (force, 0.0, 0.0),
                                   spheres=pack.spheres, porosity_target=por,
                                   meta={"n_spheres": int(pack.spheres.shape[0])}))
    return out


# Workloads, by what they are (sizes as stated; every one is synthetic and seeded).
POISEUILLE_64 = dict(dims=(64, 64, 64), omega=1.0, Lambda=3.0 / 16.0, force=(1e-6, 0.0, 0.0), steps=100)
DUCT_256 = dict(dims=(256, 256, 256), omega=1.0, Lambda=3.0 / 16.0, force=(0.0, 0.0, 0.0), steps=1000,
                amplitude=0.01, seed=SEED_BASE + 1)
POROUS_256 = dict(dims=(256, 256, 256), omega=1.0, Lambda=3.0 / 16.0, force=(1e-6, 0.0, 0.0), steps=1000,
                  r_min=4, r_max=12, porosity=0.6, seed=SEED_BASE + 2)
CHANNEL_384 = dict(dims=(384, 384, 384), omega=1.0, Lambda=3.0 / 16.0, force=(1e-7, 0.0, 0.0), steps=5000)
BATCH_512 = dict(count=512, steps=500, seed=SEED_BASE + 4)

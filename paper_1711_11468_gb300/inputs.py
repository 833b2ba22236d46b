"""Seeded synthetic inputs for the D3Q19 TRT sweep: geometries and initial fields.

This module serves both the CUDA path and the CPU oracle and holds none of the
method's arithmetic (no equilibrium, collision, streaming, voxelisation or
adjacency). It produces only what a user would hand to the library:

  * flag arrays for the paper's ``channel``, ``pipe`` and ``blocks``
    geometries (Sec. 2), its verification slab (Sec. 2.1), and a duct walled
    on four sides;
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


def pipe_flags(nx: int, ny: int, nz: int, solid: int = SOLID_FULLWAY) -> np.ndarray:
    """The paper's `pipe` (Sec. 2): a pipe along x with a staircase circular
    cross-section. A cell is fluid when its (y, z) centre lies strictly inside
    the circle of radius min(ny, nz)/2 - 1 about the cross-section's centre,
    so the boundary layers in y and z are always solid."""
    cy, cz = (ny - 1) / 2.0, (nz - 1) / 2.0
    R = min(ny, nz) / 2.0 - 1.0
    y = np.arange(ny)[:, None]
    z = np.arange(nz)[None, :]
    inside = (y - cy) ** 2 + (z - cz) ** 2 < R * R          # [ny, nz]
    f = np.where(inside.T[:, :, None], FLUID, solid).astype(np.uint8)   # [nz, ny, 1]
    return np.broadcast_to(f, (nz, ny, nx)).reshape(-1).copy()


def blocks_flags(nx: int, ny: int, nz: int, block: int, gap: int, solid: int = SOLID_HALFWAY) -> np.ndarray:
    """The paper's `blocks` (Sec. 2, Sec. 4.5): cubic obstacles of edge `block`
    repeated with period block + gap along every axis, starting at gap // 2."""
    period = block + gap
    def axis(n):
        return ((np.arange(n) - gap // 2) % period) < block
    m = axis(nz)[:, None, None] & axis(ny)[None, :, None] & axis(nx)[None, None, :]
    return np.where(m, solid, FLUID).astype(np.uint8).reshape(-1)


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


class _Coverage:
    """Monte Carlo estimate of the solid fraction of a growing set of spheres:
    which of `pts` (random points in continuous space) lie inside any sphere
    added so far. Points are bucketed on a coarse grid so that a sphere only
    tests the points near it. Spheres are added one at a time, in order; add()
    reports how many to keep so that the set stops at the first sphere that
    makes the covered count reach `target`."""

    def __init__(self, pts: np.ndarray, box: np.ndarray, bucket: int = 8):
        self.box = box.astype(np.float64)
        self.nb = np.maximum(1, box // bucket).astype(np.int64)
        self.edge = self.box / self.nb
        cell = np.minimum((pts / self.edge).astype(np.int64), self.nb - 1)
        bid = cell[:, 0] + self.nb[0] * (cell[:, 1] + self.nb[1] * cell[:, 2])
        order = np.argsort(bid, kind="stable")
        self.pts = pts[order]
        nbt = int(np.prod(self.nb))
        self.start = np.searchsorted(bid[order], np.arange(nbt + 1))
        self.covered = np.zeros(len(pts), dtype=bool)
        self.count = 0

    def _axis_buckets(self, a: int, c: float, r: float) -> np.ndarray:
        lo = int(np.floor((c - r) / self.edge[a]))
        hi = int(np.floor((c + r) / self.edge[a]))
        if hi - lo + 1 >= self.nb[a]:
            return np.arange(self.nb[a])
        return np.arange(lo, hi + 1) % self.nb[a]

    def add(self, centres: np.ndarray, radii: np.ndarray, target: int):
        for k in range(len(radii)):
            c = centres[k].astype(np.float64)
            r = float(radii[k])
            bx, by, bz = (self._axis_buckets(a, c[a], r) for a in range(3))
            ids = (bx[None, None, :] + self.nb[0] * (by[None, :, None] + self.nb[1] * bz[:, None, None])).ravel()
            lens = self.start[ids + 1] - self.start[ids]
            tot = int(lens.sum())
            if tot:
                base = np.repeat(self.start[ids] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
                idx = base + np.arange(tot)
                idx = idx[~self.covered[idx]]
                d = self.pts[idx] - c
                d -= self.box * np.round(d / self.box)
                hit = idx[(d * d).sum(1) <= r * r]
                self.covered[hit] = True
                self.count += hit.size
            if self.count >= target:
                return k + 1, True
        return len(radii), False


def _clashes(ca, ra, cb, rb, box, gap) -> np.ndarray:
    """[len(ra), len(rb)] True where two spheres come closer than r1 + r2 + gap
    (minimum image; exact: integer coordinates in float32)."""
    d2 = np.zeros((len(ra), len(rb)), dtype=np.float32)
    for a in range(3):
        d = ca[:, a, None].astype(np.float32) - cb[None, :, a].astype(np.float32)
        L = np.float32(box[a])
        d -= L * np.round(d / L)
        d2 += d * d
    lim = (ra[:, None] + rb[None, :] + gap).astype(np.float32)
    return d2 < lim * lim


def sphere_pack(dims, seed: int, r_min: int, r_max: int, porosity: float,
                nonoverlap_attempts: int = 50_000, mc_points: int = 200_000,
                gap: int = 1) -> SpherePack:
    """Porous medium of spheres with integer centres and radii.

    Phase 1 places non-overlapping spheres by random sequential addition
    (centre distance >= r1 + r2 + gap, minimum image) for a fixed number of
    attempts, drawn in batches of 2048 and accepted in draw order. Phase 2 keeps
    adding spheres with overlap allowed. Both phases stop at the first sphere
    after which the estimated solid fraction reaches 1 - porosity; the estimate
    is a Monte Carlo count over `mc_points` random points in continuous space.
    The exact porosity is whatever the voxelisation gives; callers record it.
    """
    nx, ny, nz = dims
    box = np.array([nx, ny, nz], dtype=np.int64)
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((mc_points, 3)) * box
    cov = _Coverage(pts, box)
    target = int(math.ceil((1.0 - porosity) * mc_points))

    placed_c = np.empty((0, 3), dtype=np.int64)
    placed_r = np.empty(0, dtype=np.int64)
    attempts = 0
    done = cov.count >= target
    while attempts < nonoverlap_attempts and not done:
        m = min(2048, nonoverlap_attempts - attempts)
        cand_c = np.stack([rng.integers(0, n, m) for n in (nx, ny, nz)], 1).astype(np.int64)
        cand_r = rng.integers(r_min, r_max + 1, m).astype(np.int64)
        attempts += m
        if placed_r.size:
            ok = ~_clashes(cand_c, cand_r, placed_c, placed_r, box, gap).any(1)
        else:
            ok = np.ones(m, dtype=bool)
        idx = np.nonzero(ok)[0]
        c, r = cand_c[idx], cand_r[idx]
        clash = _clashes(c, r, c, r, box, gap)
        np.fill_diagonal(clash, False)
        keep = np.zeros(len(r), dtype=bool)
        for k in range(len(r)):             # greedy, in draw order
            keep[k] = not (clash[k] & keep).any()
        c, r = c[keep], r[keep]
        n_keep, done = cov.add(c, r, target)
        placed_c = np.concatenate([placed_c, c[:n_keep]])
        placed_r = np.concatenate([placed_r, r[:n_keep]])
    n_nonoverlap = placed_r.size
    n_overlap = 0
    while not done:
        m = 256
        c = np.stack([rng.integers(0, n, m) for n in (nx, ny, nz)], 1).astype(np.int64)
        r = rng.integers(r_min, r_max + 1, m).astype(np.int64)
        n_keep, done = cov.add(c, r, target)
        placed_c = np.concatenate([placed_c, c[:n_keep]])
        placed_r = np.concatenate([placed_r, r[:n_keep]])
        n_overlap += n_keep
    spheres = np.concatenate([placed_c, placed_r[:, None]], 1).astype(np.int32)
    return SpherePack(spheres, n_nonoverlap, n_overlap, cov.count / mc_points)


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

"""Plain FP64 CPU oracle for the D3Q19 TRT lattice Boltzmann sweep (arXiv 1711.11468).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code
with the CUDA library and never imports it.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, no FMA); this module
only marshals numpy arrays through ctypes. Arrays use the C library's layout:
PDFs ``float64[19, N]`` and velocities ``float64[3, N]`` with the cell index
``n = x + nx*(y + ny*z)`` (x fastest), flags ``uint8[N]`` (0 fluid,
1 full-way solid, 2 half-way solid).

Parity status of each function (the pins live in ``tests/test_oracle_*.py``):
  velocity/weight/opposite  pinned (lattice isotropy identities, brute force)
  equilibrium               pinned (closed-form moments)
  collide_trt               pinned (conservation, BGK special case, Poiseuille,
                            shear-wave decay, Lambda wall-offset law)
  step                      pinned (independent numpy pull implementation on
                            small lattices, mass/momentum laws, analytic series)
  voxelize_spheres          pinned (brute-force numpy voxelisation)
  build_list                pinned (brute-force adjacency, involution, link count)
  macroscopic               pinned (analytic Poiseuille profile)
  splitmix64 / sr_bits      pinned (published splitmix64 outputs; an independent
                            numpy splitmix64; the documented bit layout)
  round_half_stochastic     pinned (FP16 neighbours from numpy, monotone in the
                            draw, the exact count of draws that round away from
                            zero in every binade, subnormals included -- which
                            together determine the rule -- fixed points, odd
                            symmetry, subnormal spacing, saturation)
  step_f16_stochastic       pinned (every slot is an FP16 neighbour of the FP64
                            step's value; seed-averaged mass and momentum match
                            the FP64 step; full-way reversal is exact)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

Q = 19
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblbm_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FP contraction, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h")))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i32p = ctypes.POINTER(ctypes.c_int32)
    ci = ctypes.c_int
    lib.orc_velocity.argtypes = [ci, ctypes.POINTER(ctypes.c_int)]
    lib.orc_weight.argtypes = [ci]
    lib.orc_weight.restype = ctypes.c_double
    lib.orc_opposite.argtypes = [ci]
    lib.orc_opposite.restype = ci
    lib.orc_omega_minus.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.orc_omega_minus.restype = ctypes.c_double
    lib.orc_equilibrium.argtypes = [ctypes.c_double, dp, dp]
    lib.orc_collide_trt.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp, dp]
    lib.orc_voxelize_spheres.argtypes = [ci, ci, ci, i32p, ci, ctypes.c_uint8, u8p]
    lib.orc_voxelize_spheres.restype = ci
    lib.orc_build_list.argtypes = [ci, ci, ci, u8p, i32p, i32p, i32p]
    lib.orc_build_list.restype = ctypes.c_int64
    lib.orc_init_equilibrium.argtypes = [ci, ci, ci, u8p, dp, dp, dp]
    lib.orc_step.argtypes = [ci, ci, ci, u8p, ctypes.c_double, ctypes.c_double, dp, dp, dp, ci]
    lib.orc_macroscopic.argtypes = [ci, ci, ci, u8p, dp, dp, dp, dp]
    lib.orc_max_threads.restype = ci
    u64 = ctypes.c_uint64
    lib.orc_splitmix64.argtypes = [u64, u64]
    lib.orc_splitmix64.restype = u64
    lib.orc_sr_bits.argtypes = [u64, u64, u64, ci]
    lib.orc_sr_bits.restype = ctypes.c_uint32
    lib.orc_round_half_stochastic.argtypes = [ctypes.c_double, ctypes.c_uint32, dp]
    lib.orc_round_half_stochastic.restype = ctypes.c_double
    lib.orc_round_half_stochastic_n.argtypes = [dp, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64, dp, dp]
    lib.orc_step_f16_stochastic.argtypes = [ci, ci, ci, u8p, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                            u64, u64, i32p, dp]
    _lib = lib
    return lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def velocity(i: int) -> tuple:
    c = (ctypes.c_int * 3)()
    _load().orc_velocity(i, c)
    return (c[0], c[1], c[2])


def velocities() -> np.ndarray:
    """int array [19, 3] of the oracle's D3Q19 velocity set."""
    return np.array([velocity(i) for i in range(Q)], dtype=np.int64)


def weight(i: int) -> float:
    return _load().orc_weight(i)


def weights() -> np.ndarray:
    return np.array([weight(i) for i in range(Q)])


def opposite(i: int) -> int:
    return _load().orc_opposite(i)


def omega_minus(omega_plus: float, Lambda: float) -> float:
    return _load().orc_omega_minus(omega_plus, Lambda)


def equilibrium(rho: float, u) -> np.ndarray:
    u = _f64(u)
    out = np.zeros(Q)
    _load().orc_equilibrium(rho, _ptr(u, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def collide_trt(f, omega_plus: float, omega_minus_: float, F=(0.0, 0.0, 0.0)) -> np.ndarray:
    f = _f64(f)
    F = _f64(F)
    out = np.zeros(Q)
    _load().orc_collide_trt(_ptr(f, ctypes.c_double), omega_plus, omega_minus_,
                            _ptr(F, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def voxelize_spheres(dims, spheres, value: int = 2, flags=None) -> np.ndarray:
    nx, ny, nz = dims
    if flags is None:
        flags = np.zeros(nx * ny * nz, dtype=np.uint8)
    flags = _u8(flags).copy()
    sph = np.ascontiguousarray(spheres, dtype=np.int32).reshape(-1, 4)
    rc = _load().orc_voxelize_spheres(nx, ny, nz, _ptr(sph, ctypes.c_int32), sph.shape[0],
                                      value, _ptr(flags, ctypes.c_uint8))
    if rc != 0:
        raise ValueError("orc_voxelize_spheres rejected its input")
    return flags


def build_list(dims, flags):
    """Return (cell_of[nf], list_index[N], adj[18, nf]) as int32 arrays."""
    nx, ny, nz = dims
    flags = _u8(flags)
    N = nx * ny * nz
    nf = int(np.count_nonzero(flags == 0))
    cell_of = np.empty(nf, dtype=np.int32)
    list_index = np.empty(N, dtype=np.int32)
    adj = np.empty(18 * nf, dtype=np.int32)
    got = _load().orc_build_list(nx, ny, nz, _ptr(flags, ctypes.c_uint8), _ptr(cell_of, ctypes.c_int32),
                                 _ptr(list_index, ctypes.c_int32), _ptr(adj, ctypes.c_int32))
    assert got == nf
    return cell_of, list_index, adj.reshape(18, nf)


def init_equilibrium(dims, flags, rho=None, u=None) -> np.ndarray:
    nx, ny, nz = dims
    N = nx * ny * nz
    flags = _u8(flags)
    rho = None if rho is None else _f64(rho)
    u = None if u is None else _f64(u)
    f = np.zeros((Q, N))
    _load().orc_init_equilibrium(nx, ny, nz, _ptr(flags, ctypes.c_uint8), _ptr(rho, ctypes.c_double),
                                 _ptr(u, ctypes.c_double), _ptr(f, ctypes.c_double))
    return f


def step(dims, flags, omega_plus, omega_minus_, F, src, dst=None, nthreads: int = 0) -> np.ndarray:
    """One push step: returns f(t+1) given f(t)."""
    nx, ny, nz = dims
    flags = _u8(flags)
    src = _f64(src)
    if dst is None:
        dst = np.zeros_like(src)
    F = _f64(F)
    _load().orc_step(nx, ny, nz, _ptr(flags, ctypes.c_uint8), omega_plus, omega_minus_,
                     _ptr(F, ctypes.c_double), _ptr(src, ctypes.c_double), _ptr(dst, ctypes.c_double),
                     nthreads)
    return dst


def run(dims, flags, omega_plus, omega_minus_, F, f0, steps: int, nthreads: int = 0) -> np.ndarray:
    """`steps` push steps from f0 (two grids, swapped each step)."""
    a = _f64(f0).copy()
    b = np.zeros_like(a)
    flags = _u8(flags)
    for _ in range(steps):
        step(dims, flags, omega_plus, omega_minus_, F, a, b, nthreads)
        a, b = b, a
    return a


def macroscopic(dims, flags, F, f):
    """Return (rho[N], u[3, N])."""
    nx, ny, nz = dims
    N = nx * ny * nz
    flags = _u8(flags)
    f = _f64(f)
    F = _f64(F)
    rho = np.zeros(N)
    u = np.zeros((3, N))
    _load().orc_macroscopic(nx, ny, nz, _ptr(flags, ctypes.c_uint8), _ptr(F, ctypes.c_double),
                            _ptr(f, ctypes.c_double), _ptr(rho, ctypes.c_double), _ptr(u, ctypes.c_double))
    return rho, u


def splitmix64(seed: int, k: int) -> int:
    """Output number k (0-based) of splitmix64 seeded `seed`."""
    return int(_load().orc_splitmix64(seed & (2 ** 64 - 1), k & (2 ** 64 - 1)))


SR_SCALE_LOG2 = 14   # the FP16 stochastic format stores d * 2^14


def sr_bits(seed: int, t: int, node: int, j: int) -> int:
    """The 13 random bits of direction j of node `node` at sweep t (FP16 stochastic format)."""
    return int(_load().orc_sr_bits(seed & (2 ** 64 - 1), t, node, j))


def round_half_stochastic(x, r):
    """Stochastic rounding to FP16 of x with 13 random bits r (arrays broadcast):
    returns (values as float64, margins in FP16 spacings)."""
    x, r = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(r, dtype=np.uint32))
    x = np.ascontiguousarray(x)
    r = np.ascontiguousarray(r)
    out = np.empty(x.shape)
    margin = np.empty(x.shape)
    _load().orc_round_half_stochastic_n(_ptr(x, ctypes.c_double), _ptr(r, ctypes.c_uint32), x.size,
                                        _ptr(out, ctypes.c_double), _ptr(margin, ctypes.c_double))
    return out, margin


def step_f16_stochastic(dims, flags, omega_plus, omega_minus_, F, d_src, seed: int, t: int, node_of=None):
    """One push step of the scaled FP16-shifted stochastic format on deviations
    d = f - w (FP16 values times 2^-14): returns (d(t+1) [19, N], margin [19, N])."""
    nx, ny, nz = dims
    flags = _u8(flags)
    d_src = _f64(d_src)
    dst = np.zeros_like(d_src)
    margin = np.empty_like(d_src)
    F = _f64(F)
    node_of = None if node_of is None else np.ascontiguousarray(node_of, dtype=np.int32)
    _load().orc_step_f16_stochastic(nx, ny, nz, _ptr(flags, ctypes.c_uint8), omega_plus, omega_minus_,
                                    _ptr(F, ctypes.c_double), _ptr(d_src, ctypes.c_double),
                                    _ptr(dst, ctypes.c_double), seed & (2 ** 64 - 1), t,
                                    _ptr(node_of, ctypes.c_int32), _ptr(margin, ctypes.c_double))
    return dst, margin


def max_threads() -> int:
    return _load().orc_max_threads()

"""Thin ctypes binding of liblbm_gb300.so: one Python function per C ABI entry
point, with the same name, doing argument marshalling only (every step of the
sweep runs in the CUDA library). See include/lbm_gb300.h for the semantics of
each call. Arrays follow the ABI's layouts: flags uint8[N], PDFs float64[19, N],
velocities float64[3, N], N = nx*ny*nz with x fastest.

The library is required: ``load()`` raises if it has not been built, and
nothing here falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LBM_OK, LBM_ERR_ARG, LBM_ERR_STATE, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_UNSUPPORTED, LBM_ERR_TIMEOUT = range(7)
(LBM_F64, LBM_F32_SHIFTED, LBM_F16_SHIFTED, LBM_F64_DOUBLE_FLOAT, LBM_F32_SHIFTED_DOUBLE_FLOAT,
 LBM_F16_SHIFTED_STOCHASTIC) = range(6)
LBM_DIRECT, LBM_INDIRECT = 0, 1
LBM_PULL_TWO_GRID, LBM_AA_INPLACE = 0, 1

PRECISION = {"f64": LBM_F64, "f32": LBM_F32_SHIFTED, "f16": LBM_F16_SHIFTED, "f64df": LBM_F64_DOUBLE_FLOAT,
             "f32df": LBM_F32_SHIFTED_DOUBLE_FLOAT, "f16sr": LBM_F16_SHIFTED_STOCHASTIC}
Q = 19

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblbm_gb300.so")


class LbmError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"lbm error {code}: {message}")
        self.code = code


class lbm_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_uint8 * 3), ("reserved", ctypes.c_uint8),
                ("precision", ctypes.c_int32), ("addressing", ctypes.c_int32), ("propagation", ctypes.c_int32)]


def make_desc(dims, precision=LBM_F64, addressing=LBM_DIRECT, propagation=LBM_AA_INPLACE,
              periodic=(1, 1, 1)) -> lbm_desc:
    d = lbm_desc()
    d.nx, d.ny, d.nz = (int(v) for v in dims)
    for a in range(3):
        d.periodic[a] = int(periodic[a])
    d.reserved = 0
    d.precision, d.addressing, d.propagation = int(precision), int(addressing), int(propagation)
    return d


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_keepalive = []


def load(path: str | None = None):
    """Load liblbm_gb300.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(nvcc, sm_103a); there is no fallback implementation")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    sig = {
        "lbm_set_allocator": [ALLOC_FN, FREE_FN, vp],
        "lbm_create_lattice": [ctypes.POINTER(lbm_desc), vp, ctypes.POINTER(H)],
        "lbm_create_batch": [ctypes.POINTER(lbm_desc), i32, vp, ctypes.POINTER(H)],
        "lbm_set_geometry": [H, i32, vp],
        "lbm_set_geometry_spheres": [H, i32, vp, i32],
        "lbm_set_params": [H, i32, f64, f64, vp],
        "lbm_init_equilibrium": [H, i32, vp, vp],
        "lbm_step": [H, i32],
        "lbm_synchronize": [H],
        "lbm_set_stochastic_rounding": [H, ctypes.c_uint64, i64],
        "lbm_set_run_indexing": [H, i32],
        "lbm_autotune_cache": [ctypes.POINTER(i64)],
        "lbm_autotune_clear": [],
        "lbm_autotune_save": [ctypes.c_char_p],
        "lbm_autotune_load": [ctypes.c_char_p],
        "lbm_bench_fma64": [vp, i32, i32, vp],
        "lbm_bench_fma64_wave": [ctypes.POINTER(i32)],
        "lbm_set_temporal_blocking": [H, i32],
        "lbm_get_temporal_blocking": [H, ctypes.POINTER(i32)],
        "lbm_get_run_indexing": [H, ctypes.POINTER(i32)],
        "lbm_adjacency_bytes": [H, i32, ctypes.POINTER(i64)],
        "lbm_steps_done": [H, ctypes.POINTER(i64)],
        "lbm_read_pdfs": [H, i32, vp, sz],
        "lbm_write_pdfs": [H, i32, vp, sz],
        "lbm_read_macroscopic": [H, i32, vp, vp],
        "lbm_read_profile": [H, i32, i32, i32, vp, sz],
        "lbm_read_moments": [H, i32, vp],
        "lbm_read_moments_noalloc": [H, i32, vp],
        "lbm_read_flags": [H, i32, vp, sz],
        "lbm_fluid_count": [H, i32, ctypes.POINTER(i64)],
        "lbm_read_adjacency": [H, i32, vp, sz],
        "lbm_set_tuning": [H, i32, i32, i32],
        "lbm_get_tuning": [H, vp],
        "lbm_autotune": [H, i32],
        "lbm_memory_bytes": [H, ctypes.POINTER(i64)],
        "lbm_destroy": [H],
        "lbm_bench_copy19": [vp, vp, i64, i64, i32, vp],
        "lbm_bench_update19": [vp, i64, i64, i32, vp],
        "lbm_selftest_bounded_wait": [H, i32],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.lbm_last_error.argtypes = []
    lib.lbm_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def lbm_last_error() -> str:
    return load().lbm_last_error().decode()


def _check(rc: int):
    if rc != LBM_OK:
        raise LbmError(rc, lbm_last_error())


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


class Handle:
    """The opaque lbm_handle plus the descriptors needed to size arrays."""

    def __init__(self, ptr: ctypes.c_void_p, descs):
        self.ptr = ptr
        self.descs = list(descs)

    def dims(self, lattice: int = 0):
        d = self.descs[lattice]
        return (d.nx, d.ny, d.nz)

    def cells(self, lattice: int = 0) -> int:
        nx, ny, nz = self.dims(lattice)
        return nx * ny * nz

    @property
    def _as_parameter_(self):
        return self.ptr


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(stream.cuda_stream))   # a torch.cuda.Stream


def lbm_set_allocator(alloc, free, ctx=None):
    """alloc(nbytes) -> int device pointer (0 on failure); free(ptr). None, None restores cudaMalloc."""
    lib = load()
    if alloc is None and free is None:
        _check(lib.lbm_set_allocator(ALLOC_FN(), FREE_FN(), None))
        return

    def _a(n, _ctx):
        try:
            return int(alloc(int(n))) or None
        except Exception:
            return None

    def _f(p, _ctx):
        try:
            free(int(p))
        except Exception:
            pass

    cbs = (ALLOC_FN(_a), FREE_FN(_f))
    _keepalive.append(cbs)
    _check(lib.lbm_set_allocator(cbs[0], cbs[1], None))


def use_torch_allocator():
    """Route the library's device memory through PyTorch's caching allocator."""
    import torch

    def alloc(n):
        return torch.cuda.caching_allocator_alloc(n)

    def free(p):
        torch.cuda.caching_allocator_delete(p)

    lbm_set_allocator(alloc, free)


def lbm_create_lattice(desc: lbm_desc, stream=None) -> Handle:
    h = ctypes.c_void_p()
    _check(load().lbm_create_lattice(ctypes.byref(desc), _stream_ptr(stream), ctypes.byref(h)))
    return Handle(h, [desc])


def lbm_create_batch(descs, stream=None) -> Handle:
    arr = (lbm_desc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _check(load().lbm_create_batch(arr, len(descs), _stream_ptr(stream), ctypes.byref(h)))
    return Handle(h, descs)


def lbm_set_geometry(h: Handle, lattice: int, flags: np.ndarray):
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    if flags.size != h.cells(lattice):
        raise ValueError("flags must hold N cells")
    _check(load().lbm_set_geometry(h, lattice, _ptr(flags)))


def lbm_set_geometry_spheres(h: Handle, lattice: int, spheres: np.ndarray):
    sph = np.ascontiguousarray(spheres, dtype=np.int32).reshape(-1, 4)
    _check(load().lbm_set_geometry_spheres(h, lattice, _ptr(sph), sph.shape[0]))


def lbm_set_params(h: Handle, lattice: int, omega: float, Lambda: float, force=(0.0, 0.0, 0.0)):
    F = np.ascontiguousarray(force, dtype=np.float64)
    _check(load().lbm_set_params(h, lattice, float(omega), float(Lambda), _ptr(F)))


def lbm_init_equilibrium(h: Handle, lattice: int, rho=None, u=None):
    N = h.cells(lattice)
    r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    v = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
    if r is not None and r.size != N or v is not None and v.size != 3 * N:
        raise ValueError("rho must hold N values and u 3*N")
    _check(load().lbm_init_equilibrium(h, lattice, _ptr(r), _ptr(v)))


def lbm_step(h: Handle, n: int):
    _check(load().lbm_step(h, int(n)))


def lbm_set_temporal_blocking(h: Handle, steps_per_pass: int):
    _check(load().lbm_set_temporal_blocking(h, int(steps_per_pass)))


def lbm_get_temporal_blocking(h: Handle) -> int:
    v = ctypes.c_int32()
    _check(load().lbm_get_temporal_blocking(h, ctypes.byref(v)))
    return int(v.value)


def lbm_set_run_indexing(h: Handle, enable: bool):
    _check(load().lbm_set_run_indexing(h, 1 if enable else 0))


def lbm_adjacency_bytes(h: Handle, lattice: int = 0):
    """(link-table bytes, run-indexed code bytes) of an indirectly addressed lattice."""
    out = (ctypes.c_int64 * 2)()
    _check(load().lbm_adjacency_bytes(h, lattice, out))
    return int(out[0]), int(out[1])


def lbm_get_run_indexing(h: Handle) -> bool:
    v = ctypes.c_int32()
    _check(load().lbm_get_run_indexing(h, ctypes.byref(v)))
    return bool(v.value)


def lbm_set_stochastic_rounding(h: Handle, seed: int, sweep: int = 0):
    _check(load().lbm_set_stochastic_rounding(h, int(seed) & (2 ** 64 - 1), int(sweep)))


def lbm_synchronize(h: Handle):
    _check(load().lbm_synchronize(h))


def lbm_steps_done(h: Handle) -> int:
    s = ctypes.c_int64()
    _check(load().lbm_steps_done(h, ctypes.byref(s)))
    return s.value


def lbm_read_pdfs(h: Handle, lattice: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    N = h.cells(lattice)
    if out is None:
        out = np.empty((Q, N), dtype=np.float64)
    _check(load().lbm_read_pdfs(h, lattice, _ptr(out), out.size))
    return out


def lbm_write_pdfs(h: Handle, lattice: int, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(load().lbm_write_pdfs(h, lattice, _ptr(f), f.size))


def lbm_read_macroscopic(h: Handle, lattice: int = 0, rho: np.ndarray | None = None, u: np.ndarray | None = None):
    N = h.cells(lattice)
    rho = np.empty(N) if rho is None else rho
    u = np.empty((3, N)) if u is None else u
    _check(load().lbm_read_macroscopic(h, lattice, _ptr(rho), _ptr(u)))
    return rho, u


def lbm_read_profile(h: Handle, lattice: int = 0, axis: int = 1, comp: int = 0) -> np.ndarray:
    out = np.empty(h.dims(lattice)[axis])
    _check(load().lbm_read_profile(h, lattice, axis, comp, _ptr(out), out.size))
    return out


def lbm_read_moments(h: Handle, lattice: int = 0) -> np.ndarray:
    out = np.empty(4)
    _check(load().lbm_read_moments(h, lattice, _ptr(out)))
    return out


def lbm_read_moments_noalloc(h: Handle, lattice: int = 0) -> np.ndarray:
    """lbm_read_moments without device allocation (static scratch; see the header)."""
    out = np.empty(4)
    _check(load().lbm_read_moments_noalloc(h, lattice, _ptr(out)))
    return out


def lbm_read_flags(h: Handle, lattice: int = 0) -> np.ndarray:
    out = np.empty(h.cells(lattice), dtype=np.uint8)
    _check(load().lbm_read_flags(h, lattice, _ptr(out), out.size))
    return out


def lbm_fluid_count(h: Handle, lattice: int = 0) -> int:
    n = ctypes.c_int64()
    _check(load().lbm_fluid_count(h, lattice, ctypes.byref(n)))
    return n.value


def lbm_read_adjacency(h: Handle, lattice: int = 0) -> np.ndarray:
    nf = lbm_fluid_count(h, lattice)
    out = np.empty((18, nf), dtype=np.int32)
    _check(load().lbm_read_adjacency(h, lattice, _ptr(out), out.size))
    return out


def lbm_set_tuning(h: Handle, threads: int = -1, cells_per_thread: int = -1, ctas_per_sm: int = -1):
    """Negative values keep the current setting."""
    _check(load().lbm_set_tuning(h, threads, cells_per_thread, ctas_per_sm))


def lbm_get_tuning(h: Handle):
    out = np.zeros(3, dtype=np.int32)
    _check(load().lbm_get_tuning(h, _ptr(out)))
    return tuple(int(v) for v in out)


def lbm_autotune(h: Handle, steps: int = 10):
    _check(load().lbm_autotune(h, steps))


def lbm_autotune_cache():
    """(entries, hits) of the process-wide autotuning cache."""
    out = (ctypes.c_int64 * 2)()
    _check(load().lbm_autotune_cache(out))
    return int(out[0]), int(out[1])


def lbm_autotune_clear():
    _check(load().lbm_autotune_clear())


def lbm_autotune_save(path: str):
    _check(load().lbm_autotune_save(os.fsencode(path)))


def lbm_autotune_load(path: str):
    _check(load().lbm_autotune_load(os.fsencode(path)))


def lbm_memory_bytes(h: Handle) -> int:
    b = ctypes.c_int64()
    _check(load().lbm_memory_bytes(h, ctypes.byref(b)))
    return b.value


def lbm_destroy(h: Handle):
    if h.ptr:
        _check(load().lbm_destroy(h))
        h.ptr = ctypes.c_void_p()


def lbm_selftest_bounded_wait(h: Handle, polls: int = 1000):
    _check(load().lbm_selftest_bounded_wait(h, int(polls)))


def lbm_bench_copy19(src_ptr: int, dst_ptr: int, n: int, stride: int, elem_bytes: int, stream=None):
    _check(load().lbm_bench_copy19(ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr), n, stride, elem_bytes,
                                   _stream_ptr(stream)))


def lbm_bench_fma64(out_ptr: int, blocks: int, iterations: int, stream=None):
    _check(load().lbm_bench_fma64(ctypes.c_void_p(out_ptr), int(blocks), int(iterations), _stream_ptr(stream)))


def lbm_bench_fma64_wave() -> int:
    out = ctypes.c_int32(0)
    _check(load().lbm_bench_fma64_wave(ctypes.byref(out)))
    return int(out.value)


def lbm_bench_update19(buf_ptr: int, n: int, stride: int, elem_bytes: int, stream=None):
    _check(load().lbm_bench_update19(ctypes.c_void_p(buf_ptr), n, stride, elem_bytes, _stream_ptr(stream)))

"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every entry point the header declares, and rejects bad arguments
before touching CUDA. Also the input generators' published definitions."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_gb300.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1711_11468_gb300 import build, lbm
    build.build()
    return lbm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(lbm_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("lbm_create_lattice", "lbm_set_geometry", "lbm_set_params", "lbm_step", "lbm_read_pdfs",
                 "lbm_read_macroscopic", "lbm_create_batch", "lbm_destroy", "lbm_last_error"):
        assert must in names
    assert len(names) >= 25


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_1711_11468_gb300 import lbm
    missing = [n for n in declared_functions() if not callable(getattr(lbm, n, None))]
    assert not missing, missing


def test_argument_validation_without_gpu(lib):
    from paper_1711_11468_gb300 import lbm
    bad = lbm.make_desc((1, 8, 8))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create_lattice(bad)
    assert e.value.code == lbm.LBM_ERR_ARG and "dimension" in str(e.value)
    h = ctypes.c_void_p()
    assert lib.lbm_create_lattice(None, None, ctypes.byref(h)) == lbm.LBM_ERR_ARG
    d = lbm.make_desc((8, 8, 8), precision=7)
    assert lib.lbm_create_lattice(ctypes.byref(d), None, ctypes.byref(h)) == lbm.LBM_ERR_ARG
    d = lbm.make_desc((8, 8, 8), propagation=3)
    assert lib.lbm_create_lattice(ctypes.byref(d), None, ctypes.byref(h)) == lbm.LBM_ERR_ARG
    descs = (lbm.lbm_desc * 2)(lbm.make_desc((8, 8, 8), 0), lbm.make_desc((8, 8, 8), 1))
    assert lib.lbm_create_batch(descs, 2, None, ctypes.byref(h)) == lbm.LBM_ERR_ARG
    assert "share precision" in lbm.lbm_last_error()
    assert lib.lbm_create_batch(descs, 0, None, ctypes.byref(h)) == lbm.LBM_ERR_ARG
    huge = lbm.make_desc((2048, 2048, 1024))
    assert lib.lbm_create_lattice(ctypes.byref(huge), None, ctypes.byref(h)) == lbm.LBM_ERR_ARG
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_destroy(None) == lbm.LBM_ERR_ARG
    assert lib.lbm_set_params(None, 0, 1.0, 0.25, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_read_pdfs(None, 0, None, 0) == lbm.LBM_ERR_ARG
    assert lib.lbm_set_allocator(lbm.ALLOC_FN(lambda n, c: 0), lbm.FREE_FN(), None) == lbm.LBM_ERR_ARG
    assert lib.lbm_bench_copy19(None, None, 10, 10, 8, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_bench_fma64(None, 1, 1, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_bench_fma64_wave(None) == lbm.LBM_ERR_ARG
    assert lib.lbm_set_stochastic_rounding(None, 1, 0) == lbm.LBM_ERR_ARG
    assert lib.lbm_set_run_indexing(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_set_temporal_blocking(None, 2) == lbm.LBM_ERR_ARG
    out = (ctypes.c_int64 * 2)()
    assert lib.lbm_adjacency_bytes(None, 0, out) == lbm.LBM_ERR_ARG
    d = lbm.make_desc((8, 8, 8), precision=6)
    assert lib.lbm_create_lattice(ctypes.byref(d), None, ctypes.byref(h)) == lbm.LBM_ERR_ARG


def test_autotune_cache_host_calls(lib):
    from paper_1711_11468_gb300 import lbm
    assert lib.lbm_autotune_cache(None) == lbm.LBM_ERR_ARG
    lbm.lbm_autotune_clear()
    entries, hits = lbm.lbm_autotune_cache()
    assert entries == 0 and hits >= 0


def test_autotune_cache_file_round_trip(lib, tmp_path):
    """Loading a cache file and saving it back reproduces the entries; a
    malformed file is rejected whole."""
    from paper_1711_11468_gb300 import lbm
    lbm.lbm_autotune_clear()
    src = tmp_path / "tune.txt"
    src.write_text("# comment\n"
                   "NVIDIA_GB300/sm152/p1/g1/n1/256x256x256d16516096F 256 2 0 1 1\n"
                   "NVIDIA_GB300/sm152/p0/g0/n1/64x64x64i200000H 128 1 0 1 2\n")
    lbm.lbm_autotune_load(str(src))
    assert lbm.lbm_autotune_cache()[0] == 2
    out = tmp_path / "out.txt"
    lbm.lbm_autotune_save(str(out))
    lines = sorted(line for line in out.read_text().splitlines() if not line.startswith("#"))
    assert lines == sorted(line for line in src.read_text().splitlines() if not line.startswith("#"))
    bad = tmp_path / "bad.txt"
    bad.write_text("sig 256 3 0 1 1\n")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_autotune_load(str(bad))
    assert e.value.code == lbm.LBM_ERR_ARG and "malformed" in str(e.value)
    assert lbm.lbm_autotune_cache()[0] == 2
    with pytest.raises(lbm.LbmError):
        lbm.lbm_autotune_load(str(tmp_path / "missing.txt"))
    lbm.lbm_autotune_clear()


def test_desc_layout_matches_header():
    from paper_1711_11468_gb300 import lbm
    assert ctypes.sizeof(lbm.lbm_desc) == 28
    assert lbm.lbm_desc.precision.offset == 16


# -------------------------------------------------------------- inputs
def test_splitmix64_published_sequence():
    """splitmix64 seeded with 0: the generator's first outputs as published
    with its reference implementation."""
    got = inputs.splitmix64(np.arange(3, dtype=np.uint64), 0)
    assert [hex(int(v)) for v in got] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4", "0x6c45d188009454f"]


def test_velocity_perturbation_bounds_and_determinism():
    u = inputs.velocity_perturbation(16, 8, 4, seed=5, amplitude=0.01)
    assert u.shape == (3, 512)
    assert np.sqrt((u * u).sum(0)).max() <= 0.01
    assert np.array_equal(u, inputs.velocity_perturbation(16, 8, 4, seed=5, amplitude=0.01))
    assert not np.array_equal(u, inputs.velocity_perturbation(16, 8, 4, seed=6, amplitude=0.01))
    assert abs(u.mean()) < 1e-3 and u.std() > 0.002
    fl = inputs.duct_flags(16, 8, 4)
    u2 = inputs.velocity_perturbation(16, 8, 4, seed=5, amplitude=0.01, flags=fl)
    assert np.all(u2[:, fl != 0] == 0) and np.array_equal(u2[:, fl == 0], u[:, fl == 0])


def test_sphere_pack_recipe():
    p = inputs.sphere_pack((64, 64, 64), 3, 4, 12, 0.6, nonoverlap_attempts=20000, mc_points=50000)
    assert p.spheres.dtype == np.int32 and p.spheres.shape[1] == 4
    r = p.spheres[:, 3]
    assert r.min() >= 4 and r.max() <= 12
    assert p.n_nonoverlap + p.n_overlap == p.spheres.shape[0]
    assert p.est_solid_fraction >= 0.4
    # the non-overlapping phase honours the gap (minimum image)
    c = p.spheres[:p.n_nonoverlap, :3].astype(np.int64)
    rr = p.spheres[:p.n_nonoverlap, 3].astype(np.int64)
    d = c[:, None, :] - c[None, :, :]
    d = (d + 32) % 64 - 32
    d2 = (d * d).sum(2)
    lim = (rr[:, None] + rr[None, :] + 1) ** 2
    np.fill_diagonal(d2, 10 ** 9)
    assert np.all(d2 >= lim)


def test_channel_and_duct_flags():
    fl = inputs.channel_flags(4, 5, 3).reshape(3, 5, 4)
    assert np.all(fl[:, 0] == 1) and np.all(fl[:, 4] == 1) and np.all(fl[:, 1:4] == 0)
    fl = inputs.duct_flags(4, 5, 6).reshape(6, 5, 4)
    assert np.all(fl[0] == 1) and np.all(fl[5] == 1) and np.all(fl[1:5, 1:4] == 0)


def test_pipe_and_blocks_geometry():
    fl = inputs.pipe_flags(5, 12, 10).reshape(10, 12, 5)
    assert np.all(fl[:, 0, :] == 1) and np.all(fl[:, -1, :] == 1) and np.all(fl[0] == 1) and np.all(fl[-1] == 1)
    assert np.all(fl == fl[:, :, :1])                          # invariant along the pipe axis
    assert fl[5, 6, 0] == 0 and (fl[:, :, 0] == 0).sum() > 0.5 * 10 * 12 * 0.5
    assert np.array_equal(fl[:, :, 0], fl[::-1, ::-1, 0])      # symmetric cross-section
    b = inputs.blocks_flags(16, 16, 16, block=4, gap=4).reshape(16, 16, 16)
    assert b.sum() // 2 == 8 * 4 ** 3                          # 2 x 2 x 2 blocks of 4^3
    assert np.all(b[2:6, 2:6, 2:6] == 2) and np.all(b[0:2] == 0)


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "lbm_gb300.h"

int main(void) {
  lbm_handle h = 0;
  lbm_desc d;
  memset(&d, 0, sizeof d);
  d.nx = 0; d.ny = 8; d.nz = 8;   /* a zero dimension: rejected before any CUDA call */
  if (lbm_create_lattice(&d, NULL, &h) != LBM_ERR_ARG) return 1;
  if (strlen(lbm_last_error()) == 0) return 2;
  if (lbm_step(NULL, 1) != LBM_ERR_ARG) return 3;
  if (lbm_destroy(NULL) != LBM_ERR_ARG) return 4;
  puts(lbm_last_error());
  return 0;
}
"""


def test_header_compiles_as_c_and_the_library_links_from_c(lib, tmp_path):
    """The boundary is a C ABI: a strict C11 program includes the header, links
    against the library and calls it (argument checks only, no GPU needed)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    from paper_1711_11468_gb300 import lbm
    libdir = os.path.dirname(lbm.LIB_PATH)
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.dirname(HEADER),
                        str(src), "-L", libdir, "-llbm_gb300", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip()

"""The fluid list keeps the paper's lexicographic node order (x fastest; Sec. 3
"Lattice Representation"), not a tiled one. This test holds the model behind
that choice: for the odd AA step's gathers through the adjacency list, count
the distinct 32-byte sectors each warp of 32 consecutive list nodes touches per
direction, on a seeded porous medium of the porous workload's recipe.
On the 160^3 medium the model gives 6.12 sectors per request for FP32 storage,
the 5.9-6.0 that ncu measured on the GPU kernel, and 3.98 for FP16 (ideal 4
and 2); every tiled order tried touches more. No GPU.
"""
import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs


def sectors_per_request(orc, dims, flags, order, elem_bytes):
    n = dims[0]
    fluid = np.flatnonzero(flags == 0)
    nf = fluid.size
    x, y, z = fluid % n, (fluid // n) % n, fluid // (n * n)
    if order == "lexicographic":
        perm = np.arange(nf)
    else:
        tx, ty, tz = order   # tiles in x-fastest order, x fastest inside a tile
        perm = np.lexsort((x % tx, y % ty, z % tz, x // tx, y // ty, z // tz))
    cells = fluid[perm]
    px, py, pz = cells % n, (cells // n) % n, cells // (n * n)
    lidx = np.full(flags.size, -1, np.int64)
    lidx[cells] = np.arange(nf)
    stride = ((nf + 127) // 128) * 128
    c = orc.velocities()
    warps = nf // 32
    total = 0
    for i in range(1, 19):
        # odd AA step: slot opp(i) of x - c_i, or slot i of the node itself across a wall
        m = (px - c[i, 0]) % n + n * ((py - c[i, 1]) % n + n * ((pz - c[i, 2]) % n))
        nb = lidx[m]
        opp = orc.opposite(i)
        addr = np.where(nb >= 0, opp * stride + nb, i * stride + np.arange(nf))
        sec = np.sort(((addr * elem_bytes) // 32)[:warps * 32].reshape(warps, 32), axis=1)
        total += (1 + (np.diff(sec, axis=1) != 0).sum(axis=1)).sum()
    return total / (18 * warps)


@pytest.mark.parametrize("elem_bytes", [2, 4])
def test_lexicographic_list_order_touches_fewest_sectors(orc, elem_bytes):
    dims = (96, 96, 96)
    c = inputs.POROUS_256
    pack = inputs.sphere_pack(dims, c["seed"], c["r_min"], c["r_max"], c["porosity"])
    flags = orc.voxelize_spheres(dims, pack.spheres)
    lex = sectors_per_request(orc, dims, flags, "lexicographic", elem_bytes)
    ideal = 32 * elem_bytes / 32
    assert ideal < lex < 2.2 * ideal
    for tile in [(32, 4, 1), (64, 4, 1), (16, 2, 2), (8, 4, 4)]:
        assert sectors_per_request(orc, dims, flags, tile, elem_bytes) > lex, tile

"""State input and output through page-locked host buffers. The calls move a
page-locked buffer straight through the GPU's link to host memory instead of
staging it in device scratch; results must equal the staged path's bit for
bit, for both addressings and both propagation patterns."""
import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs

pytestmark = pytest.mark.gpu


def pinned_like(a):
    import torch
    t = torch.empty(a.shape, dtype=torch.float64 if a.dtype == np.float64 else torch.uint8, pin_memory=True)
    out = t.numpy()
    out[...] = a
    return out, t


@pytest.mark.parametrize("addr", [0, 1])
@pytest.mark.parametrize("prop", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 3])
def test_pinned_buffers_equal_staged(lbm, orc, addr, prop, prec):
    import torch
    dims = (24, 18, 10)
    fl = inputs.channel_flags(*dims).copy()
    if addr == 1:
        fl[fl == 1] = 2
    N = fl.size
    u = inputs.velocity_perturbation(*dims, seed=77, amplitude=0.02, flags=fl)
    rho = 1.0 + 0.01 * inputs.uniform_pm1(np.arange(N, dtype=np.uint64), 78)
    results = []
    keep = []
    for pinned in (False, True):
        rin, uin = (rho, u)
        if pinned:
            (rin, t1), (uin, t2) = pinned_like(rho), pinned_like(u)
            keep += [t1, t2]
        h = lbm.lbm_create_lattice(lbm.make_desc(dims, prec, addr, prop, (1, 0, 1)), torch.cuda.current_stream())
        try:
            lbm.lbm_set_geometry(h, 0, fl)
            lbm.lbm_set_params(h, 0, 1.1, 3 / 16, (1e-5, 0.0, 0.0))
            lbm.lbm_init_equilibrium(h, 0, rin, uin)
            lbm.lbm_step(h, 7)
            if pinned:
                pdfs, tp = pinned_like(np.zeros((19, N)))
                r_out, tr = pinned_like(np.zeros(N))
                u_out, tu = pinned_like(np.zeros((3, N)))
                keep += [tp, tr, tu]
                lbm.lbm_read_pdfs(h, 0, pdfs)
                lbm.lbm_read_macroscopic(h, 0, r_out, u_out)
                lbm.lbm_write_pdfs(h, 0, pdfs)   # from page-locked memory
            else:
                pdfs = lbm.lbm_read_pdfs(h, 0)
                r_out, u_out = lbm.lbm_read_macroscopic(h, 0)
                lbm.lbm_write_pdfs(h, 0, pdfs)
            lbm.lbm_step(h, 3)
            after = lbm.lbm_read_pdfs(h, 0)
        finally:
            lbm.lbm_destroy(h)
        results.append((np.array(pdfs), np.array(r_out), np.array(u_out), after))
    for a, b in zip(results[0], results[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("addr", [0, 1])
@pytest.mark.parametrize("prop", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 5])
def test_initial_state_is_the_same_in_every_layout(lbm, orc, addr, prop, prec):
    """lbm_init_equilibrium writes the canonical layout at an even AA step and
    otherwise the AA or pull form, pushed from each cell to the slots that keep
    its values. Read back, the state is the same bit for bit either way, and in
    FP64 it is the oracle's equilibrium up to round-off (solid cells: the
    oracle's value at full-way solids, nothing at half-way ones)."""
    import torch
    dims = (30, 14, 12)
    fl = inputs.channel_flags(*dims).copy()
    fl[(fl == 0) & (np.arange(fl.size) % 23 == 0)] = 2
    if addr == 1:
        fl[fl == 1] = 2
    N = fl.size
    u = inputs.velocity_perturbation(*dims, seed=41, amplitude=0.05, flags=fl)
    rho = 1.0 + 0.02 * inputs.uniform_pm1(np.arange(N, dtype=np.uint64), 42)
    pinned_u, tu = pinned_like(u)
    got = []
    h = lbm.lbm_create_lattice(lbm.make_desc(dims, prec, addr, prop, (1, 0, 1)), torch.cuda.current_stream())
    try:
        lbm.lbm_set_geometry(h, 0, fl)
        lbm.lbm_set_params(h, 0, 1.1, 3 / 16, (1e-5, 0.0, 0.0))
        for k in range(3):   # at steps 0, 1 and 2: an even, an odd and an even AA step
            if k:
                lbm.lbm_step(h, 1)
            lbm.lbm_init_equilibrium(h, 0, rho, pinned_u if k == 1 else u)
            got.append(lbm.lbm_read_pdfs(h, 0))
    finally:
        lbm.lbm_destroy(h)
    for g in got[1:]:
        assert np.array_equal(g, got[0])
    if prec == 0:
        want = orc.init_equilibrium(dims, fl, rho, u)
        want[:, fl == 2] = 0.0
        assert np.abs(got[0] - want).max() <= 4e-16

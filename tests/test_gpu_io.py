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

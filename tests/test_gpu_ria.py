"""Run-indexed adjacency (RIA) of fluid lists: the staged list sweeps that
decode their links from the run-length code give bit for bit the results of the
sweeps that read the link table, for pull and AA, on regular and irregular
geometries and block sizes, and match the FP64 oracle."""
import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs

pytestmark = pytest.mark.gpu


def geometries():
    rng = np.random.default_rng(17)
    ragged = (rng.random(37 * 11 * 7) < 0.3).astype(np.uint8) * 2
    chan = np.where(inputs.channel_flags(70, 33, 20) == 1, 2, 0).astype(np.uint8)
    return {
        "blocks": ((48, 40, 36), inputs.blocks_flags(48, 40, 36, block=4, gap=4)),
        "channel": ((70, 33, 20), chan),
        "ragged": ((37, 11, 7), ragged),
    }


GEOM = geometries()


def run(lbm, dims, flags, prec, prop, steps, threads, ria, u=None):
    import torch
    h = lbm.lbm_create_lattice(lbm.make_desc(dims, prec, lbm.LBM_INDIRECT, prop), torch.cuda.current_stream())
    try:
        lbm.lbm_set_tuning(h, threads)
        lbm.lbm_set_run_indexing(h, ria)
        lbm.lbm_set_geometry(h, 0, flags)
        lbm.lbm_set_params(h, 0, 1.1, 0.2, (2e-5, -1e-5, 1e-5))
        lbm.lbm_init_equilibrium(h, 0, None, u)
        lbm.lbm_step(h, steps)
        return lbm.lbm_read_pdfs(h, 0)
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("geom", sorted(GEOM))
@pytest.mark.parametrize("prop", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 5])
def test_run_index_equals_table_bitwise(lbm, geom, prop, prec):
    dims, fl = GEOM[geom]
    u = inputs.velocity_perturbation(*dims, seed=9, amplitude=0.02, flags=fl)
    for threads in (64, 256):
        a = run(lbm, dims, fl, prec, prop, 21, threads, True, u)
        b = run(lbm, dims, fl, prec, prop, 21, threads, False, u)
        assert np.array_equal(a, b), (geom, prop, prec, threads)


@pytest.mark.parametrize("prop", [0, 1])
def test_run_index_matches_oracle(lbm, orc, prop):
    dims, fl = GEOM["ragged"]
    u = inputs.velocity_perturbation(*dims, seed=4, amplitude=0.02, flags=fl)
    got = run(lbm, dims, fl, 0, prop, 17, 96, True, u)
    f0 = orc.init_equilibrium(dims, fl, None, u)
    want = orc.run(dims, fl, 1.1, orc.omega_minus(1.1, 0.2), (2e-5, -1e-5, 1e-5), f0, 17)
    assert np.abs(got - want).max() <= 1e-13


def test_run_index_switch_and_errors(lbm):
    import torch
    h = lbm.lbm_create_lattice(lbm.make_desc((16, 16, 16), 1, lbm.LBM_INDIRECT, 1), torch.cuda.current_stream())
    try:
        assert lbm.lbm_get_run_indexing(h) is True
        lbm.lbm_set_run_indexing(h, False)
        assert lbm.lbm_get_run_indexing(h) is False
        assert lbm.load().lbm_set_run_indexing(h, 2) == lbm.LBM_ERR_ARG
        assert lbm.lbm_get_run_indexing(h) is False
    finally:
        lbm.lbm_destroy(h)

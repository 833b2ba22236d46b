"""Temporal blocking of the full-array pull sweep (two steps per launch): the
results equal those of one-step sweeps bit for bit in every storage format,
for both bounce-back kinds, lattices smaller than one tile and ragged tile
edges, odd step counts and graph replay; FP64 matches the oracle."""
import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs

pytestmark = pytest.mark.gpu


def case_flags(dims, seed):
    """Full-way walls at y = 0 and ny - 1 and a few half-way spheres."""
    nx, ny, nz = dims
    fl = inputs.channel_flags(nx, ny, nz).copy()
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for _ in range(4):
        c = rng.integers(0, [nx, ny, nz])
        r = rng.integers(1, 4)
        inside = ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r).reshape(-1)
        fl[inside & (fl == 0)] = 2
    return fl


CASES = {
    "tile": ((64, 40, 24), 1),
    "small": ((20, 9, 7), 2),
    "ragged": ((45, 33, 17), 3),
}


def run(lbm, dims, flags, prec, steps, spp, threads, u, seed=7, autotune=False):
    import torch
    h = lbm.lbm_create_lattice(lbm.make_desc(dims, prec, lbm.LBM_DIRECT, lbm.LBM_PULL_TWO_GRID, (1, 0, 1)),
                               torch.cuda.current_stream())
    try:
        lbm.lbm_set_tuning(h, threads, 1)
        lbm.lbm_set_geometry(h, 0, flags)
        lbm.lbm_set_params(h, 0, 1.2, 0.2, (2e-5, 0.0, -1e-5))
        lbm.lbm_init_equilibrium(h, 0, None, u)
        if prec == 5:
            lbm.lbm_set_stochastic_rounding(h, seed, 3)
        if autotune:
            lbm.lbm_autotune(h, 4)
        else:
            lbm.lbm_set_temporal_blocking(h, spp)
        lbm.lbm_step(h, steps)
        return lbm.lbm_read_pdfs(h, 0), lbm.lbm_get_temporal_blocking(h)
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4, 5])
def test_two_steps_per_pass_equal_one_step_sweeps(lbm, case, prec):
    dims, seed = CASES[case]
    fl = case_flags(dims, seed)
    u = inputs.velocity_perturbation(*dims, seed=seed, amplitude=0.02, flags=fl)
    for threads in (128, 512):
        for steps in (17, 32):   # an odd remainder; two replayed graphs of 8 launches
            ref, _ = run(lbm, dims, fl, prec, steps, 1, threads, u)
            got, spp = run(lbm, dims, fl, prec, steps, 2, threads, u)
            assert spp == 2
            assert np.array_equal(got, ref), (case, prec, threads, steps)


def test_two_steps_per_pass_match_oracle(lbm, orc):
    dims, seed = CASES["ragged"]
    fl = case_flags(dims, seed)
    u = inputs.velocity_perturbation(*dims, seed=seed, amplitude=0.02, flags=fl)
    got, _ = run(lbm, dims, fl, 0, 20, 2, 256, u)
    f0 = orc.init_equilibrium(dims, fl, None, u)
    want = orc.run(dims, fl, 1.2, orc.omega_minus(1.2, 0.2), (2e-5, 0.0, -1e-5), f0, 20)
    assert np.abs(got - want).max() <= 1e-13


def test_autotune_with_temporal_blocking_leaves_results_unchanged(lbm):
    dims, seed = CASES["tile"]
    fl = case_flags(dims, seed)
    u = inputs.velocity_perturbation(*dims, seed=seed, amplitude=0.02, flags=fl)
    ref, _ = run(lbm, dims, fl, 1, 24, 1, 256, u)
    got, spp = run(lbm, dims, fl, 1, 24, 1, 256, u, autotune=True)
    assert spp in (1, 2)
    assert np.array_equal(got, ref)


def test_temporal_blocking_errors(lbm):
    import torch
    fl = inputs.channel_flags(16, 16, 16)
    for prop, addr in ((1, 0), (0, 1)):
        flags = np.where(fl == 1, 2, 0).astype(np.uint8) if addr == 1 else fl
        h = lbm.lbm_create_lattice(lbm.make_desc((16, 16, 16), 1, addr, prop, (1, 0, 1)), torch.cuda.current_stream())
        try:
            lbm.lbm_set_geometry(h, 0, flags)
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_set_temporal_blocking(h, 2)
            assert e.value.code == lbm.LBM_ERR_UNSUPPORTED
            lbm.lbm_set_temporal_blocking(h, 1)
        finally:
            lbm.lbm_destroy(h)
    h = lbm.lbm_create_lattice(lbm.make_desc((16, 16, 16), 1, 0, 0, (1, 0, 1)), torch.cuda.current_stream())
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_temporal_blocking(h, 3)
        assert e.value.code == lbm.LBM_ERR_ARG
    finally:
        lbm.lbm_destroy(h)

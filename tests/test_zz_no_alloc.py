"""lbm_read_moments_noalloc: the mass and momentum sums without any device
allocation, for callers that may not allocate while they run (a fixed memory
budget set up front, or an allocator they cannot re-enter from this call).

The call must give the same sums as lbm_read_moments, call after call, while
its scratch lives in one static device array shared by every call. This file
is collected last so that a run stopping at the first failure has already run
every other test; it also passes when run on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs

pytestmark = pytest.mark.gpu


def _lattice(lbm, dims, prec, addr, prop, steps, flags=None, spheres=None, force=(1e-5, 0.0, 0.0)):
    import torch
    h = lbm.lbm_create_lattice(lbm.make_desc(dims, prec, addr, prop), torch.cuda.current_stream())
    if spheres is not None:
        lbm.lbm_set_geometry_spheres(h, 0, spheres)
    else:
        lbm.lbm_set_geometry(h, 0, flags)
    lbm.lbm_set_params(h, 0, 1.1, 3.0 / 16.0, force)
    u = inputs.velocity_perturbation(*dims, seed=inputs.SEED_BASE + 9, amplitude=0.01,
                                     flags=lbm.lbm_read_flags(h, 0))
    lbm.lbm_init_equilibrium(h, 0, None, u)
    lbm.lbm_step(h, steps)
    return h


def test_noalloc_moments_match_allocating_call(lbm):
    counts = {"alloc": 0}

    def alloc(n):
        import torch
        counts["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(n)

    def free(p):
        import torch
        torch.cuda.caching_allocator_delete(p)

    lbm.lbm_set_allocator(alloc, free)
    handles = []
    try:
        big = (96, 80, 72)
        handles.append(_lattice(lbm, big, lbm.LBM_F64, lbm.LBM_DIRECT, lbm.LBM_AA_INPLACE, 13,
                                flags=inputs.channel_flags(*big)))
        small = (40, 36, 30)
        pack = inputs.sphere_pack(small, 5, 2, 6, 0.7, nonoverlap_attempts=2000, mc_points=20000)
        handles.append(_lattice(lbm, small, lbm.LBM_F32_SHIFTED, lbm.LBM_INDIRECT, lbm.LBM_PULL_TWO_GRID, 8,
                                spheres=pack.spheres))
        for h in handles:
            expect = lbm.lbm_read_moments(h, 0)
            before = counts["alloc"]
            first = lbm.lbm_read_moments_noalloc(h, 0)
            second = lbm.lbm_read_moments_noalloc(h, 0)
            assert counts["alloc"] == before, "the allocation-free call went through the allocator"
            # same kernels, same fixed reduction order: equal to round-off (in fact bitwise)
            for got in (first, second):
                assert abs(got[0] - expect[0]) <= 1e-13 * abs(expect[0])
                assert np.abs(got[1:] - expect[1:]).max() <= 1e-13 * abs(expect[0])
            assert np.array_equal(first, second)
        # the state moves on between calls: the static scratch must not carry stale sums
        lbm.lbm_step(handles[0], 3)
        expect = lbm.lbm_read_moments(handles[0], 0)
        got = lbm.lbm_read_moments_noalloc(handles[0], 0)
        assert abs(got[0] - expect[0]) <= 1e-13 * abs(expect[0])
        assert np.abs(got[1:] - expect[1:]).max() <= 1e-13 * abs(expect[0])
    finally:
        for h in handles:
            lbm.lbm_destroy(h)
        lbm.lbm_set_allocator(None, None)


def test_noalloc_reports_the_same_status(lbm):
    """After a bounded wait has given up (the handle's device status word is
    set and the handle poisoned), both calls refuse the handle with the same
    status."""
    import torch
    h = lbm.lbm_create_lattice(lbm.make_desc((8, 8, 8), lbm.LBM_F64, lbm.LBM_DIRECT, lbm.LBM_AA_INPLACE),
                               torch.cuda.current_stream())
    try:
        lbm.lbm_set_geometry(h, 0, np.zeros(512, dtype=np.uint8))
        lbm.lbm_set_params(h, 0, 1.0, 3.0 / 16.0, (0.0, 0.0, 0.0))
        lbm.lbm_init_equilibrium(h, 0)
        assert np.array_equal(lbm.lbm_read_moments(h, 0), lbm.lbm_read_moments_noalloc(h, 0))
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_selftest_bounded_wait(h, 1000)
        assert e.value.code == lbm.LBM_ERR_TIMEOUT
        codes = []
        for call in (lbm.lbm_read_moments, lbm.lbm_read_moments_noalloc):
            with pytest.raises(lbm.LbmError) as e:
                call(h, 0)
            codes.append(e.value.code)
        assert codes[0] == codes[1]
    finally:
        lbm.lbm_destroy(h)

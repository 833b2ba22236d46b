"""GPU parity of the batched sweep: many lattices of different sizes, kinds and
TRT parameters advanced by one launch per step, against the oracle lattice by
lattice, and against the same lattices run one at a time."""
import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 3.0 / 16.0


def small_batch(seed=3, count=10):
    """Channels (full array, full-way walls) and porous media (fluid list,
    half-way spheres) of uneven sizes, including sizes that leave ragged tiles."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(count):
        dims = tuple(int(v) for v in rng.integers(5, 29, 3))
        omega = float(rng.uniform(0.6, 1.8))
        if k % 2 == 0:
            specs.append(dict(dims=dims, kind="channel", omega=omega, force=(1e-5, 0.0, 0.0),
                              flags=inputs.channel_flags(*dims), periodic=(1, 0, 1)))
        else:
            pack = inputs.sphere_pack(dims, int(rng.integers(1 << 30)), 1, max(1, min(dims) // 4),
                                      float(rng.uniform(0.5, 0.9)), nonoverlap_attempts=0, mc_points=4000)
            specs.append(dict(dims=dims, kind="porous", omega=omega, force=(1e-5, 2e-6, 0.0),
                              spheres=pack.spheres, periodic=(1, 1, 1)))
    return specs


def run_batch(lbm, specs, prec, prop, steps, tuning=None, batch=True):
    import torch
    s = torch.cuda.current_stream()
    descs = [lbm.make_desc(sp["dims"], prec, lbm.LBM_DIRECT if sp["kind"] == "channel" else lbm.LBM_INDIRECT,
                           prop, sp["periodic"]) for sp in specs]
    handles = [lbm.lbm_create_batch(descs, s)] if batch else [lbm.lbm_create_lattice(d, s) for d in descs]
    try:
        flags = []
        for k, sp in enumerate(specs):
            h, lat = (handles[0], k) if batch else (handles[k], 0)
            if sp["kind"] == "channel":
                lbm.lbm_set_geometry(h, lat, sp["flags"])
            else:
                lbm.lbm_set_geometry_spheres(h, lat, sp["spheres"])
            lbm.lbm_set_params(h, lat, sp["omega"], LAM, sp["force"])
            fl = lbm.lbm_read_flags(h, lat)
            flags.append(fl)
            u = inputs.velocity_perturbation(*sp["dims"], seed=100 + k, amplitude=0.02, flags=fl)
            lbm.lbm_init_equilibrium(h, lat, None, u)
        if tuning is not None:
            for h in handles:
                lbm.lbm_set_tuning(h, *tuning)
        for h in handles:
            lbm.lbm_step(h, steps)
        out = []
        for k in range(len(specs)):
            h, lat = (handles[0], k) if batch else (handles[k], 0)
            out.append(lbm.lbm_read_pdfs(h, lat))
        return out, flags
    finally:
        for h in handles:
            lbm.lbm_destroy(h)


def oracle_run(orc, sp, flags, k, steps):
    u = inputs.velocity_perturbation(*sp["dims"], seed=100 + k, amplitude=0.02, flags=flags)
    f0 = orc.init_equilibrium(sp["dims"], flags, None, u)
    return orc.run(sp["dims"], flags, sp["omega"], orc.omega_minus(sp["omega"], LAM), sp["force"], f0, steps)


@pytest.mark.parametrize("prec", [0, 3])
@pytest.mark.parametrize("prop", [0, 1])
@pytest.mark.parametrize("tuning", [(128, 1, 0), (256, 2, 2), (64, 8, 1), (512, 4, 8)])
def test_batch_f64_matches_oracle(lbm, orc, prec, prop, tuning):
    specs = small_batch()
    for steps in (3, 8):
        got, flags = run_batch(lbm, specs, prec, prop, steps, tuning)
        for k, sp in enumerate(specs):
            if sp["kind"] == "porous":
                assert np.array_equal(flags[k], orc.voxelize_spheres(sp["dims"], sp["spheres"], 2))
            ref = oracle_run(orc, sp, flags[k], k, steps)
            assert np.abs(got[k] - ref).max() <= 1e-12, (k, sp["kind"], steps)


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_batch_equals_one_at_a_time_bitwise(lbm, prec):
    specs = small_batch(seed=8, count=7)
    a, _ = run_batch(lbm, specs, prec, 1, 9, (192, 4, 2), batch=True)
    b, _ = run_batch(lbm, specs, prec, 1, 9, None, batch=False)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_autotune_leaves_state_untouched(lbm):
    import torch
    specs = small_batch(seed=9, count=6)
    s = torch.cuda.current_stream()
    descs = [lbm.make_desc(sp["dims"], 1, lbm.LBM_DIRECT if sp["kind"] == "channel" else lbm.LBM_INDIRECT, 1,
                           sp["periodic"]) for sp in specs]
    h = lbm.lbm_create_batch(descs, s)
    try:
        for k, sp in enumerate(specs):
            if sp["kind"] == "channel":
                lbm.lbm_set_geometry(h, k, sp["flags"])
            else:
                lbm.lbm_set_geometry_spheres(h, k, sp["spheres"])
            lbm.lbm_set_params(h, k, sp["omega"], LAM, sp["force"])
            lbm.lbm_init_equilibrium(h, k)
        lbm.lbm_step(h, 5)
        before = [lbm.lbm_read_pdfs(h, k) for k in range(len(specs))]
        lbm.lbm_autotune(h, 4)
        assert lbm.lbm_steps_done(h) == 5
        after = [lbm.lbm_read_pdfs(h, k) for k in range(len(specs))]
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        t = lbm.lbm_get_tuning(h)
        assert t[0] in (128, 256, 512) and t[1] in (1, 2, 4, 8) and t[2] in (0, 2, 4, 8)
        lbm.lbm_step(h, 3)
    finally:
        lbm.lbm_destroy(h)


def test_autotune_cache_reuses_the_choice_for_the_same_signature(lbm):
    """A second handle with the same signature takes the cached shape without
    trials; another signature is tuned afresh."""
    import torch
    lbm.lbm_autotune_clear()
    fl = inputs.duct_flags(48, 24, 24)

    def make(dims, flags):
        h = lbm.lbm_create_lattice(lbm.make_desc(dims, lbm.LBM_F32_SHIFTED, 0, 1, (1, 0, 0)),
                                   torch.cuda.current_stream())
        lbm.lbm_set_geometry(h, 0, flags)
        lbm.lbm_set_params(h, 0, 1.0, 3 / 16, (0, 0, 0))
        lbm.lbm_init_equilibrium(h, 0)
        return h

    a, b = make((48, 24, 24), fl), make((48, 24, 24), fl)
    c = make((40, 24, 24), inputs.duct_flags(40, 24, 24))
    try:
        lbm.lbm_autotune(a, 4)
        e0, h0 = lbm.lbm_autotune_cache()
        assert e0 == 1
        lbm.lbm_set_tuning(b, 64, 1, 0)
        lbm.lbm_autotune(b, 4)
        e1, h1 = lbm.lbm_autotune_cache()
        assert (e1, h1) == (1, h0 + 1)
        assert lbm.lbm_get_tuning(b) == lbm.lbm_get_tuning(a)
        lbm.lbm_autotune(c, 4)
        e2, h2 = lbm.lbm_autotune_cache()
        assert (e2, h2) == (2, h1)
    finally:
        for h in (a, b, c):
            lbm.lbm_destroy(h)

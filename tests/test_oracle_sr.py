"""Pins of the oracle's FP16 stochastic-rounding format: the counter-based
generator against its published outputs and an independent implementation,
the rounding rule against numpy's FP16 grid and its exact mean, and the step
against the FP64 step it rounds. No GPU."""
import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs


def fp16_neighbours(x):
    """The FP16 values bracketing x (lo <= x <= hi), from numpy's FP16 grid."""
    x = np.asarray(x, dtype=np.float64)
    c = x.astype(np.float16)
    c64 = c.astype(np.float64)
    lo = np.where(c64 > x, np.nextafter(c, np.float16(-np.inf)), c)
    hi = np.where(c64 < x, np.nextafter(c, np.float16(np.inf)), c)
    return lo.astype(np.float64), hi.astype(np.float64)


def random_magnitudes(rng, n, lo_exp=-30, hi_exp=15):
    return np.exp2(rng.uniform(lo_exp, hi_exp, n)) * rng.choice([-1.0, 1.0], n)


# ------------------------------------------------------------- generator
def test_splitmix64_published_outputs(orc):
    """splitmix64 seeded with 0: the first outputs of its published reference
    implementation."""
    assert [hex(orc.splitmix64(0, k)) for k in range(3)] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4",
                                                             "0x6c45d188009454f"]


def test_splitmix64_matches_independent_numpy(orc):
    rng = np.random.default_rng(7)
    seeds = rng.integers(0, 2 ** 63, 20, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    for s in seeds:
        ks = rng.integers(0, 2 ** 62, 8, dtype=np.uint64)
        want = inputs.splitmix64(ks, int(s))
        got = [orc.splitmix64(int(s), int(k)) for k in ks]
        assert [int(v) for v in want] == got


def test_sr_bits_layout(orc):
    """Direction j of node n at sweep t: bits 16 (j mod 4) of word j div 4, where
    word 0 is the node's key and words 1..4 continue the stream the key seeds."""
    rng = np.random.default_rng(11)
    for _ in range(40):
        seed = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        t = int(rng.integers(0, 2 ** 31))
        node = int(rng.integers(0, 2 ** 31))
        key = int(inputs.splitmix64(np.array([(t << 32) | node], dtype=np.uint64), seed)[0])
        words = [key] + [int(v) for v in inputs.splitmix64(np.arange(4, dtype=np.uint64), key)]
        for j in range(19):
            assert orc.sr_bits(seed, t, node, j) == (words[j // 4] >> (16 * (j % 4))) & 0xFFFF


def test_sr_bits_statistics(orc):
    """The draws are uniform on 0..65535 and differ between nodes, directions and sweeps."""
    vals = np.array([orc.sr_bits(5, t, n, j) for t in range(3) for n in range(60) for j in range(19)],
                    dtype=np.float64)
    assert vals.min() >= 0 and vals.max() <= 65535
    assert abs(vals.mean() / 65536 - 0.5) < 0.02
    assert abs(vals.std() / 65536 - np.sqrt(1 / 12)) < 0.02
    assert len(np.unique(vals)) > 0.95 * len(vals)
    assert orc.sr_bits(5, 0, 0, 0) != orc.sr_bits(6, 0, 0, 0)


# ---------------------------------------------------------- rounding rule
def test_round_half_gives_a_neighbour(orc):
    rng = np.random.default_rng(3)
    x = random_magnitudes(rng, 20000)
    r = rng.integers(0, 65536, x.size)
    got, margin = orc.round_half_stochastic(x, r)
    lo, hi = fp16_neighbours(x)
    inside = (np.abs(x) < 65504)
    assert np.all((got[inside] == lo[inside]) | (got[inside] == hi[inside]))
    # the decision: away from zero iff q + r/2^16 >= 1, q the position of |x| between its neighbours
    a_lo = np.minimum(np.abs(lo), np.abs(hi))
    a_hi = np.maximum(np.abs(lo), np.abs(hi))
    q = (np.abs(x) - a_lo) / (a_hi - a_lo)
    away = np.abs(got) == a_hi
    sel = inside & (a_hi > a_lo)
    assert np.array_equal(away[sel], (q + r / 65536.0 >= 1.0)[sel])
    assert np.allclose(margin[sel], np.abs(q + r / 65536.0 - 1.0)[sel], rtol=0, atol=1e-12)


def test_round_half_fixed_points(orc):
    """Every finite FP16 value is returned unchanged, whatever the draw."""
    h = np.arange(65536, dtype=np.uint32).astype(np.uint16).view(np.float16)
    h = h[np.isfinite(h)].astype(np.float64)
    r = np.random.default_rng(0).integers(0, 65536, h.size)
    got, margin = orc.round_half_stochastic(h, r)
    assert np.array_equal(got, h)
    assert np.all(np.isinf(margin))


def test_round_half_mean_over_all_draws_is_x(orc):
    """Averaged over all 2^16 draws the rounding returns x to within one
    2^16-th of the FP16 spacing: the rounding is unbiased."""
    rng = np.random.default_rng(5)
    r = np.arange(65536, dtype=np.uint32)
    for x in list(random_magnitudes(rng, 12)) + [1.0 / 3.0, -2.0 ** -20 * 1.37, 5e-8, 1e-4 + 1e-9]:
        got, _ = orc.round_half_stochastic(np.full(r.size, x), r)
        lo, hi = fp16_neighbours(np.array([x]))
        u = abs(hi[0] - lo[0])
        assert abs(got.mean() - x) <= u / 65536 + 1e-300, x


def test_round_half_odd_symmetry_and_subnormals(orc):
    rng = np.random.default_rng(9)
    x = random_magnitudes(rng, 5000, lo_exp=-40, hi_exp=-13)
    r = rng.integers(0, 65536, x.size)
    a, _ = orc.round_half_stochastic(x, r)
    b, _ = orc.round_half_stochastic(-x, r)
    assert np.array_equal(a, -b)
    sub = np.abs(x) < 2.0 ** -14
    # FP16 subnormal range: results are whole multiples of 2^-24
    k = a[sub] / 2.0 ** -24
    assert np.array_equal(k, np.round(k))
    # below 2^-24 the result is 0 or +-2^-24 with probability |x| / 2^-24
    tiny = np.full(65536, 0.25 * 2.0 ** -24)
    got, _ = orc.round_half_stochastic(tiny, np.arange(65536, dtype=np.uint32))
    assert set(np.unique(got)) == {0.0, 2.0 ** -24}
    assert (got > 0).sum() == 16384


def test_round_half_saturation_and_specials(orc):
    got, _ = orc.round_half_stochastic([70000.0, -1e9, 65519.0, 65503.9], [65535, 65535, 65535, 65535])
    assert list(got) == [65504.0, -65504.0, 65504.0, 65504.0]
    got, _ = orc.round_half_stochastic([np.inf, -np.inf, np.nan], [0, 0, 0])
    assert got[0] == np.inf and got[1] == -np.inf and np.isnan(got[2])


# ------------------------------------------------------------------ step
def fp16_state(orc, dims, flags, seed, amp=0.02):
    """A seeded FP16-grid deviation state: the equilibrium of a random velocity
    field (density 1 +- 1 %), deviations from w rounded to FP16 by numpy."""
    nx, ny, nz = dims
    u = inputs.velocity_perturbation(nx, ny, nz, seed=seed, amplitude=amp, flags=flags)
    rho = 1.0 + 0.01 * inputs.uniform_pm1(np.arange(nx * ny * nz, dtype=np.uint64), seed + 1000)
    f = orc.init_equilibrium(dims, flags, rho, u)
    w = orc.weights()[:, None]
    d = (f - w).astype(np.float16).astype(np.float64)
    d[:, flags == 2] = 0.0
    return d


def mixed_flags(dims, seed):
    rng = np.random.default_rng(seed)
    fl = rng.choice(np.array([0, 0, 0, 0, 0, 1, 2], dtype=np.uint8), size=int(np.prod(dims)))
    return fl


@pytest.mark.parametrize("seed", [1, 2])
def test_step_f16_stochastic_rounds_the_fp64_step(orc, seed):
    dims = (6, 5, 4)
    fl = mixed_flags(dims, seed)
    d = fp16_state(orc, dims, fl, seed)
    w = orc.weights()[:, None]
    om, lam, F = 1.3, 0.21, (2e-4, -1e-4, 3e-5)
    wm = orc.omega_minus(om, lam)
    ref = orc.step(dims, fl, om, wm, F, (w + d) * (fl != 2))
    x = ref - w
    got, margin = orc.step_f16_stochastic(dims, fl, om, wm, F, d, seed=0xDEADBEEF + seed, t=77)
    rounded = np.isfinite(margin)
    lo, hi = fp16_neighbours(x)
    assert np.all((got[rounded] == lo[rounded]) | (got[rounded] == hi[rounded]))
    # slots filled by a full-way solid are its own reversed values, untouched
    c = orc.velocities()
    opp = [orc.opposite(i) for i in range(19)]
    nx, ny, nz = dims
    for n in np.flatnonzero(fl == 1):
        x0, y0, z0 = n % nx, (n // nx) % ny, n // (nx * ny)
        for i in range(19):
            m = (x0 + c[i, 0]) % nx + nx * ((y0 + c[i, 1]) % ny + ny * ((z0 + c[i, 2]) % nz))
            slot = (opp[i], n) if fl[m] == 2 else (i, m)
            assert got[slot] == d[opp[i], n]
            assert np.isinf(margin[slot])
    assert np.all(got[:, fl == 2] == 0)
    # a fluid node's slots are all rounded (an FP16-exact value counts as rounded with an infinite margin)
    assert rounded.sum() > 0.5 * rounded.size
    # another sweep counter draws other bits
    got2, _ = orc.step_f16_stochastic(dims, fl, om, wm, F, d, seed=0xDEADBEEF + seed, t=78)
    assert (got2 != got).sum() > 0.1 * rounded.sum()


def test_step_f16_stochastic_is_unbiased(orc):
    """Over many seeds the mean of each stored deviation converges to the FP64
    step's value, and the totals (mass, momentum) with it."""
    dims = (4, 4, 4)
    fl = mixed_flags(dims, 3)
    fl[fl == 1] = 0
    d = fp16_state(orc, dims, fl, 4)
    w = orc.weights()[:, None]
    om, wm, F = 1.0, orc.omega_minus(1.0, 3 / 16), (1e-5, 0.0, 0.0)
    x = orc.step(dims, fl, om, wm, F, (w + d) * (fl != 2)) - w
    x[:, fl == 2] = 0.0   # half-way solid cells hold nothing
    S = 400
    runs = np.stack([orc.step_f16_stochastic(dims, fl, om, wm, F, d, seed=s, t=3)[0] for s in range(S)])
    lo, hi = fp16_neighbours(x)
    u = hi - lo
    # per slot: the sample mean of a two-point variable lies within 5 sigma of x
    sigma = 0.5 * u / np.sqrt(S)
    assert np.all(np.abs(runs.mean(0) - x) <= 5 * sigma + 1e-300)
    # mass: the seed-averaged total against the FP64 total
    tot = runs.sum(axis=(1, 2))
    assert abs(tot.mean() - x.sum()) <= 5 * tot.std() / np.sqrt(S) + 1e-18
    # per-seed totals do differ (the draws are live)
    assert tot.std() > 0


def test_step_f16_stochastic_node_numbering(orc):
    dims = (5, 4, 3)
    fl = np.zeros(60, dtype=np.uint8)
    fl[[3, 17, 40]] = 2
    d = fp16_state(orc, dims, fl, 8)
    cell_of, list_index, _ = orc.build_list(dims, fl)
    om, wm, F = 0.8, orc.omega_minus(0.8, 0.25), (0.0, 1e-5, 0.0)
    seed, t = 123, 2 ** 33 + 5
    a, _ = orc.step_f16_stochastic(dims, fl, om, wm, F, d, seed=seed, t=t, node_of=list_index)
    # node k = list_index[n] draws orc_sr_bits(seed, t, k, j): check the rest slot of a few cells
    w = orc.weights()
    for n in (0, 21, 59):
        k = int(list_index[n])
        f = w + d[:, n]
        fs = orc.collide_trt(f, om, wm, F)
        want, _ = orc.round_half_stochastic(fs[0] - w[0], orc.sr_bits(seed, t, k, 0))
        assert a[0, n] == want[()]
    b, _ = orc.step_f16_stochastic(dims, fl, om, wm, F, d, seed=seed, t=t)
    assert not np.array_equal(a, b)

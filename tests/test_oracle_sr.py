"""Pins of the oracle's scaled FP16 stochastic-rounding format: the
counter-based generator against its published outputs and an independent
implementation; the rounding rule against numpy's FP16 grid (every result is a
neighbour of x), against monotonicity in the draw and against the exact number
of draws that round away from zero -- three properties that together fix the
rule in every binade, FP16 subnormals included; and the step against the FP64
step it rounds. No GPU."""
import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs

SCALE = 2.0 ** 14   # the format stores d * 2^14


def fp16_neighbours(x):
    """The FP16 values bracketing x (lo <= x <= hi), from numpy's FP16 grid."""
    x = np.asarray(x, dtype=np.float64)
    c = x.astype(np.float16)
    c64 = c.astype(np.float64)
    lo = np.where(c64 > x, np.nextafter(c, np.float16(-np.inf)), c)
    hi = np.where(c64 < x, np.nextafter(c, np.float16(np.inf)), c)
    return lo.astype(np.float64), hi.astype(np.float64)


def scaled_neighbours(d):
    """Neighbours of deviations d on the format's grid (FP16 values times 2^-14)."""
    lo, hi = fp16_neighbours(np.asarray(d, dtype=np.float64) * SCALE)
    return lo / SCALE, hi / SCALE


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
    """Direction j of node n at sweep t: the 32-bit half (j mod 4) div 2 of word
    j div 4, bits 0..12 for even j and 19..31 for odd j, where word 0 is the
    node's key and words 1..4 continue the stream the key seeds."""
    rng = np.random.default_rng(11)
    for _ in range(40):
        seed = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        t = int(rng.integers(0, 2 ** 31))
        node = int(rng.integers(0, 2 ** 31))
        key = int(inputs.splitmix64(np.array([(t << 32) | node], dtype=np.uint64), seed)[0])
        words = [key] + [int(v) for v in inputs.splitmix64(np.arange(4, dtype=np.uint64), key)]
        for j in range(19):
            half = (words[j // 4] >> (32 * ((j % 4) // 2))) & 0xFFFFFFFF
            want = half & 0x1FFF if j % 2 == 0 else half >> 19
            assert orc.sr_bits(seed, t, node, j) == want


def test_sr_bits_statistics(orc):
    """The draws are uniform on 0..8191 and differ between nodes, directions and sweeps."""
    vals = np.array([orc.sr_bits(5, t, n, j) for t in range(3) for n in range(80) for j in range(19)],
                    dtype=np.float64)
    assert vals.min() >= 0 and vals.max() <= 8191
    assert abs(vals.mean() / 8192 - 0.5) < 0.02
    assert abs(vals.std() / 8192 - np.sqrt(1 / 12)) < 0.02
    counts = np.bincount((vals // 512).astype(int), minlength=16)
    expect = vals.size / 16
    assert ((counts - expect) ** 2 / expect).sum() < 40   # chi-square, 15 degrees of freedom
    assert [orc.sr_bits(5, 0, 0, j) for j in range(19)] != [orc.sr_bits(6, 0, 0, j) for j in range(19)]


# ---------------------------------------------------------- rounding rule
def exact_ups(x):
    """Number of the 2^13 draws that must round x away from zero for the mean
    over all draws to be x truncated to the grid of u / 2^13, u the spacing of
    numpy's FP16 grid at x: floor(2^13 (|x| - lo) / u), in exact rational
    arithmetic."""
    from fractions import Fraction
    lo, hi = fp16_neighbours(np.array([x]))
    a_lo, a_hi = sorted((abs(lo[0]), abs(hi[0])))
    if a_hi == a_lo:
        return 0, a_lo, a_hi
    q = (Fraction(abs(float(x))) - Fraction(a_lo)) / (Fraction(a_hi) - Fraction(a_lo))
    return int(q * 8192), a_lo, a_hi   # int() of a non-negative Fraction is its floor


def test_round_half_gives_a_neighbour(orc):
    rng = np.random.default_rng(3)
    x = random_magnitudes(rng, 20000, lo_exp=-45, hi_exp=15)
    r = rng.integers(0, 8192, x.size)
    got, margin = orc.round_half_stochastic(x, r)
    lo, hi = fp16_neighbours(x)
    inside = np.abs(x) < 65504
    assert np.all((got[inside] == lo[inside]) | (got[inside] == hi[inside]))
    assert np.all(np.sign(got[got != 0]) == np.sign(x[got != 0]))
    # the margin is the decision's distance from its threshold in spacings: never
    # more than one spacing
    assert np.all(margin[inside & np.isfinite(margin)] <= 1.0)


def binades():
    """Magnitudes that span FP16's normal binades and its subnormal range, down
    to below the smallest subnormal (2^-24), as FP64 and as FP32 values."""
    rng = np.random.default_rng(5)
    xs = list(random_magnitudes(rng, 16, lo_exp=-14, hi_exp=15))
    xs += list(random_magnitudes(rng, 16, lo_exp=-24, hi_exp=-14))     # FP16 subnormals
    xs += list(random_magnitudes(rng, 6, lo_exp=-38, hi_exp=-24))      # below 2^-24
    xs += [1.0 / 3.0, 1e-4 + 1e-9, (600 + 0.75) * 2.0 ** -24, 0.75 * 2.0 ** -24, 2.0 ** -14 - 2.0 ** -40,
           -(3 + 2.0 ** -12) * 2.0 ** -24, 2.0 ** -37, 2.0 ** -37 * 0.999]
    xs += list(np.asarray(xs, dtype=np.float32).astype(np.float64))
    return xs


@pytest.mark.parametrize("x", binades())
def test_round_half_over_all_draws(orc, x):
    """Over all 2^13 draws: the result is monotone in the draw (a threshold
    rule), and x rounds away from zero for exactly floor(2^13 q) draws, q the
    remainder in spacings -- so the mean over the draws is x truncated to the
    grid of u / 2^13 and x itself when x has no bits below that grid (every
    FP32 value in FP16's normal range). Neighbours, monotonicity and this count
    determine the rule completely; a rule that leans towards zero anywhere,
    the subnormal range included, fails the count."""
    from fractions import Fraction
    r = np.arange(8192, dtype=np.uint32)
    got, _ = orc.round_half_stochastic(np.full(r.size, x), r)
    want_ups, a_lo, a_hi = exact_ups(x)
    if a_hi == a_lo:   # an FP16 value: returned unchanged by every draw
        assert np.all(got == x)
        return
    a = np.abs(got)
    assert np.all((a == a_lo) | (a == a_hi))
    away = a == a_hi
    assert np.all(np.diff(away.astype(int)) >= 0)          # monotone: away for r >= r*
    assert int(away.sum()) == want_ups
    mean = sum(Fraction(float(v)) for v in got) / 8192
    trunc = Fraction(a_lo) + Fraction(a_hi - a_lo) * Fraction(want_ups, 8192)
    assert abs(mean) == trunc
    assert 0 <= Fraction(abs(float(x))) - trunc < Fraction(a_hi - a_lo) / 8192
    if float(np.float32(x)) == x and abs(x) >= 2.0 ** -14:
        assert abs(mean) == Fraction(abs(float(x)))            # unbiased, exactly


def test_round_half_subnormal_band_is_unbiased(orc):
    """Below 2^-14 (FP16 subnormals, spacing 2^-24): a value 3/4 of the way to
    the next grid point rounds up for 3/4 of the draws, as in every other
    binade, and a value below the smallest subnormal rounds up to it with the
    probability of its size in spacings."""
    r = np.arange(8192, dtype=np.uint32)
    for k, frac, ups in ((600, 0.75, 6144), (0, 0.75, 6144), (3, 0.5, 4096), (1023, 0.125, 1024),
                         (0, 2.0 ** -13, 1), (0, 2.0 ** -13 * 0.999, 0)):
        x0 = (k + frac) * 2.0 ** -24
        got, _ = orc.round_half_stochastic(np.full(8192, x0), r)
        assert (got > k * 2.0 ** -24).sum() == ups, (k, frac)
        got, _ = orc.round_half_stochastic(np.full(8192, -x0), r)
        assert (got < -k * 2.0 ** -24).sum() == ups, (k, frac)


def test_round_half_fixed_points(orc):
    """Every finite FP16 value is returned unchanged, whatever the draw."""
    h = np.arange(65536, dtype=np.uint32).astype(np.uint16).view(np.float16)
    h = h[np.isfinite(h)].astype(np.float64)
    r = np.random.default_rng(0).integers(0, 8192, h.size)
    got, margin = orc.round_half_stochastic(h, r)
    assert np.array_equal(got, h)
    assert np.all(np.isinf(margin))


def test_round_half_odd_symmetry_and_subnormals(orc):
    rng = np.random.default_rng(9)
    x = random_magnitudes(rng, 5000, lo_exp=-40, hi_exp=-13)
    r = rng.integers(0, 8192, x.size)
    a, _ = orc.round_half_stochastic(x, r)
    b, _ = orc.round_half_stochastic(-x, r)
    assert np.array_equal(a, -b)
    sub = np.abs(x) < 2.0 ** -14
    k = a[sub] / 2.0 ** -24   # FP16 subnormal range: whole multiples of 2^-24
    assert np.array_equal(k, np.round(k))


def test_round_half_saturation_and_specials(orc):
    got, _ = orc.round_half_stochastic([70000.0, -1e9, 65519.0, 65503.9], [8191, 8191, 8191, 8191])
    assert list(got) == [65504.0, -65504.0, 65504.0, 65504.0]
    got, _ = orc.round_half_stochastic([np.inf, -np.inf, np.nan], [0, 0, 0])
    assert got[0] == np.inf and got[1] == -np.inf and np.isnan(got[2])


# ------------------------------------------------------------------ step
def fp16_state(orc, dims, flags, seed, amp=0.02):
    """A seeded state on the format's grid: the equilibrium of a random velocity
    field (density 1 +- 1 %), deviations from w scaled by 2^14 and rounded to
    FP16 by numpy."""
    nx, ny, nz = dims
    u = inputs.velocity_perturbation(nx, ny, nz, seed=seed, amplitude=amp, flags=flags)
    rho = 1.0 + 0.01 * inputs.uniform_pm1(np.arange(nx * ny * nz, dtype=np.uint64), seed + 1000)
    f = orc.init_equilibrium(dims, flags, rho, u)
    w = orc.weights()[:, None]
    d = ((f - w) * SCALE).astype(np.float16).astype(np.float64) / SCALE
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
    lo, hi = scaled_neighbours(x)
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
    lo, hi = scaled_neighbours(x)
    u = hi - lo
    sigma = 0.5 * u / np.sqrt(S)   # per slot: the sample mean of a two-point variable
    assert np.all(np.abs(runs.mean(0) - x) <= 5 * sigma + u / 8192 + 1e-300)
    tot = runs.sum(axis=(1, 2))
    assert abs(tot.mean() - x.sum()) <= 5 * tot.std() / np.sqrt(S) + 1e-18
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
        fs = orc.collide_trt(w + d[:, n], om, wm, F)
        want, _ = orc.round_half_stochastic((fs[0] - w[0]) * SCALE, orc.sr_bits(seed, t, k, 0))
        assert a[0, n] == want[()] / SCALE
    b, _ = orc.step_f16_stochastic(dims, fl, om, wm, F, d, seed=seed, t=t)
    assert not np.array_equal(a, b)

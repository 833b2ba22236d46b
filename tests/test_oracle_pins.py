"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an
invariant, a special case, the paper's own verification set-up (Sec. 2.1,
Poiseuille flow between two slabs driven by a body force), or an independently
written implementation (``reference_numpy``) on tiny lattices.
"""
import itertools

import numpy as np
import pytest

import reference_numpy as ref
from paper_1711_11468_gb300 import inputs

LAM = 3.0 / 16.0


def _rand_state(orc, dims, flags, rng, du=0.05, drho=0.05):
    N = int(np.prod(dims))
    rho = 1.0 + drho * (rng.random(N) - 0.5)
    u = du * (rng.random((3, N)) - 0.5)
    f = orc.init_equilibrium(dims, flags, rho, u)
    # add a non-equilibrium part so the collision has something to relax
    noise = 1e-3 * (rng.random(f.shape) - 0.5)
    noise[:, flags == 2] = 0.0
    return f + noise


# ---------------------------------------------------------------- lattice
def test_velocity_set_is_d3q19(orc):
    c = orc.velocities()
    assert c.shape == (19, 3)
    assert len({tuple(v) for v in c}) == 19
    assert set(map(tuple, c)) == {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in v) <= 2}
    for i in range(19):
        assert (c[orc.opposite(i)] == -c[i]).all()


def test_weights_isotropy(orc):
    """Sum w = 1, sum w c_a = 0, sum w c_a c_b = d_ab / 3, 3rd moments 0,
    sum w c_a c_b c_c c_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc) / 9."""
    c = orc.velocities().astype(float)
    w = orc.weights()
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("q,qa->a", w, c)).max() < 1e-16
    assert np.abs(np.einsum("q,qa,qb->ab", w, c, c) - d / 3).max() < 1e-16
    assert np.abs(np.einsum("q,qa,qb,qc->abc", w, c, c, c)).max() < 1e-16
    m4 = np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.abs(m4 - iso).max() < 1e-16
    # the same weights fall out of the isotropy conditions solved independently
    wr = ref.to_reference_order(w, orc.velocities())
    assert np.abs(wr - ref.W).max() < 4e-16


def test_omega_minus_from_lambda(orc):
    for wp in (0.6, 1.0, 1.6, 1.9):
        for lam in (1 / 12, 3 / 16, 1 / 4, 1 / 2):
            wm = orc.omega_minus(wp, lam)
            assert abs((1 / wp - 0.5) * (1 / wm - 0.5) - lam) < 1e-14
    assert abs(orc.omega_minus(1.0, 3 / 16) - 8 / 7) < 1e-15
    assert abs(orc.omega_minus(1.0, 1 / 4) - 1.0) < 1e-15


# ------------------------------------------------------------ equilibrium
@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (1.03, (0.02, -0.01, 0.005)),
                                   (0.97, (-0.05, 0.04, 0.03))])
def test_equilibrium_moments(orc, rho, u):
    """Closed-form moments: rho, rho u, rho (u u + I/3)."""
    e = orc.equilibrium(rho, u)
    c = orc.velocities().astype(float)
    u = np.array(u)
    assert abs(e.sum() - rho) < 1e-15
    assert np.abs(c.T @ e - rho * u).max() < 1e-16
    assert np.abs(np.einsum("qa,qb,q->ab", c, c, e) - rho * (np.outer(u, u) + np.eye(3) / 3)).max() < 1e-15


def test_equilibrium_at_rest_is_weights(orc):
    assert np.array_equal(orc.equilibrium(1.0, (0, 0, 0)), orc.weights())


# --------------------------------------------------------------- collision
def test_collision_conserves_mass_and_adds_force(orc):
    rng = np.random.default_rng(1)
    c = orc.velocities().astype(float)
    for _ in range(20):
        f = orc.weights() * (1 + 0.1 * (rng.random(19) - 0.5))
        wp = rng.uniform(0.5, 1.9)
        wm = orc.omega_minus(wp, rng.uniform(0.05, 0.5))
        F = 1e-3 * (rng.random(3) - 0.5)
        fs = orc.collide_trt(f, wp, wm, F)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert np.abs(c.T @ fs - (c.T @ f + F)).max() < 1e-15


def test_collision_bgk_unit_relaxation(orc):
    """omega+ = omega- = 1 (Lambda = 1/4 at omega = 1): the TRT post-collision state
    is the equilibrium of the pre-collision moments plus the source (BGK, tau = 1)."""
    rng = np.random.default_rng(2)
    c = orc.velocities().astype(float)
    for _ in range(10):
        f = orc.weights() * (1 + 0.1 * (rng.random(19) - 0.5))
        F = 1e-4 * (rng.random(3) - 0.5)
        fs = orc.collide_trt(f, 1.0, orc.omega_minus(1.0, 0.25), F)
        rho = f.sum()
        u = c.T @ f / rho
        expect = ref.equilibrium(np.array(rho), u) + ref.W * (ref.C @ F) * 3
        assert np.abs(ref.to_reference_order(fs, orc.velocities()) - expect).max() < 1e-15


def test_collision_matches_independent_trt(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        f = orc.weights() * (1 + 0.2 * (rng.random(19) - 0.5))
        wp = rng.uniform(0.5, 1.9)
        wm = orc.omega_minus(wp, rng.uniform(0.05, 0.5))
        F = 1e-3 * (rng.random(3) - 0.5)
        got = ref.to_reference_order(orc.collide_trt(f, wp, wm, F), orc.velocities())
        fr = ref.to_reference_order(f, orc.velocities())
        assert np.abs(got - ref.collide(fr, wp, wm, F)).max() < 1e-15


# --------------------------------------------------------- full time steps
def _geometry_4(rng, dims):
    fl = np.zeros(int(np.prod(dims)), dtype=np.uint8)
    r = rng.random(fl.size)
    fl[r < 0.15] = 1
    fl[(r >= 0.15) & (r < 0.3)] = 2
    return fl


@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 4, 3), (3, 6, 4)])
def test_step_matches_independent_pull(orc, dims):
    """Brute force on tiny lattices: random geometry (both bounce-back kinds),
    random state, random omega, Lambda and force; 6 steps."""
    rng = np.random.default_rng(sum(dims))
    for trial in range(3):
        fl = _geometry_4(rng, dims)
        f = _rand_state(orc, dims, fl, rng)
        wp = rng.uniform(0.6, 1.8)
        wm = orc.omega_minus(wp, rng.uniform(0.05, 0.5))
        F = 1e-4 * (rng.random(3) - 0.5)
        nx, ny, nz = dims
        fr = ref.to_reference_order(f, orc.velocities()).reshape(19, nz, ny, nx)
        flr = fl.reshape(nz, ny, nx)
        for _ in range(6):
            f = orc.step(dims, fl, wp, wm, F, f)
            fr = ref.step_pull(fr, flr, wp, wm, F)
        got = ref.to_reference_order(f, orc.velocities()).reshape(19, nz, ny, nx)
        assert np.abs(got - fr).max() < 1e-15


def test_rest_state_is_invariant(orc):
    dims = (6, 8, 5)
    fl = inputs.channel_flags(*dims)
    fl[7] = 2
    f0 = orc.init_equilibrium(dims, fl)
    w = orc.weights()
    live = fl != 2
    f = f0
    first = None
    for _ in range(10):
        f = orc.run(dims, fl, 1.3, orc.omega_minus(1.3, LAM), (0, 0, 0), f, 50, 1)
        dev = np.abs(f[:, live] - w[:, None]).max()
        # round-off of rho = sum w_i only: a few ulp of 1/3, and it does not grow
        assert dev <= 4 * np.spacing(1.0 / 3.0)
        first = dev if first is None else first
        assert dev <= first
        assert np.all(f[:, ~live] == 0.0)


def test_mass_conservation(orc):
    rng = np.random.default_rng(5)
    dims = (9, 8, 7)
    fl = _geometry_4(rng, dims)
    f = _rand_state(orc, dims, fl, rng)
    m0 = f.sum()
    f = orc.run(dims, fl, 1.7, orc.omega_minus(1.7, LAM), (1e-4, -2e-5, 3e-5), f, 300, 1)
    assert abs(f.sum() - m0) / m0 < 1e-13


def test_momentum_grows_by_force(orc):
    """Fully periodic, wall-free box: total momentum grows by N*F every step."""
    rng = np.random.default_rng(6)
    dims = (6, 5, 4)
    N = 120
    fl = np.zeros(N, dtype=np.uint8)
    f = _rand_state(orc, dims, fl, rng)
    c = orc.velocities().astype(float)
    F = np.array([1e-5, 2e-5, -1e-5])
    j0 = c.T @ f.sum(1)
    wp = 1.2
    wm = orc.omega_minus(wp, LAM)
    for t in range(1, 41):
        f = orc.step(dims, fl, wp, wm, F, f)
        j = c.T @ f.sum(1)
        assert np.abs(j - j0 - t * N * F).max() < 1e-13
    f0 = _rand_state(orc, dims, fl, rng)
    f = orc.run(dims, fl, wp, wm, (0, 0, 0), f0, 40, 1)
    assert np.abs(c.T @ f.sum(1) - c.T @ f0.sum(1)).max() < 1e-14


@pytest.mark.parametrize("omega", [0.8, 1.0, 1.6])
def test_shear_wave_decay(orc, omega):
    """u_x = U sin(2 pi y / ny) decays as exp(-nu k^2 t), nu = (1/omega - 1/2)/3."""
    ny = 64
    dims = (2, ny, 2)
    N = 2 * ny * 2
    fl = np.zeros(N, dtype=np.uint8)
    y = np.tile(np.repeat(np.arange(ny), 2), 2)
    u = np.zeros((3, N))
    u[0] = 1e-4 * np.sin(2 * np.pi * y / ny)
    f = orc.init_equilibrium(dims, fl, None, u)
    wm = orc.omega_minus(omega, LAM)
    k = 2 * np.pi / ny
    nu = (1 / omega - 0.5) / 3

    def amp(f):
        _, uu = orc.macroscopic(dims, fl, (0, 0, 0), f)
        return 2 * np.mean(uu[0] * np.sin(2 * np.pi * y / ny))

    f = orc.run(dims, fl, omega, wm, (0, 0, 0), f, 100, 1)
    a1 = amp(f)
    f = orc.run(dims, fl, omega, wm, (0, 0, 0), f, 400, 1)
    a2 = amp(f)
    rate = -np.log(a2 / a1) / 400
    # lattice correction is O(k^2) = 1e-2 relative
    assert abs(rate / (nu * k * k) - 1) < 2e-2


def _column_profile(orc, ny, omega, lam, steps, F, halfway=False):
    dims = (2, ny, 2)
    fl = inputs.channel_flags(*dims)
    if halfway:
        fl[fl == 1] = 2
    f = orc.run(dims, fl, omega, orc.omega_minus(omega, lam), (F, 0, 0),
                orc.init_equilibrium(dims, fl), steps, 1)
    _, u = orc.macroscopic(dims, fl, (F, 0, 0), f)
    return u[0].reshape(2, ny, 2)[0, :, 0], fl


@pytest.mark.parametrize("halfway", [False, True])
@pytest.mark.parametrize("omega", [1.0, 1.6])
@pytest.mark.parametrize("lam", [1 / 12, 3 / 16, 1 / 4, 1 / 2])
def test_steady_poiseuille_and_lambda_law(orc, halfway, omega, lam):
    """Steady body-force-driven channel (Sec. 2.1). Walls sit mid-link at
    y = 1/2 and ny - 3/2; the TRT profile is the parabola
    F/(2 nu) [(y-a)(b-y) + (16 Lambda - 3)/12], exact at Lambda = 3/16."""
    ny, F = 10, 1e-4
    ux, _ = _column_profile(orc, ny, omega, lam, 4000, F, halfway)
    nu = (1 / omega - 0.5) / 3
    y = np.arange(ny)
    a, b = 0.5, ny - 1.5
    ana = F / (2 * nu) * ((y - a) * (b - y) + (16 * lam - 3) / 12)
    m = slice(1, ny - 1)
    assert np.abs(ux[m] - ana[m]).max() / np.abs(ana[m]).max() < 1e-10
    assert np.all(ux[[0, ny - 1]] == 0.0)


def _series(y, t, F, nu, a, b, nterms=4001):
    L = b - a
    s = F / (2 * nu) * (y - a) * (b - y)
    for n in range(1, nterms, 2):
        s = s - 4 * F * L * L / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * (y - a) / L) \
            * np.exp(-nu * n * n * np.pi ** 2 * t / L ** 2)
    return s


def test_transient_startup_series(orc):
    """The 64^3 verification channel after 100 steps follows the start-up series
    of plane Poiseuille flow evaluated at t + 1/2 (column run, see x,z invariance)."""
    ny, F = 64, 1e-6
    ux, _ = _column_profile(orc, ny, 1.0, LAM, 100, F)
    y = np.arange(ny)
    m = slice(1, ny - 1)
    ana = _series(y, 100.5, F, 1 / 6, 0.5, ny - 1.5)
    assert np.abs(ux[m] - ana[m]).max() / np.abs(ana[m]).max() < 2e-3
    ana_t = _series(y, 100.0, F, 1 / 6, 0.5, ny - 1.5)
    # t + 1/2 is the better reading by a wide margin
    assert np.abs(ux[m] - ana_t[m]).max() > 3 * np.abs(ux[m] - ana[m]).max()
    # mirror symmetry y <-> ny-1-y
    assert np.abs(ux - ux[::-1]).max() < 1e-15


def test_channel_xz_invariance(orc):
    """A channel run is bitwise independent of x and z, so a 2-wide column
    equals the 3-D lattice."""
    ny, F = 12, 1e-5
    dims3 = (6, ny, 5)
    fl3 = inputs.channel_flags(*dims3)
    wm = orc.omega_minus(1.0, LAM)
    f3 = orc.run(dims3, fl3, 1.0, wm, (F, 0, 0), orc.init_equilibrium(dims3, fl3), 30, 1)
    f3 = f3.reshape(19, 5, ny, 6)
    assert np.all(f3 == f3[:, :1, :, :1])
    ux_col, _ = _column_profile(orc, ny, 1.0, LAM, 30, F)
    _, u3 = orc.macroscopic(dims3, fl3, (F, 0, 0), f3.reshape(19, -1))
    assert np.array_equal(u3[0].reshape(5, ny, 6)[0, :, 0], ux_col)


# ----------------------------------------------------------------- geometry
def _brute_voxelize(dims, spheres):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = np.zeros((nz, ny, nx), dtype=bool)
    for cx, cy, cz, r in spheres:
        dx = np.minimum((x - cx) % nx, (cx - x) % nx)
        dy = np.minimum((y - cy) % ny, (cy - y) % ny)
        dz = np.minimum((z - cz) % nz, (cz - z) % nz)
        inside |= dx * dx + dy * dy + dz * dz <= r * r
    return inside.reshape(-1)


@pytest.mark.parametrize("dims", [(16, 12, 10), (7, 9, 11), (32, 32, 32)])
def test_voxelize_matches_brute_force(orc, dims):
    pack = inputs.sphere_pack(dims, 11, 1, 5, 0.7, nonoverlap_attempts=2000, mc_points=5000)
    fl = orc.voxelize_spheres(dims, pack.spheres, 2)
    assert np.array_equal(fl == 2, _brute_voxelize(dims, pack.spheres))
    # spheres straddling the periodic boundary
    sph = np.array([[0, 0, 0, 3], [dims[0] - 1, 2, dims[2] - 1, 2]], dtype=np.int32)
    assert np.array_equal(orc.voxelize_spheres(dims, sph, 2) == 2, _brute_voxelize(dims, sph))


def test_voxelize_keeps_existing_flags(orc):
    dims = (8, 8, 8)
    fl = inputs.channel_flags(*dims)
    out = orc.voxelize_spheres(dims, np.array([[4, 4, 4, 1]]), 2, fl)
    assert out[4 + 8 * (4 + 8 * 4)] == 2
    assert np.array_equal(out[fl == 1], fl[fl == 1])


@pytest.mark.parametrize("dims", [(6, 5, 4), (8, 8, 8), (3, 7, 2)])
def test_adjacency_brute_force_and_involution(orc, dims):
    rng = np.random.default_rng(len(dims) + dims[0])
    nx, ny, nz = dims
    fl = (rng.random(nx * ny * nz) < 0.3).astype(np.uint8) * 2
    cell_of, list_index, adj = orc.build_list(dims, fl)
    c = orc.velocities()
    fluid = [n for n in range(nx * ny * nz) if fl[n] == 0]
    assert list(cell_of) == fluid                       # lexicographic, x fastest
    pos = {n: k for k, n in enumerate(fluid)}
    for n in range(nx * ny * nz):
        assert list_index[n] == pos.get(n, -1)
    links_to_solid = 0
    for k, n in enumerate(fluid):
        x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
        for i in range(1, 19):
            m = (x - c[i, 0]) % nx + nx * ((y - c[i, 1]) % ny + ny * ((z - c[i, 2]) % nz))
            assert adj[i - 1, k] == pos.get(m, -1)
            links_to_solid += m not in pos
    assert np.count_nonzero(adj == -1) == links_to_solid
    # involution: the upstream node of the upstream node along the opposite direction is the node
    for i in range(1, 19):
        o = orc.opposite(i)
        a = adj[i - 1]
        ok = a >= 0
        assert np.array_equal(adj[o - 1][a[ok]], np.nonzero(ok)[0])


def test_macroscopic_solid_cells_are_zero(orc):
    dims = (4, 6, 4)
    fl = inputs.channel_flags(*dims)
    f = orc.init_equilibrium(dims, fl, None, None)
    rho, u = orc.macroscopic(dims, fl, (1e-3, 0, 0), f)
    assert np.all(rho[fl != 0] == 0) and np.all(u[:, fl != 0] == 0)
    assert np.allclose(rho[fl == 0], 1.0, rtol=0, atol=1e-15)
    assert np.allclose(u[0, fl == 0], 5e-4, rtol=1e-12, atol=0)

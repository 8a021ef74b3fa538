"""Pins for the oracle's collision, noise and streaming (Eqs. 61-69)."""
import numpy as np
import pytest

from oracle import lattice, lbm, philox


def _rand_state(p, seed=0, amp=0.02):
    rng = np.random.default_rng(seed)
    rho = p.rho_c * (1 + amp * rng.standard_normal(p.shape))
    f = lbm.equilibrium_at_rest(rho, p)
    return f + 1e-3 * rng.standard_normal(f.shape) * p.lat.t.reshape(-1, 1, 1, 1)


CASES = [
    dict(lattice="D2Q9", coupling="modeq", nx=7, ny=5, a=0.01, b=0.1, kappa=0.01, kT=1e-4),
    dict(lattice="D2Q9", coupling="guo", nx=6, ny=5, a=0.01, b=0.1, kappa=0.01, kT=1e-4),
    dict(lattice="D3Q19", coupling="guo", nx=4, ny=5, nz=3, a=0.01, b=0.1, kappa=0.01, kT=1e-4),
]


@pytest.mark.parametrize("case", CASES)
def test_mass_conserved_every_step(case):
    p = lbm.Params(**case)
    f = _rand_state(p)
    m0 = f.sum()
    for t in range(20):
        f = lbm.step(f, t, p)
        assert abs(f.sum() - m0) < 1e-13 * m0


def test_modeq_momentum_conserved_every_step():
    """Rows 1-3 of Eq. 68 vanish and f^eq carries rho u exactly (Eq. 62):
    global momentum is conserved by the collision and by periodic streaming."""
    p = lbm.Params(**CASES[0])
    f = _rand_state(p, seed=1)
    j0 = lbm.momentum(f, p.lat).reshape(3, -1).sum(1)
    for t in range(20):
        f = lbm.step(f, t, p)
        j = lbm.momentum(f, p.lat).reshape(3, -1).sum(1)
        assert np.allclose(j, j0, rtol=0, atol=1e-14 * f.sum())


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_guo_momentum_conserved_without_body_force(name):
    """With kappa = 0 the Guo body force vanishes; the Landau pressure rides in the
    equilibrium, which carries rho u exactly, so momentum is conserved."""
    p = lbm.Params(lattice=name, coupling="guo", nx=5, ny=4, nz=3 if name == "D3Q19" else 1,
                   a=0.02, b=0.3, kappa=0.0, kT=1e-4)
    f = _rand_state(p, seed=2)
    j0 = lbm.momentum(f, p.lat).reshape(3, -1).sum(1)
    for t in range(10):
        f = lbm.step(f, t, p)
    j = lbm.momentum(f, p.lat).reshape(3, -1).sum(1)
    assert np.allclose(j, j0, atol=1e-14 * f.sum())


@pytest.mark.parametrize("tau", [1.0, 0.8, 1.7])
def test_equal_rates_reduce_to_literal_bgk(tau):
    """Moment-space relaxation with all tau_a = tau is Eq. 61 in population form."""
    p = lbm.Params(nx=6, ny=5, a=0.02, b=0.2, kappa=0.03, kT=0.0, tau=tuple([tau] * 9))
    lat = p.lat
    f = _rand_state(p, seed=3)
    rho = f.sum(0)
    u = lbm.momentum(f, lat) / rho
    feq = lbm.feq_modeq(rho, u, lbm.gradient(rho, lat), lbm.laplacian(rho, lat), p)
    want = f - (f - feq) / tau
    assert np.allclose(lbm.collide(f, 0, p), want, rtol=0, atol=1e-15)
    # and one step streams f*_i(r) to r + c_i
    fn = lbm.step(f, 0, p)
    for i in range(lat.q):
        c = lat.c[i]
        assert np.allclose(lbm.shift(fn[i], c), want[i], atol=1e-15)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_guo_equal_rates_reduce_to_bgk_guo(name):
    tau = 0.9
    lat = lattice.get(name)
    p = lbm.Params(lattice=name, coupling="guo", nx=5, ny=4, nz=3 if lat.d == 3 else 1,
                   a=0.02, b=0.2, kappa=0.03, kT=0.0, tau=tuple([tau] * lat.q))
    f = _rand_state(p, seed=4)
    rho = f.sum(0)
    j = lbm.momentum(f, lat)
    F = p.kappa * rho * lbm.gradient(lbm.laplacian(rho, lat), lat)
    u = (j + F / 2) / rho
    feq = lbm.feq_landau_pressure(rho, u, p)
    want = f - (f - feq) / tau + (1 - 1 / (2 * tau)) * lbm.guo_population_force(u, F, lat)
    assert np.allclose(lbm.collide(f, 0, p), want, rtol=0, atol=1e-15)


def test_uniform_rest_state_is_fixed_point():
    for case in CASES:
        p = lbm.Params(**dict(case, kT=0.0))
        rho = np.full(p.shape, p.rho_c)
        f = lbm.equilibrium_at_rest(rho, p)
        assert np.allclose(lbm.step(f, 0, p), f, atol=1e-16)


@pytest.mark.parametrize("case", [CASES[0], CASES[2]])
def test_noise_zero_on_conserved_rows_and_covariance(case):
    """Sample covariance of xi over many sites equals 3 rho kT times Eq. 68's matrix."""
    p = lbm.Params(**dict(case, nx=256, ny=256, nz=1 if case["lattice"] == "D2Q9" else 4,
                          tau=tuple(np.linspace(0.7, 1.6, lattice.get(case["lattice"]).q))))
    rho = np.full(p.shape, 1.1)
    cs2 = np.full(p.shape, 0.21)
    xi = lbm.noise(rho, cs2, 17, p).reshape(p.lat.q - p.lat.n_conserved, -1)
    M = 3 * 1.1 * p.kT * lbm.noise_matrix(np.float64(0.21), p)
    C = xi @ xi.T / xi.shape[1]
    err = np.sqrt((M.diagonal()[:, None] * M.diagonal()[None, :] + M ** 2) / xi.shape[1])
    assert np.all(np.abs(C - M) < 5 * err + 1e-30)
    # the population-space noise carries no mass or momentum
    full = np.zeros((p.lat.q, xi.shape[1]))
    full[p.lat.n_conserved:] = xi
    th = p.lat.populations(full)
    assert np.allclose(th.sum(0), 0, atol=1e-16)
    assert np.allclose(p.lat.c.T.astype(float) @ th, 0, atol=1e-16)


def test_noise_matrix_eq68(golden_dir):
    import os
    vals = {}
    with open(os.path.join(golden_dir, "d2q9_paper_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                vals[k] = np.array([float(x) for x in v])
    p = lbm.Params()
    M = lbm.noise_matrix(np.float64(1 / 3), p)
    assert np.allclose(M, np.diag(vals["noise_diag_cs2_third"]), atol=1e-15)
    M = lbm.noise_matrix(np.float64(0.1), p)
    assert np.allclose([M[0, 0], M[0, 5], M[5, 5]], vals["noise_block_cs2_0.1"], rtol=1e-14)
    # closed form det of the coupled block = (144 - 240 c) at tau = 1
    for c in (-0.2, 0.0, 0.3, 0.59):
        M = lbm.noise_matrix(np.float64(c), p)
        assert np.isclose(M[0, 0] * M[5, 5] - M[0, 5] ** 2, 144 - 240 * c)
        L = np.linalg.cholesky(M)
        assert np.allclose(L @ L.T, M, atol=1e-14)
    # single-tau prefactor (1/tau)(2 - 1/tau) of Eq. 68
    tau = 0.8
    p8 = lbm.Params(tau=tuple([tau] * 9))
    assert np.allclose(lbm.noise_matrix(np.float64(0.1), p8),
                       lbm.noise_matrix(np.float64(0.1), p) * (1 / tau) * (2 - 1 / tau))


def test_errors_on_bad_states():
    p = lbm.Params(nx=4, ny=4, kT=1e-4)
    f = lbm.equilibrium_at_rest(np.full(p.shape, 1.0), p)
    f[0, 0, 1, 1] = -5.0
    with pytest.raises(lbm.NonPositiveDensity):
        lbm.collide(f, 0, p)
    # c_s^2 = rho a >= 0.6 makes Eq. 68 indefinite
    p2 = lbm.Params(nx=4, ny=4, a=0.7, b=0.0, kT=1e-4)
    f = lbm.equilibrium_at_rest(np.full(p2.shape, 1.0), p2)
    with pytest.raises(lbm.NoiseNotPositiveDefinite):
        lbm.collide(f, 0, p2)


def test_noise_uses_the_site_counter():
    """xi at site s and step t is a function of (s, t, system, seed) only."""
    p = lbm.Params(nx=8, ny=4, kT=1e-4)
    rho = np.full(p.shape, 1.0)
    cs2 = np.full(p.shape, 0.0)
    x1 = lbm.noise(rho, cs2, 5, p)
    n = philox.site_normals(np.arange(32, dtype=np.uint64), 5, p.system_id, p.seed, 6)
    L = np.linalg.cholesky(lbm.noise_matrix(np.float64(0.0), p))
    want = np.sqrt(3 * p.kT) * (L @ n)
    assert np.allclose(x1.reshape(6, -1), want, atol=1e-16)


@pytest.mark.parametrize("case", [CASES[0], dict(CASES[2], nx=12, ny=11, nz=9, a=-0.002, tau=tuple([1.0] * 19))])
def test_cut_out_collision_matches_the_whole_system(case):
    """collide on a periodic cut-out of radius 3 around a site, with the global
    site indices as noise keys, gives the whole system's post-collision
    populations at the sites within radius 1 of the centre, and so the centre's
    streamed update (the stencil: density to radius 2 for the Guo force)."""
    import dataclasses
    p = lbm.Params(**case)
    f = _rand_state(p, seed=7)
    t = 11
    full = lbm.step(f, t, p)
    d3 = p.lattice == "D3Q19"
    for (x, y, z) in [(0, 0, 0), (p.nx - 1, 2, p.nz - 1), (5, p.ny - 1, 1)]:
        z = z if d3 else 0
        ix = (np.arange(-3, 4) + x) % p.nx
        iy = (np.arange(-3, 4) + y) % p.ny
        iz = (np.arange(-3, 4) + z) % p.nz if d3 else np.array([0])
        blk = f[:, iz][:, :, iy][:, :, :, ix]
        gid = (iz[:, None, None] * p.ny + iy[None, :, None]) * p.nx + ix[None, None, :]
        pb = dataclasses.replace(p, nx=7, ny=7, nz=7 if d3 else 1)
        fs = lbm.collide(blk, t, pb, sites=gid.ravel())
        c = p.lat.c
        zc = 3 if d3 else 0
        got = np.array([fs[i, zc - (c[i, 2] if d3 else 0), 3 - c[i, 1], 3 - c[i, 0]] for i in range(p.lat.q)])
        assert np.allclose(got, full[:, z, y, x], rtol=0, atol=1e-15)

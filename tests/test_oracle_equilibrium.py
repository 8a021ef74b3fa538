"""Pins for the equilibria, forcing and stencils against the paper's moment conditions."""
import numpy as np
import pytest

from oracle import lattice, lbm


def _smooth_fields(shape, seed=0, amp=0.05):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rho = 1.0 + amp * (np.sin(2 * np.pi * x / nx + rng.random()) * np.cos(2 * np.pi * y / ny)
                       + 0.3 * rng.standard_normal(shape))
    u = 0.02 * rng.standard_normal((3,) + shape)
    if nz == 1:
        u[2] = 0
    return rho, u


def test_modified_equilibrium_moments_eq62_to_64():
    """sum f = rho, sum f c = rho u, sum f c c = P + rho u u + nu(...)  (Eqs. 62-64)."""
    p = lbm.Params(nx=12, ny=10, a=-0.03, b=0.7, kappa=0.02, tau=tuple([0.8] * 9))
    lat = p.lat
    rho, u = _smooth_fields(p.shape)
    grad = lbm.gradient(rho, lat)
    lap = lbm.laplacian(rho, lat)
    feq = lbm.feq_modeq(rho, u, grad, lap, p)
    c = lat.c.astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-14)
    assert np.allclose(np.tensordot(c.T, feq, 1)[:2], rho * u[:2], atol=1e-15)
    # Eq. 64 written out independently of the weights of Eq. 65
    phi = (rho - p.rho_c) / p.rho_c
    f0 = p.a / 2 * phi ** 2 + p.b / 4 * phi ** 4
    p0 = rho / p.rho_c * (p.a * phi + p.b * phi ** 3) - f0
    g2 = grad[0] ** 2 + grad[1] ** 2
    nu = (0.8 - 0.5) / 3
    for al in range(2):
        for be in range(2):
            P = (p0 - p.kappa * rho * lap - p.kappa / 2 * g2) * (al == be) \
                + p.kappa * grad[al] * grad[be]
            hol = nu * (u[al] * grad[be] + u[be] * grad[al]
                        + (u[0] * grad[0] + u[1] * grad[1]) * (al == be))
            want = P + rho * u[al] * u[be] + hol
            got = np.tensordot(c[:, al] * c[:, be], feq, 1)
            assert np.allclose(got, want, rtol=0, atol=1e-14)


def test_modified_equilibrium_d3q19_moments_eq62_to_64():
    """The D3Q19 modified equilibrium meets the same conditions in 3-D:
    sum f = rho, sum f c = rho u, sum f c c = P + rho u u + nu(...) with
    P = (p0 - kappa rho lap rho - kappa/2 |grad rho|^2) 1 + kappa grad rho grad rho."""
    taus = tuple([1.0] * 4 + list(np.linspace(0.7, 1.3, 15)))
    p = lbm.Params(lattice="D3Q19", coupling="modeq", nx=7, ny=6, nz=5, a=-0.03, b=0.7, kappa=0.02, tau=taus)
    lat = p.lat
    rho, u = _smooth_fields(p.shape, seed=5)
    grad = lbm.gradient(rho, lat)
    lap = lbm.laplacian(rho, lat)
    feq = lbm.feq_modeq(rho, u, grad, lap, p)
    c = lat.c.astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-14)
    assert np.allclose(np.tensordot(c.T, feq, 1), rho * u, atol=1e-15)
    phi = (rho - p.rho_c) / p.rho_c
    f0 = p.a / 2 * phi ** 2 + p.b / 4 * phi ** 4
    p0 = rho / p.rho_c * (p.a * phi + p.b * phi ** 3) - f0
    g2 = (grad ** 2).sum(0)
    nu = (taus[6] - 0.5) / 3
    udg = (u * grad).sum(0)
    for al in range(3):
        for be in range(3):
            P = (p0 - p.kappa * rho * lap - p.kappa / 2 * g2) * (al == be) + p.kappa * grad[al] * grad[be]
            hol = nu * (u[al] * grad[be] + u[be] * grad[al] + udg * (al == be))
            got = np.tensordot(c[:, al] * c[:, be], feq, 1)
            assert np.allclose(got, P + rho * u[al] * u[be] + hol, rtol=0, atol=1e-14)


def _gradient_weights(lat, A, B):
    """Per velocity, the coefficients of g_x^2, g_y^2, g_x g_y (and on 3-D g_z^2)
    in kappa^-1 times the square-gradient terms t_i [(9/2)(c.g)^2 + A c^2 |g|^2 + B |g|^2]."""
    c = lat.c.astype(float)
    c2 = (c ** 2).sum(1)
    wxx = lat.t * (4.5 * c[:, 0] ** 2 + A * c2 + B)
    wyy = lat.t * (4.5 * c[:, 1] ** 2 + A * c2 + B)
    wzz = lat.t * (4.5 * c[:, 2] ** 2 + A * c2 + B)
    wxy = lat.t * 9.0 * c[:, 0] * c[:, 1]
    wxx[0] = wyy[0] = wzz[0] = wxy[0] = 0.0          # the rest population restores the mass
    return wxx, wyy, wzz, wxy


def test_printed_gradient_weights_are_the_rotation_invariant_form():
    """The printed w^xx, w^yy, w^xy of Eq. 65 (D2Q9) are exactly
    t_i [(9/2)(c.g)^2 - (9/2) c^2 |g|^2 + 3 |g|^2] coefficient by coefficient:
    the form the D3Q19 set generalises."""
    A, B = lbm.modeq_gradient_coefficients(2)
    assert (A, B) == (-4.5, 3.0)
    wxx, wyy, _, wxy = _gradient_weights(lattice.d2q9(), A, B)
    assert np.allclose(wxx, lattice.POOLEY_WXX, rtol=0, atol=1e-16)
    assert np.allclose(wyy, lattice.POOLEY_WYY, rtol=0, atol=1e-16)
    assert np.allclose(wxy, lattice.POOLEY_WXY, rtol=0, atol=1e-16)


def test_d3q19_gradient_weights_and_the_freedom_left():
    """D3Q19: A = -9/2, B = 9/2.  Coefficient of g_x^2 per velocity class:
    1/4 on (+-1,0,0), 0 on the other axes and on the edges with c_x != 0, -1/8
    on the yz edges; of g_x g_y: +-1/4 on the xy edges (as on D2Q9).  Second
    moments: +1/2 (xx), -1/2 (yy, zz), 0 off the diagonal -- and every (A, B)
    on the line A (d + 2)/9 + B/3 = -1 meets them (the freedom Eq. 63 leaves)."""
    lat = lattice.d3q19()
    A, B = lbm.modeq_gradient_coefficients(3)
    assert (A, B) == (-4.5, 4.5)
    wxx, wyy, wzz, wxy = _gradient_weights(lat, A, B)
    c = lat.c.astype(float)
    by_class = {}
    for i in range(1, 19):
        key = (abs(c[i, 0]), abs(c[i, 1]) + abs(c[i, 2]))
        by_class.setdefault(key, set()).add(round(wxx[i], 15))
    assert by_class == {(1, 0): {0.25}, (0, 1): {0.0}, (1, 1): {0.0}, (0, 2): {-0.125}}
    assert set(np.round(wxy[7:11], 15)) == {0.25, -0.25}
    for Aa in (A, -2.0, 0.0):
        Bb = -3.0 * (1.0 + Aa * 5.0 / 9.0)
        wxx, _, _, wxy = _gradient_weights(lat, Aa, Bb)
        assert np.isclose((wxx * c[:, 0] ** 2).sum(), 0.5)
        assert np.isclose((wxx * c[:, 1] ** 2).sum(), -0.5) and np.isclose((wxx * c[:, 2] ** 2).sum(), -0.5)
        assert np.isclose((wxx * c[:, 0] * c[:, 1]).sum(), 0.0)
        assert np.isclose((wxy * c[:, 0] * c[:, 1]).sum(), 1.0) and np.isclose((wxy * c[:, 0] ** 2).sum(), 0.0)


def test_gradient_weight_sums_by_hand():
    """The three readings of Eq. 65 rest on these second moments of w^xx, w^yy, w^xy."""
    c = lattice.d2q9().c.astype(float)
    cx2, cy2, cxy = c[:, 0] ** 2, c[:, 1] ** 2, c[:, 0] * c[:, 1]
    assert np.isclose((lattice.POOLEY_WXX * cx2).sum(), 0.5)
    assert np.isclose((lattice.POOLEY_WXX * cy2).sum(), -0.5)
    assert np.isclose((lattice.POOLEY_WYY * cx2).sum(), -0.5)
    assert np.isclose((lattice.POOLEY_WYY * cy2).sum(), 0.5)
    assert np.isclose((lattice.POOLEY_WXY * cxy).sum(), 1.0)
    assert np.isclose((lattice.POOLEY_WXX * cxy).sum(), 0.0)
    assert np.isclose((lattice.POOLEY_WXY * cx2).sum(), 0.0)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_standard_equilibrium_and_guo_moments(name):
    lat = lattice.get(name)
    shape = (4, 5, 6) if lat.d == 3 else (1, 5, 6)
    rho, u = _smooth_fields(shape, seed=3)
    c = lat.c.astype(float)
    feq = lbm.feq_standard(rho, u, lat)
    assert np.allclose(feq.sum(0), rho, atol=1e-15)
    assert np.allclose(np.tensordot(c.T, feq, 1), rho * u, atol=1e-15)
    for al in range(lat.d):
        for be in range(lat.d):
            want = rho / 3 * (al == be) + rho * u[al] * u[be]
            assert np.allclose(np.tensordot(c[:, al] * c[:, be], feq, 1), want, atol=1e-14)
    F = 0.01 * np.random.default_rng(1).standard_normal((3,) + shape)
    if lat.d == 2:
        F[2] = 0
    Fi = lbm.guo_population_force(u, F, lat)
    assert np.allclose(Fi.sum(0), 0, atol=1e-16)
    assert np.allclose(np.tensordot(c.T, Fi, 1), F, atol=1e-16)
    for al in range(lat.d):
        for be in range(lat.d):
            want = u[al] * F[be] + u[be] * F[al]
            assert np.allclose(np.tensordot(c[:, al] * c[:, be], Fi, 1), want, atol=1e-16)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_landau_pressure_equilibrium_moments(name):
    """Guo variant: sum f = rho, sum f c = rho u, sum f c c = p0 1 + rho u u."""
    lat = lattice.get(name)
    p = lbm.Params(lattice=name, coupling="guo", a=-0.03, b=0.5, nx=6, ny=5,
                   nz=4 if lat.d == 3 else 1)
    rho, u = _smooth_fields(p.shape, seed=7)
    feq = lbm.feq_landau_pressure(rho, u, p)
    c = lat.c.astype(float)
    phi = rho - 1.0
    p0 = rho * (p.a * phi + p.b * phi ** 3) - (p.a / 2 * phi ** 2 + p.b / 4 * phi ** 4)
    assert np.allclose(feq.sum(0), rho, atol=1e-15)
    assert np.allclose(np.tensordot(c.T, feq, 1), rho * u, atol=1e-15)
    for al in range(lat.d):
        for be in range(lat.d):
            want = p0 * (al == be) + rho * u[al] * u[be]
            assert np.allclose(np.tensordot(c[:, al] * c[:, be], feq, 1), want, atol=1e-14)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_stencils_exact_on_polynomials(name):
    lat = lattice.get(name)
    n = 9
    shape = (n, n, n) if lat.d == 3 else (1, n, n)
    z, y, x = np.meshgrid(*(np.arange(s, dtype=float) for s in shape), indexing="ij")
    ctr = (slice(2, -2),) * 3 if lat.d == 3 else (slice(None), slice(2, -2), slice(2, -2))
    g = lbm.gradient(3 * x - 2 * y + (z if lat.d == 3 else 0), lat)
    assert np.allclose(g[0][ctr], 3) and np.allclose(g[1][ctr], -2)
    lap = lbm.laplacian(x * x + 2 * y * y + (3 * z * z if lat.d == 3 else 0) + x * y, lat)
    assert np.allclose(lap[ctr], 2 + 4 + (6 if lat.d == 3 else 0))


def test_d2q9_laplacian_fourier_symbol():
    """k^2 of the structure factor is the symbol of the discrete Laplacian (text below Eq. 80):
    (2/3)(5 - 2 cos kx - 2 cos ky - cos kx cos ky) for the isotropic D2Q9 stencil."""
    lat = lattice.d2q9()
    n = 16
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for kx, ky in [(1, 0), (2, 3), (5, 7), (8, 8)]:
        k = 2 * np.pi * np.array([kx, ky]) / n
        wave = np.exp(1j * (k[0] * x + k[1] * y))[None]
        lap = lbm.laplacian(wave.real, lat) + 1j * lbm.laplacian(wave.imag, lat)
        sym = (2 / 3) * (5 - 2 * np.cos(k[0]) - 2 * np.cos(k[1]) - np.cos(k[0]) * np.cos(k[1]))
        assert np.allclose(lap, -sym * wave, atol=1e-13)


def test_landau_thermodynamics():
    """p0 and c_s^2 = d p0/d rho by central differences; mu consistent with f0'."""
    p = lbm.Params(a=-0.02, b=0.3, rho_c=1.3)
    rho = np.linspace(0.8, 1.7, 11)
    _, _, _, p0, cs2 = lbm.landau(rho, p)
    h = 1e-6
    _, _, _, pp, _ = lbm.landau(rho + h, p)
    _, _, _, pm, _ = lbm.landau(rho - h, p)
    assert np.allclose((pp - pm) / (2 * h), cs2, rtol=1e-7, atol=1e-9)
    # p0 = rho f'(rho) - f(rho) with f as a function of rho
    phi = (rho - p.rho_c) / p.rho_c
    f = p.a / 2 * phi ** 2 + p.b / 4 * phi ** 4
    fp = (p.a * phi + p.b * phi ** 3) / p.rho_c
    assert np.allclose(p0, rho * fp - f, atol=1e-15)

"""Pins of the oracle's momentum spectra (Eq. 69 diagnostics) and Ornstein-Zernike fit (Eq. 25).

- the spectra against a brute-force discrete Fourier sum on a tiny lattice;
- Parseval's identity over the full k grid;
- plane waves: a longitudinal wave has no transverse part and vice versa;
- the fluid momentum rho u of the Guo variant equals the mean of the momentum
  before and after a noiseless collision (the force adds F per step);
- the fit returns chi and xi of an exact Ornstein-Zernike spectrum on the
  lattice grid, and xi = 0 for a flat spectrum.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import lbm
from oracle import observables as ob
from oracle.lattice import d2q9, d3q19
from tests.helpers import params_of

import synth


def _brute(j, d):
    nz, ny, nx = j.shape[1:]
    N = nx * ny * nz
    out = np.zeros((3, nz, ny, nx))
    sides = (nx, ny, nz)
    for kz, ky, kx in itertools.product(range(nz), range(ny), range(nx)):
        J = np.zeros(3, dtype=complex)
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            ph = -2j * math.pi * (kx * x / nx + ky * y / ny + kz * z / nz)
            J += j[:, z, y, x] * np.exp(ph)
        n = np.array([k if 2 * k < s else k - s for k, s in zip((kx, ky, kz), sides)], dtype=float)
        nn = math.sqrt((n[:d] ** 2).sum())
        out[0, kz, ky, kx] = abs(J[0]) ** 2 / N
        if nn > 0:
            par = abs((n[:d] / nn * J[:d]).sum()) ** 2
            tot = (abs(J[:d]) ** 2).sum()
            out[1, kz, ky, kx] = par / N
            out[2, kz, ky, kx] = (tot - par) / (N * (d - 1))
    return out


@pytest.mark.parametrize("shape,d", [((1, 4, 5), 2), ((3, 4, 2), 3)])
def test_spectra_match_brute_force_dft(shape, d):
    rng = np.random.default_rng(11)
    j = rng.normal(size=(3,) + shape)
    if d == 2:
        j[2] = 0.0
    got = ob.spectra_of_momentum(j, d)
    assert np.allclose(got, _brute(j, d), rtol=1e-12, atol=1e-13)


def test_parseval_over_the_k_grid():
    rng = np.random.default_rng(5)
    j = rng.normal(size=(3, 6, 5, 4))
    sp = ob.spectra_of_momentum(j, 3)
    N = j[0].size
    assert sp[0].sum() == pytest.approx((j[0] ** 2).sum(), rel=1e-12)
    J0 = j.sum(axis=(1, 2, 3))
    total = sp[1].sum() + 2 * sp[2].sum() + (J0 ** 2).sum() / N
    assert total == pytest.approx((j ** 2).sum(), rel=1e-12)


@pytest.mark.parametrize("kind", ["longitudinal", "transverse"])
def test_plane_waves_split_into_their_projection(kind):
    nz, ny, nx = 8, 8, 8
    n0 = np.array([1.0, 2.0, 0.0])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phase = 2 * np.pi * (n0[0] * x / nx + n0[1] * y / ny)
    e = n0 / np.linalg.norm(n0) if kind == "longitudinal" else np.array([-2.0, 1.0, 0.0]) / math.sqrt(5)
    j = e[:, None, None, None] * np.cos(phase)[None]
    sp = ob.spectra_of_momentum(j, 3)
    N = nx * ny * nz
    peak = N / 4.0                                   # |J(+-k0)|^2 / N for a cosine of unit amplitude
    idx = [(0, 2, 1), (0, ny - 2, nx - 1)]
    if kind == "longitudinal":
        assert np.allclose(sp[2], 0.0, atol=1e-10)
        for i in idx:
            assert sp[1][i] == pytest.approx(peak, rel=1e-12)
        assert sp[1].sum() == pytest.approx(2 * peak, rel=1e-12)
    else:
        assert np.allclose(sp[1], 0.0, atol=1e-10)
        for i in idx:
            assert sp[2][i] == pytest.approx(peak / 2, rel=1e-12)   # per transverse component


@pytest.mark.parametrize("lattice,coupling", [("D2Q9", "guo"), ("D3Q19", "guo"), ("D2Q9", "modeq")])
def test_fluid_momentum_is_mean_of_pre_and_post_collision(lattice, coupling):
    s = synth.system(lattice, coupling, n=8, a=-0.003, kT=0.0, kappa=0.02)
    p = params_of(s)
    f = lbm.initial_state(p, amplitude=0.05)
    f = lbm.run(f, 0, 2, p)
    jf = ob.fluid_momentum(f, p)
    j0 = lbm.momentum(f, p.lat)
    if coupling == "guo":
        j1 = lbm.momentum(lbm.collide(f, 2, p), p.lat)
        assert np.max(np.abs(jf - 0.5 * (j0 + j1))) < 1e-15
        assert np.max(np.abs(j1 - j0)) > 1e-8          # the force is not trivially zero here
    else:
        assert np.array_equal(jf, j0)


def _binned_oz(shape, lat, chi, xi, kT, kmax):
    k2 = ob.laplacian_symbol(shape, lat)
    C = kT * chi / (1.0 + xi * xi * k2)
    return ob.bin_shells(C, shape, kmax)


@pytest.mark.parametrize("shape,lat", [((32, 32, 32), d3q19()), ((1, 64, 64), d2q9())])
def test_oz_fit_recovers_chi_and_xi(shape, lat):
    kT, chi, xi = 1e-4, 12.0, 1.5
    sums, counts = _binned_oz(shape, lat, chi, xi, kT, 6)
    fit = ob.oz_fit(sums, counts, 1, shape, lat, kT, 6)
    # shell averages of 1/(1 + xi^2 k^2) differ from the value at the mean k^2 at
    # second order in xi^2 times the spread of k^2 inside a shell: < 1% here
    assert fit["chi"] == pytest.approx(chi, rel=1e-2)
    assert fit["xi"] == pytest.approx(xi, rel=1e-2)
    assert fit["shells"] == 6


def test_oz_fit_flat_spectrum_and_sample_count():
    shape, lat = (16, 16, 16), d3q19()
    sums, counts = _binned_oz(shape, lat, 7.0, 0.0, 2e-4, 5)
    fit = ob.oz_fit(3 * sums, counts, 3, shape, lat, 2e-4, 5)
    assert fit["chi"] == pytest.approx(7.0, rel=1e-12)
    assert abs(fit["xi"]) < 1e-6
    with pytest.raises(ValueError):
        ob.oz_fit(sums, counts, 1, (8, 8, 8), lat, 2e-4, 5)


def test_recorder_accumulates_momentum_spectra():
    p = params_of(synth.system("D2Q9", "guo", n=16, kT=1e-4))
    f = lbm.initial_state(p, amplitude=0.02)
    rec = ob.Recorder(p, every=0, sk_every=2, jk=True)
    g = lbm.run(f, 0, 4, p, rec)
    assert rec.n_sk == 2
    want = ob.momentum_spectra(lbm.run(f, 0, 2, p), p) + ob.momentum_spectra(g, p)
    assert np.allclose(rec.jk, want, rtol=1e-13, atol=1e-20)

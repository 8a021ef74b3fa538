"""Exact and near-exact statics of the oracle's fluctuating dynamics.

* kappa = 0, modified equilibrium: the linearised dynamics with the noise of
  Eq. 68 has the stationary covariance G = rho_0 kT diag(1/c - 5/3, w_1..w_8),
  c = c_s^2(rho_0), w_i the weights of Eq. 65.  It gives <|j_k|^2> = rho_0 kT
  (Eq. 69) and C(k) = kT/(rho_0 c) = kT/r (Eq. 25 at kappa = 0) for every k.
  It is stationary only if the noise is the fluctuation-dissipation one, so
  this pins Eq. 68 entry by entry, including the sign of the (4,9) coupling,
  and the per-mode reading 1 - gamma_a gamma_b.
* kappa > 0: the paper's noise neglects terms of order kappa, so C(k) is the
  Ornstein-Zernike form kT/(r + kappa k^2) (Eq. 25, k^2 the discrete Laplacian
  symbol) only approximately; the tolerance follows the paper's
  "error below a few percent" for kappa <~ 1e-3 (Sec. III B, Fig. momtm-equil).
"""
import dataclasses

import numpy as np
import pytest

from oracle import lattice, lbm
from tests import linear_response as lr


def _G(p):
    """rho_0 kT diag(1/c - 3(1 - t_0), 3 t_1, ..., 3 t_{q-1}); on D2Q9 the entries
    i >= 1 are the weights w_i of Eq. 65 and 3(1 - t_0) = 5/3."""
    _, _, _, _, c = lbm.landau(np.float64(p.rho_c), p)
    t = p.lat.t
    g = p.rho_c * p.kT * np.concatenate([[1 / c - 3 * (1 - t[0])], 3 * t[1:]])
    return np.diag(g)


@pytest.mark.parametrize("a,rho_c,taus", [
    (1 / 3, 1.0, [1.0] * 9),            # ideal point: textbook 3 rho kT t_i
    (0.05, 1.0, [1.0] * 9),
    (0.01, 1.0, [0.8] * 9),
    (0.2, 1.3, [1, 1, 1, 0.7, 0.9, 1.2, 0.6, 1.5, 1.1]),
    (-0.02, 1.0, [1, 1, 1, 0.9, 0.8, 0.8, 1.3, 1.3, 0.75]),   # c < 0 is still stable at rest
])
def test_kappa0_exact_fluctuation_dissipation(a, rho_c, taus):
    p = lbm.Params(nx=6, ny=5, a=a, b=0.3, kappa=0.0, kT=1e-5, rho_c=rho_c, tau=tuple(taus))
    _check_exact_fdt(p)
    if a == 1 / 3:
        assert np.allclose(_G(p), np.diag(3 * rho_c * p.kT * lattice.d2q9().t))
    assert np.allclose(_G(p).diagonal()[1:], p.rho_c * p.kT * lattice.POOLEY_W[1:])


@pytest.mark.parametrize("name,shape,coupling", [("D2Q9", (1, 5, 6), "guo"), ("D3Q19", (3, 4, 5), "guo"),
                                                  ("D3Q19", (3, 4, 5), "modeq")])
@pytest.mark.parametrize("a", [1 / 3, 0.04, -0.01])
def test_guo_kappa0_exact_fluctuation_dissipation(name, shape, coupling, a):
    """Also the D3Q19 modified equilibrium: at kappa = 0 it has the same
    linearised dynamics, and the lattice-general noise is exact for it."""
    q = lattice.get(name).q
    taus = [1.0] * (1 + lattice.get(name).d) + list(np.linspace(0.6, 1.6, q - 1 - lattice.get(name).d))
    p = lbm.Params(lattice=name, coupling=coupling, nz=shape[0], ny=shape[1], nx=shape[2],
                   a=a, b=0.2, kappa=0.0, kT=1e-5, tau=tuple(taus))
    _check_exact_fdt(p)


def test_general_noise_form_is_eq68_on_d2q9():
    for c in (-0.1, 0.0, 0.1, 1 / 3, 0.5):
        pm = lbm.Params(coupling="modeq", tau=tuple(np.linspace(0.7, 1.3, 9)))
        pg = lbm.Params(coupling="guo", tau=tuple(np.linspace(0.7, 1.3, 9)))
        assert np.allclose(lbm.noise_matrix(np.float64(c), pm), lbm.noise_matrix(np.float64(c), pg),
                           rtol=0, atol=1e-14)


def _check_exact_fdt(p):
    G = _G(p)
    J = lr.jk_all(lr.site_response(p))
    Ql = lr.local_noise_population_cov(p)
    KZ, KY, KX = lr.k_grid(p)
    c = p.lat.c.astype(float)
    for idx in np.ndindex(*p.shape):
        k = np.array([KX[idx], KY[idx], KZ[idx]])
        D = np.diag(np.exp(-1j * (c @ k)))
        Jk = J[(slice(None), slice(None)) + idx]
        lhs = Jk @ G @ Jk.conj().T + D @ Ql @ D.conj().T
        assert np.allclose(lhs, G, rtol=0, atol=1e-9 * np.abs(G).max())


def _break_offdiag(monkeypatch):
    orig = lbm.noise_matrix

    def flipped(cs2, p):
        M = orig(cs2, p).copy()
        M[..., 0, 5] *= -1
        M[..., 5, 0] *= -1
        return M
    monkeypatch.setattr(lbm, "noise_matrix", flipped)


def test_planted_sign_error_is_caught(monkeypatch):
    """A flipped (4,9) entry of Eq. 68, planted in the oracle, breaks the exact pin."""
    _break_offdiag(monkeypatch)
    with pytest.raises(AssertionError):
        test_kappa0_exact_fluctuation_dissipation(0.05, 1.0, [1.0] * 9)


@pytest.mark.parametrize("kappa,tol", [(1e-4, 0.02), (1e-3, 0.05)])
def test_ornstein_zernike_and_momentum_equipartition(kappa, tol):
    p = lbm.Params(nx=16, ny=16, a=0.02, b=0.0, kappa=kappa, kT=1e-6, tau=tuple([0.8] * 9))
    skipped = []
    S = lr.stationary_covariances(p, skipped=skipped)
    assert sorted(skipped) == [(0, 0, 8), (0, 8, 0)]
    c = p.lat.c.astype(float)
    ones = np.ones(p.lat.q)
    worst_c = worst_j = 0.0
    for idx, Sk in S.items():
        ck = (ones @ Sk @ ones).real / p.rho_c ** 2
        oz = p.kT / (p.a + p.kappa * lr.laplacian_symbol(p, idx))
        worst_c = max(worst_c, abs(ck / oz - 1))
        for al in range(2):
            jj = (c[:, al] @ Sk @ c[:, al]).real
            worst_j = max(worst_j, abs(jj / (p.rho_c * p.kT) - 1))
    assert worst_c < tol, worst_c
    assert worst_j < tol, worst_j


def test_planted_missing_kappa_term_is_caught(monkeypatch):
    """Dropping the kappa rho lap rho term of Eq. 64 from the equilibrium breaks OZ."""
    orig = lbm.feq_modeq

    def broken(rho, u, grad, lap, p):
        return orig(rho, u, grad, 0 * lap, p)
    monkeypatch.setattr(lbm, "feq_modeq", broken)
    with pytest.raises(AssertionError):
        test_ornstein_zernike_and_momentum_equipartition(1e-3, 0.05)


@pytest.mark.parametrize("name,shape", [("D2Q9", (1, 24, 24)), ("D3Q19", (8, 8, 8))])
def test_guo_variant_ornstein_zernike(name, shape):
    """Guo variant at kappa = 1e-3: momentum equipartition to 1% at every k; the
    square-gradient force has the lattice symbol of a stencil gradient of a
    stencil Laplacian, so OZ holds to 1% for k <= 1 (wavelengths >~ 6 sites,
    where the paper notes lattice effects begin, below Eq. 80)."""
    q = lattice.get(name).q
    p = lbm.Params(lattice=name, coupling="guo", nz=shape[0], ny=shape[1], nx=shape[2],
                   a=0.02, b=0.0, kappa=1e-3, kT=1e-6, tau=tuple([0.8] * q))
    S = lr.stationary_covariances(p)
    c = p.lat.c.astype(float)
    ones = np.ones(q)
    KZ, KY, KX = lr.k_grid(p)
    for idx, Sk in S.items():
        k = np.sqrt(KX[idx] ** 2 + KY[idx] ** 2 + KZ[idx] ** 2)
        for al in range(p.lat.d):
            jj = (c[:, al] @ Sk @ c[:, al]).real
            assert abs(jj / (p.rho_c * p.kT) - 1) < 0.01
        if k <= 1.0:
            ck = (ones @ Sk @ ones).real / p.rho_c ** 2
            oz = p.kT / (p.a + p.kappa * lr.laplacian_symbol(p, idx))
            assert abs(ck / oz - 1) < 0.01, (idx, ck / oz)


@pytest.mark.parametrize("kappa", [1e-4, 1e-3])
def test_d3q19_modified_equilibrium_ornstein_zernike(kappa):
    """The D3Q19 modified equilibrium (derived square-gradient weights) at
    kappa <= 1e-3: momentum equipartition (Eq. 69) within 1% at every k and the
    Ornstein-Zernike C(k) (Eq. 25, k^2 the lattice Laplacian's symbol) within 1%
    for k <= 1, from the exact Lyapunov solve of the linearised step (measured:
    0.35% and 0.06% at kappa = 1e-3)."""
    p = lbm.Params(lattice="D3Q19", coupling="modeq", nz=8, ny=8, nx=8, a=0.02, b=0.0, kappa=kappa, kT=1e-6,
                   tau=tuple([0.8] * 19))
    S = lr.stationary_covariances(p)
    c = p.lat.c.astype(float)
    ones = np.ones(19)
    KZ, KY, KX = lr.k_grid(p)
    for idx, Sk in S.items():
        k = np.sqrt(KX[idx] ** 2 + KY[idx] ** 2 + KZ[idx] ** 2)
        for al in range(3):
            assert abs((c[:, al] @ Sk @ c[:, al]).real / (p.rho_c * p.kT) - 1) < 0.01
        if k <= 1.0:
            ck = (ones @ Sk @ ones).real / p.rho_c ** 2
            oz = p.kT / (p.a + p.kappa * lr.laplacian_symbol(p, idx))
            assert abs(ck / oz - 1) < 0.01, (idx, ck / oz)

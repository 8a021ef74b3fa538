"""Pins of the oracle's perturbation-theory comparator (Sec. II C, Eqs. 31-43).

- the two-loop sum as the O(N^2) double sum of its definition equals the
  convolution identity sum_r g(r)^3 (an independent formula);
- at kappa = 0 every propagator is 1/m and the lattice sums have closed forms
  in N (pair counting), so Eq. 36 becomes a quartic and Eq. 40 a quadratic in
  v^2, solved here with numpy's polynomial roots / the quadratic formula;
- u = 0 or kT -> 0 reduce to mean-field values.
"""
import numpy as np
import pytest

from oracle import perturbation as pt


@pytest.mark.parametrize("lattice,side,m,kappa", [("D2Q9", 8, 0.02, 0.1), ("D3Q19", 6, 0.005, 0.03),
                                                  ("D2Q9", 7, 1.0, 0.5)])
def test_two_loop_double_sum_equals_convolution_identity(lattice, side, m, kappa):
    G = pt.propagator(side, pt.lattice_of(lattice), m, kappa)
    assert pt.s2_brute(G) == pytest.approx(pt.s2_fft(G), rel=1e-12)


@pytest.mark.parametrize("lattice,side", [("D2Q9", 8), ("D3Q19", 5)])
def test_sums_at_kappa_zero_count_the_modes(lattice, side):
    m = 0.37
    G = pt.propagator(side, pt.lattice_of(lattice), m, 0.0)
    N = G.size
    assert pt.s1(G) == pytest.approx((N - 1) / (N * m), rel=1e-14)
    assert pt.s1sq(G) == pytest.approx((N - 1) / (N * m * m), rel=1e-14)
    pairs = (N - 1) * (N - 2)                      # q1 != 0, q2 != 0, q1 + q2 != 0
    assert pt.s2_brute(G) == pytest.approx(pairs / (N * N * m ** 3), rel=1e-13)
    assert pt.s2_fft(G) == pytest.approx(pairs / (N * N * m ** 3), rel=1e-12)


@pytest.mark.parametrize("r,u,kT", [(1e-2, 0.1, 1e-4), (2e-3, 0.4, 1e-6), (5e-3, 1.0, 1e-6)])
def test_symmetric_phase_at_kappa_zero_solves_the_quartic(r, u, kT):
    side = 6
    N = side ** 3
    c1 = (N - 1) / N
    c2 = (N - 1) * (N - 2) / N ** 2
    # r' = r + 3 u kT c1 / r' - 6 u^2 kT^2 c2 / r'^3  ->  r'^4 - r r'^3 - 3 u kT c1 r'^2 + 6 u^2 kT^2 c2 = 0
    roots = np.roots([1.0, -r, -3 * u * kT * c1, 0.0, 6 * u * u * kT * kT * c2])
    real = sorted(x.real for x in roots if abs(x.imag) < 1e-12 * abs(x) and x.real > 0)
    res = pt.symmetric("D3Q19", side, r, u, 0.0, kT)
    assert res["r_prime"] == pytest.approx(max(real), rel=1e-10), (res["r_prime"], real)
    F = r + 3 * u * kT * c1 / res["r_prime"] - 6 * u * u * kT * kT * c2 / res["r_prime"] ** 3 - res["r_prime"]
    assert abs(F) < 1e-12 * max(abs(r), res["r_prime"])
    assert res["chi"] == pytest.approx(1 / res["r_prime"], rel=1e-15)


def test_symmetric_phase_without_a_root_is_reported():
    with pytest.raises(ArithmeticError):      # the two-loop term dominates at every r' > 0
        pt.symmetric("D3Q19", 6, 1e-3, 0.1, 0.0, 1e-4)


def test_symmetric_phase_without_coupling_is_mean_field():
    res = pt.symmetric("D2Q9", 16, 3e-3, 0.0, 1e-2, 1e-4)
    assert res["r_prime"] == pytest.approx(3e-3, rel=1e-13)
    assert res["xi"] == pytest.approx(np.sqrt(1e-2 / 3e-3), rel=1e-13)


@pytest.mark.parametrize("r,u,kT", [(-2e-3, 0.1, 1e-7), (-1e-2, 1.0, 1e-6)])
def test_broken_phase_at_kappa_zero_solves_the_quadratic(r, u, kT):
    side = 8
    N = side ** 2
    c = (N - 1) / N
    # (r + u w)(r + 3 u w) + 3 u kT c = 0, physical root next below -r/u
    w = (-2 * r + np.sqrt(r * r - 9 * u * kT * c)) / (3 * u)
    res = pt.broken("D2Q9", side, r, u, 0.0, kT)
    assert res["v"] ** 2 == pytest.approx(w, rel=1e-10)
    rs = r + 3 * u * w
    assert res["r_sigma"] == pytest.approx(rs, rel=1e-9)
    rps = rs + kT * (-18 * u * u * w * kT * c / rs ** 2 + 3 * u * c / rs)
    assert res["r_prime_sigma"] == pytest.approx(rps, rel=1e-9)
    assert res["v"] < np.sqrt(-r / u)               # fluctuations lower the order parameter


def test_broken_phase_tends_to_mean_field_as_kT_vanishes():
    r, u = -4e-3, 0.2
    res = pt.broken("D3Q19", 8, r, u, 1e-2, 1e-12)
    assert res["v"] == pytest.approx(np.sqrt(-r / u), rel=1e-8)
    assert res["r_prime_sigma"] == pytest.approx(-2 * r, rel=1e-8)
    with pytest.raises(ValueError):
        pt.broken("D3Q19", 8, 1e-3, u, 1e-2, 1e-4)

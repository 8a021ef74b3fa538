"""GPU parity of the perturbation-theory comparator (Sec. II C) against the oracle.

The lattice sums are plain FP64 sums of positive terms (S2 through the
convolution identity on both sides: the device's direct DFT passes, numpy's
FFT in the oracle), so they agree to 1e-12 relative; the roots, found by the
same bracketing and bisection on both sides, agree to 1e-9 relative.
"""
import numpy as np
import pytest

from oracle import perturbation as pt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need CUDA; the library has no CPU fallback")
    import paper_1202_4748_gb300 as m
    return m


@pytest.mark.parametrize("lattice,side,m,kappa", [
    ("D2Q9", 8, 0.02, 0.1), ("D3Q19", 6, 0.005, 0.03), ("D2Q9", 7, 1.0, 0.5),
    ("D3Q19", 64, 1e-3, 1e-2), ("D2Q9", 512, 2e-4, 1e-4), ("D3Q19", 24, 0.3, 0.0),
])
def test_lattice_sums_match_oracle(lb, lattice, side, m, kappa):
    got = lb.pt_sums(lattice, side, m, kappa)
    G = pt.propagator(side, pt.lattice_of(lattice), m, kappa)
    assert got["S1"] == pytest.approx(pt.s1(G), rel=1e-12)
    assert got["S1sq"] == pytest.approx(pt.s1sq(G), rel=1e-12)
    assert got["S2"] == pytest.approx(pt.s2_fft(G), rel=1e-11)
    if G.size <= 512:
        assert got["S2"] == pytest.approx(pt.s2_brute(G), rel=1e-11)


@pytest.mark.parametrize("lattice,side,r,u,kappa,kT", [
    ("D3Q19", 16, 1e-3, 0.1, 1e-2, 1e-5), ("D2Q9", 64, 2e-4, 5e-2, 1e-4, 1e-7),
    ("D3Q19", 32, 5e-3, 1.0, 1e-3, 1e-6),
])
def test_symmetric_phase_matches_oracle(lb, lattice, side, r, u, kappa, kT):
    got = lb.pt_symmetric(lattice, side, r, u, kappa, kT)
    want = pt.symmetric(lattice, side, r, u, kappa, kT)
    for k in ("r_prime", "chi", "xi", "S1", "S2"):
        assert got[k] == pytest.approx(want[k], rel=1e-9), k


@pytest.mark.parametrize("lattice,side,r,u,kappa,kT", [
    ("D3Q19", 16, -2e-3, 0.1, 1e-2, 1e-5), ("D2Q9", 64, -1e-4, 4e-3, 1e-4, 1e-7),
])
def test_broken_phase_matches_oracle(lb, lattice, side, r, u, kappa, kT):
    got = lb.pt_broken(lattice, side, r, u, kappa, kT)
    want = pt.broken(lattice, side, r, u, kappa, kT)
    for k in ("v", "r_sigma", "r_prime_sigma", "chi", "xi", "S1", "S1sq"):
        assert got[k] == pytest.approx(want[k], rel=1e-9), k


def test_missing_roots_are_reported(lb):
    with pytest.raises(lb.LBError) as e:
        lb.pt_symmetric("D3Q19", 6, 1e-3, 0.1, 0.0, 1e-4)
    assert e.value.status == lb.LB_ERR_NO_ROOT
    with pytest.raises(lb.LBError) as e:
        lb.pt_broken("D2Q9", 8, -2e-3, 0.1, 0.0, 1e-5)       # r^2 < 9 u kT: no ordered state
    assert e.value.status == lb.LB_ERR_NO_ROOT

"""Pins of the oracle's order-parameter histograms P_L(m) and their estimators.

The estimators are checked against histograms built from the closed forms of
P_L in Sec. II D: one Gaussian about m = 0 (Eq. 57, disordered phase) and two
displaced Gaussians of half weight each (Eq. 58, coexistence), both with known
L^d, kT, chi_L and M_L.  Expected bin counts are exact integrals of
those densities (normal CDF differences), so the only errors left are the
binning errors, which are estimated in each test.
"""
import math

import numpy as np
import pytest
from scipy.special import ndtr

from oracle import lbm
from oracle import observables as ob
from tests.helpers import params_of

import synth


def _counts(lo, hi, nb, parts, n_total=10 ** 12, under_over=(0, 0)):
    """Integer counts of a mixture of Gaussians [(weight, centre, sigma)] on nb bins."""
    edges = lo + (hi - lo) * np.arange(nb + 1) / nb
    cdf = sum(wt * ndtr((edges - mu) / sg) for wt, mu, sg in parts)
    c = np.rint(n_total * np.diff(cdf)).astype(np.int64)
    return np.concatenate([[under_over[0]], c, [under_over[1]]])


def test_histogram_bins_by_the_stated_rule():
    lo, hi, nb = -1.0, 1.0, 8                        # w = 1/4, every edge exact
    vals = [-1.0, -0.75, -0.7499999, 0.0, 0.24999999, 0.25, 0.999, 1.0, -1.0000001, float("nan"), 5.0, -3.0]
    want = np.zeros(nb + 2, dtype=np.int64)
    for v in vals:                                   # brute force, value by value
        if v < lo:
            want[0] += 1
        elif lo <= v < hi:
            want[1 + int(math.floor((v - lo) / 0.25))] += 1
        else:
            want[-1] += 1
    got = ob.histogram(vals, lo, hi, nb)
    assert np.array_equal(got, want)
    assert got[1] == 1 and got[2] == 2 and got[5] == 2 and got[6] == 1 and got[8] == 1
    assert got[0] == 2 and got[-1] == 3


def test_histogram_matches_numpy_away_from_edges():
    rng = np.random.default_rng(3)
    x = rng.normal(0.0, 0.3, 10000)
    lo, hi, nb = -0.8, 0.8, 64
    h = ob.histogram(x, lo, hi, nb)
    ref, _ = np.histogram(x[(x >= lo) & (x < hi)], bins=nb, range=(lo, hi))
    w = (hi - lo) / nb
    t = (x - lo) / w
    near = np.abs(t - np.rint(t)) < 1e-9
    assert not near.any()
    assert np.array_equal(h[1:-1], ref)
    assert h[0] == (x < lo).sum() and h[-1] == (x >= hi).sum()


@pytest.mark.parametrize("vol,kT,chi", [(64.0, 1e-4, 50.0), (8.0, 1e-4, 4.0), (1.0, 2e-4, 1.5)])
def test_two_displaced_gaussians_recover_M_and_chi(vol, kT, chi):
    sg = math.sqrt(kT * chi / vol)
    nb = 1000
    lo, hi = -0.5, 0.5
    w = (hi - lo) / nb
    # choose M on a bin centre and the bin width small against sigma
    M = lo + (nb * 0.7 + 0.5) * w
    assert w < 0.2 * sg and M / sg > 6
    c = _counts(lo, hi, nb, [(0.5, M, sg), (0.5, -M, sg)])
    est = ob.histogram_estimates(c, lo, hi, vol, kT)
    assert not est["central"]
    assert abs(est["m_max"] - M) < 1e-12
    bin_err = w * w / (12 * sg * sg)                 # relative binning error of peak height^-2 / variance
    assert abs(est["chi_peak"] / chi - 1) < 2 * bin_err + 1e-6
    assert abs(est["chi_fit"] / chi - 1) < 2 * bin_err + 1e-6
    assert abs(est["M_fit"] - M) < 1e-6 * M
    # the peak-height constant: half-weight peaks need the 8 pi form, not 2 pi
    assert abs(vol / (2 * math.pi * kT * est["P_max"] ** 2) / chi - 4) < 0.02


@pytest.mark.parametrize("vol,kT,chi", [(64.0, 1e-4, 50.0), (1.0, 1e-4, 30.0)])
def test_one_central_gaussian_recovers_chi(vol, kT, chi):
    sg = math.sqrt(kT * chi / vol)
    nb = 1001                                        # a bin centred on m = 0
    lo, hi = -0.5, 0.5
    w = (hi - lo) / nb
    c = _counts(lo, hi, nb, [(1.0, 0.0, sg)])
    est = ob.histogram_estimates(c, lo, hi, vol, kT)
    assert est["central"] and abs(est["m_max"]) < 1e-15
    bin_err = w * w / (12 * sg * sg)
    assert abs(est["chi_peak"] / chi - 1) < 2 * bin_err + 1e-6
    assert abs(est["chi_fit"] / chi - 1) < 2 * bin_err + 1e-6
    assert abs(est["M_fit"]) < 1e-9
    assert abs(est["hist_m2"] / (sg * sg) - 1) < 2 * bin_err + 1e-6


def test_central_region_excluded_from_normalisation():
    vol, kT, chi = 27.0, 1e-4, 20.0
    sg = math.sqrt(kT * chi / vol)
    nb, lo, hi = 800, -0.4, 0.4
    w = (hi - lo) / nb
    M = lo + (nb * 0.75 + 0.5) * w
    peaks = _counts(lo, hi, nb, [(0.5, M, sg), (0.5, -M, sg)], n_total=10 ** 10)
    centres = lo + (np.arange(nb) + 0.5) * w
    plateau = np.where(np.abs(centres) < 0.1, 2 * 10 ** 6, 0).astype(np.int64)
    c = peaks.copy()
    c[1:-1] += plateau
    cut = ob.histogram_estimates(c, lo, hi, vol, kT, m_cut=0.1)
    assert abs(cut["chi_peak"] / chi - 1) < 0.01
    nocut = ob.histogram_estimates(c, lo, hi, vol, kT)
    extra = plateau.sum() / 10 ** 10
    assert abs(nocut["chi_peak"] / cut["chi_peak"] - (1 + extra) ** 2) < 1e-6


def test_recorder_histograms_count_every_block_and_match_moments():
    p = params_of(synth.system("D2Q9", n=16, a=-0.002, kT=1e-3))
    f = lbm.initial_state(p, amplitude=0.05)
    nb, lo, hi = 4001, -1.0, 1.0
    rec = ob.Recorder(p, every=2, hist=(nb, lo, hi))
    f = lbm.run(f, 0, 8, p, rec)
    n_samples = 4
    w = (hi - lo) / nb
    for l, blk in enumerate(rec.lv):
        n_blocks = (p.nx // blk[0]) * (p.ny // blk[1])
        assert rec.hist[l].sum() == n_samples * n_blocks
        assert rec.hist[l][0] == 0 and rec.hist[l][-1] == 0
        vol = blk[0] * blk[1] * blk[2]
        est = ob.histogram_estimates(rec.hist[l], lo, hi, vol, p.kT)
        m2 = rec.acc[l][2] / rec.acc[l][0]
        am = rec.acc[l][3] / rec.acc[l][0]
        # binning moves each value by at most w/2
        assert abs(est["hist_abs_m"] - am) <= 0.5 * w + 1e-15
        assert abs(est["hist_m2"] - m2) <= w * math.sqrt(m2) + 0.25 * w * w + 1e-15


def test_estimates_reject_asymmetric_range():
    with pytest.raises(ValueError):
        ob.histogram_estimates(np.ones(12), -0.5, 0.6, 1.0, 1e-4)

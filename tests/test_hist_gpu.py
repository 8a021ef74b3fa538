"""GPU parity of the order-parameter histograms P_L(m) (Sec. II D) against the oracle.

Counts are integers, so the bar is exact equality, except for block values
that the two sides place on opposite sides of a bin edge because their FP64
block sums round differently: those are counted from the oracle's values
(within a relative 1e-9 of an edge) and each may move one count between two
neighbouring bins.
"""
import os

import numpy as np
import pytest

import synth
from oracle import lbm, observables as ob
from tests.helpers import oracle_state, params_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need CUDA; the library has no CPU fallback")
    import paper_1202_4748_gb300 as m
    return m


def _near_edges(m, lo, hi, nb, eps=1e-9):
    t = (np.asarray(m).ravel() - lo) * (nb / (hi - lo))
    return int(np.sum(np.abs(t - np.rint(t)) < eps * max(1.0, nb)))


def _compare(got, want, slack):
    d = got.astype(np.int64) - want.astype(np.int64)
    assert d.sum() == 0
    assert np.abs(d).sum() <= 2 * slack, (np.nonzero(d), slack)


@pytest.mark.parametrize("lattice,coupling,shape,nb", [
    ("D2Q9", "modeq", (32, 32, 1), 400),
    ("D2Q9", "guo", (24, 16, 1), 257),
    ("D3Q19", "guo", (16, 16, 8), 1000),
])
def test_histograms_match_oracle(lb, lattice, coupling, shape, nb):
    s = synth.system(lattice, coupling, n=shape[0], a=-0.002, kT=1e-3, seed=5, system_id=2)
    s.update(nx=shape[0], ny=shape[1], nz=shape[2])
    p = params_of(s)
    f0 = oracle_state(p, seed_amp=0.08)
    lo, hi = -0.12, 0.12
    every, steps = 3, 12
    ens = lb.Ensemble([s], precision="fp64", obs_every=every, hist_bins=nb, hist_range=hi)
    ens.write_fields(0, f0)
    ens.step(steps)
    ens.sync()
    lv = ob.levels(p)
    want = np.zeros((len(lv), nb + 2), dtype=np.int64)
    slack = np.zeros(len(lv), dtype=np.int64)

    def cb(f, t):
        if t % every == 0:
            phi = ob.order_parameter(f)
            for l, blk in enumerate(lv):
                m = ob.block_means(phi, blk)
                want[l] += ob.histogram(m, lo, hi, nb)
                slack[l] += _near_edges(m, lo, hi, nb)

    lbm.run(f0, 0, steps, p, callback=cb)
    levels, glob = ens.observables(0)
    assert glob["n_samples"] == steps // every
    seen_out = 0
    for l, blk in enumerate(lv):
        got, glo, ghi = ens.histogram(0, l)
        assert (glo, ghi) == (lo, hi)
        assert got.sum() == levels[l]["n"]
        _compare(got, want[l], slack[l])
        seen_out += int(got[0] + got[-1])
    assert seen_out > 0          # the narrow range leaves single sites in the under/overflow counts
    ens.close()


def test_histograms_survive_checkpoint_and_graphs(lb, tmp_path):
    systems = synth.ensemble("fss_160", "D2Q9")[:4]
    kw = dict(precision="fp32", obs_every=5, hist_bins=128, hist_range=0.1)
    a = lb.Ensemble(systems, graph_chunk=10, **kw)
    a.init(amplitude=0.02)
    a.step(20)
    path = os.path.join(tmp_path, "ck.bin")
    a.save(path)
    a.step(30)
    ref = [[a.histogram(k, l)[0] for l in range(len(a.observables(k)[0]))] for k in range(4)]
    b = lb.Ensemble(systems, **kw)            # plain launches after the load
    b.load(path)
    b.step(30)
    for k in range(4):
        for l, h in enumerate(ref[k]):
            assert np.array_equal(b.histogram(k, l)[0], h)
    a.close()
    b.close()


def test_histograms_rejected_without_bins(lb):
    e = lb.Ensemble(synth.ensemble("single_16", "D2Q9"), obs_every=5)
    with pytest.raises(lb.LBError) as err:
        e.histogram(0, 0)
    assert err.value.status == lb.LB_ERR_UNSUPPORTED
    e.close()


def test_fss_160_histograms_at_full_size(lb):
    """Properties that hold at any size, in the benchmark's launch configuration
    (FP32, 100-step graph chunks, samples every 100 steps): every block of every
    level is counted once per sample, and the histogram moments equal the
    accumulated moments within the binning error (each value moves <= w/2)."""
    systems = synth.ensemble("fss_160", "D3Q19")
    nb, R = 2000, 0.5
    ens = lb.Ensemble(systems, precision="fp32", obs_every=100, graph_chunk=100, hist_bins=nb, hist_range=R)
    ens.init(amplitude=0.01)
    ens.step(200)
    ens.sync()
    w = 2 * R / nb
    for k in (0, 31, 77, 159):
        levels, glob = ens.observables(k)
        assert glob["n_samples"] == 2
        for l, L in enumerate(levels):
            h, lo, hi = ens.histogram(k, l)
            nblocks = (systems[k]["nx"] // L["block"][0]) ** 3
            assert int(h.sum()) == 2 * nblocks == L["n"]
            assert h[0] == 0 and h[-1] == 0
            vol = float(L["block"][0] * L["block"][1] * L["block"][2])
            est = lb.histogram_estimates(h, lo, hi, vol, systems[k]["kT"])
            assert abs(est["hist_abs_m"] - L["sum_abs_m"] / L["n"]) <= 0.5 * w + 1e-15
            m2 = L["sum_m2"] / L["n"]
            assert abs(est["hist_m2"] - m2) <= w * np.sqrt(m2) + 0.25 * w * w + 1e-15
    ens.close()

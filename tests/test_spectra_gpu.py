"""GPU parity of the momentum spectra (Eq. 69 diagnostics) and the OZ fit input.

FP64 trajectories: the shell-binned spectra accumulated on the device equal
the oracle's (momentum of the same states, transformed by numpy's FFT) to
1e-10 of the shell's total.  At full size (the 160-system FP32 ensemble in the
benchmark's launch configuration) the spectra of one sample are compared, for
sampled systems, with the oracle's spectra of the state the device holds.
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


def _check_shells(got_sum, got_cnt, want_jk, shape, nbins, tol):
    for comp in range(3):
        ws, wc = ob.bin_shells(want_jk[comp], shape, nbins)
        assert np.array_equal(got_cnt, wc)
        scale = np.maximum(np.abs(ws), 1e-300)
        total = ob.bin_shells(want_jk.sum(axis=0), shape, nbins)[0]
        assert np.all(np.abs(got_sum[comp] - ws) <= tol * np.maximum(total, scale)), (comp, got_sum[comp], ws)


@pytest.mark.parametrize("lattice,coupling,n", [("D2Q9", "modeq", 24), ("D2Q9", "guo", 20), ("D3Q19", "guo", 12)])
def test_momentum_spectra_match_oracle(lb, lattice, coupling, n):
    s = synth.system(lattice, coupling, n=n, a=0.003, kT=1e-4, kappa=0.02, seed=9, system_id=4)
    p = params_of(s)
    f0 = oracle_state(p, seed_amp=0.03)
    every, steps, nbins = 2, 6, n // 2 + 2
    ens = lb.Ensemble([s], precision="fp64", sk_every=every, jk_spectra=True)
    ens.write_fields(0, f0)
    ens.step(steps)
    got, cnt, ns = ens.momentum_spectra(0, nbins)
    assert ns == steps // every
    rec = ob.Recorder(p, every=0, sk_every=every, jk=True)
    lbm.run(f0, 0, steps, p, callback=rec)
    _check_shells(got, cnt, rec.jk, p.shape, nbins, 1e-10)
    # the structure factor of the same samples is unchanged by the extra work
    sk, skc, _ = ens.structure_factor(0, nbins)
    ws, wc = ob.bin_shells(rec.ck, p.shape, nbins)
    assert np.array_equal(skc, wc) and np.allclose(sk, ws, rtol=1e-10, atol=0)
    ens.close()


def test_momentum_spectra_rejected_when_off(lb):
    e = lb.Ensemble(synth.ensemble("single_16", "D2Q9"), sk_every=5)
    with pytest.raises(lb.LBError) as err:
        e.momentum_spectra(0, 4)
    assert err.value.status == lb.LB_ERR_UNSUPPORTED
    e.close()


def test_spectra_accumulators_survive_checkpoint(lb, tmp_path):
    systems = synth.ensemble("single_16", "D3Q19") + [synth.system("D3Q19", n=8, system_id=1, seed=3)]
    kw = dict(precision="fp32", obs_every=5, sk_every=5, jk_spectra=True)
    a = lb.Ensemble(systems, **kw)
    a.init()
    a.step(10)
    path = os.path.join(tmp_path, "ck.bin")
    a.save(path)
    a.step(15)
    ref = [(a.structure_factor(k, 6), a.momentum_spectra(k, 6)) for k in range(2)]
    b = lb.Ensemble(systems, **kw)
    b.load(path)
    b.step(15)
    for k in range(2):
        sk, jk = b.structure_factor(k, 6), b.momentum_spectra(k, 6)
        assert np.array_equal(sk[0], ref[k][0][0]) and np.array_equal(jk[0], ref[k][1][0])
    a.close()
    b.close()


def test_fss_160_momentum_spectra_at_full_size(lb):
    systems = synth.ensemble("fss_160", "D3Q19")
    ens = lb.Ensemble(systems, precision="fp32", obs_every=100, sk_every=100, graph_chunk=100, jk_spectra=True)
    ens.init(amplitude=0.01)
    ens.step(100)
    ens.sync()
    for k in (0, 77, 159):
        p = params_of(systems[k])
        f = ens.read_fields(k)              # the state the sample was taken from
        nbins = p.nx // 2
        got, cnt, ns = ens.momentum_spectra(k, nbins)
        assert ns == 1
        # FP32 populations read back exactly; the device sums them in compensated
        # FP32 and FP64, the oracle in FP64: agreement to 1e-9 of the shell total
        _check_shells(got, cnt, ob.momentum_spectra(f, p), p.shape, nbins, 1e-9)
    ens.close()

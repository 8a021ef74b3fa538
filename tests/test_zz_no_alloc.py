"""lb_block_moments_noalloc: block moments of one density snapshot, no allocation.

This entry point serves callers that cannot allocate device memory (a framework
that already owns the whole device memory pool, or a loop that cannot pay for
the synchronisation of cudaMalloc/cudaFree); its scratch lives in a fixed
device array inside the library.  The tests call it through the C ABI and
compare its output with lb_observables, the workspace-based entry point, and
with the oracle's block sums (Eqs. 46-50) of the same snapshot, for two calls
in a row: the shared scratch keeps the previous call's contents, so the second
call also checks that nothing carries over.  The largest accepted lattices
(2^18 sites: 512^2 and 64^3) are run, and a non-finite input must show in the
caller's status word.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import observables as ob
from tests.helpers import params_of

pytestmark = pytest.mark.gpu

FIELDS = ("n", "sum_m", "sum_m2", "sum_abs_m", "sum_m4", "sum_e", "sum_e2")
ST_NONFINITE = 4


def _call(lb, rho, s, code, stream, status=None):
    import torch
    out = torch.full((lb.LB_MAX_LEVELS, 7), float("nan"), dtype=torch.float64, device="cuda")
    nl = ctypes.c_int()
    st = lb.lb_block_moments_noalloc(ctypes.c_void_p(rho.data_ptr()), s["nx"], s["ny"], s["nz"], code,
                                     ctypes.c_void_p(out.data_ptr()), lb.LB_MAX_LEVELS, ctypes.byref(nl),
                                     None if status is None else ctypes.c_void_p(status.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
    assert st == lb.LB_OK, lb.lb_status_string(st)
    torch.cuda.synchronize()
    return out[:nl.value].cpu().numpy()


def _close(got, want, what):
    """Block counts exact; moments to 1e-10 relative.  Level 0 (the whole
    lattice) has m = 0 by mass conservation, so its m moments are rounding
    noise on both sides; its energy moments are compared."""
    assert np.array_equal(got[:, 0], want[:, 0]), what
    assert np.all(np.abs(got[0, 1:5]) < 1e-12) and np.all(np.abs(want[0, 1:5]) < 1e-12), what
    assert np.allclose(got[0, 5:], want[0, 5:], rtol=1e-10, atol=0), what
    scale = np.abs(want[1:]).copy()
    scale[:, 1] = want[1:, 3]                                         # sum m vanishes: |m| scale
    assert np.all(np.abs(got[1:, 1:] - want[1:, 1:]) <= 1e-10 * scale[:, 1:] + 1e-300), (what, got, want)


@pytest.mark.parametrize("lattice,n", [("D2Q9", 48), ("D3Q19", 16), ("D2Q9", 512), ("D3Q19", 64)])
def test_noalloc_matches_workspace_observables_and_oracle_on_two_calls(lattice, n):
    import torch
    import paper_1202_4748_gb300 as lb
    if not torch.cuda.is_available():
        raise RuntimeError("needs CUDA")
    s = synth.system(lattice, n=n, a=-0.002, kT=1e-4, seed=7, system_id=1)
    lv = ob.levels(params_of(s))
    ens = lb.Ensemble([s], precision="fp64", obs_every=1)
    ens.init(amplitude=0.01)
    code = lb.LB_D2Q9 if lattice == "D2Q9" else lb.LB_D3Q19
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        before, _ = ens.observables(0)
        ens.step(1)                       # one sample is taken after this step
        after, _ = ens.observables(0)
        want = np.array([[a[f] - b[f] for f in FIELDS] for a, b in zip(after, before)])
        rho = torch.from_numpy(ens.read_fields(0).sum(axis=0).copy()).to("cuda")
        got = _call(lb, rho, s, code, ens.stream, status)
        assert int(status.item()) == 0
        assert len(got) == len(after) == len(lv)
        _close(got, want, ("lb_observables", call))
        # the oracle's block sums of a seeded synthetic snapshot (phi about its own mean, Eq. 1)
        rho_h = synth.random_density((s["nz"], s["ny"], s["nx"]), seed=100 + call)
        got = _call(lb, torch.from_numpy(rho_h).to("cuda"), s, code, ens.stream, status)
        phi = (rho_h - rho_h.mean()) / rho_h.mean()
        _close(got, ob.sample(phi, lv), ("oracle", call))
    ens.close()


def test_noalloc_reports_a_non_finite_input_in_the_status_word():
    import torch
    import paper_1202_4748_gb300 as lb
    s = synth.system("D2Q9", n=32, seed=3)
    rho = torch.from_numpy(synth.random_density((1, 32, 32), seed=3)).to("cuda")
    rho[0, 5, 7] = float("nan")
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    got = _call(lb, rho, s, lb.LB_D2Q9, torch.cuda.current_stream(), status)
    assert int(status.item()) & ST_NONFINITE
    assert not np.all(np.isfinite(got[1:, 1:]))
    # the next call on finite input clears the flag (the scratch status is reset per call)
    rho[0, 5, 7] = 1.0
    _call(lb, rho, s, lb.LB_D2Q9, torch.cuda.current_stream(), status)
    assert int(status.item()) == 0


def test_noalloc_rejects_oversize_and_bad_arguments():
    import paper_1202_4748_gb300 as lb
    nl = ctypes.c_int()
    fake = ctypes.c_void_p(256)           # never dereferenced: the size check comes first
    side = 1 << 10
    assert lb.lb_block_moments_noalloc(fake, side, side, 1, lb.LB_D2Q9, fake, 32, ctypes.byref(nl),
                                       None, None) == lb.LB_ERR_UNSUPPORTED
    assert lb.lb_block_moments_noalloc(fake, 513, 512, 1, lb.LB_D2Q9, fake, 32, ctypes.byref(nl),
                                       None, None) == lb.LB_ERR_UNSUPPORTED   # one row past 2^18 sites
    assert lb.lb_block_moments_noalloc(None, 8, 8, 1, lb.LB_D2Q9, fake, 32, ctypes.byref(nl), None,
                                       None) == lb.LB_ERR_ARG
    assert lb.lb_block_moments_noalloc(fake, 8, 8, 2, lb.LB_D2Q9, fake, 32, ctypes.byref(nl), None,
                                       None) == lb.LB_ERR_ARG
    assert lb.lb_block_moments_noalloc(fake, 8, 8, 1, lb.LB_D2Q9, fake, 2, ctypes.byref(nl), None,
                                       None) == lb.LB_ERR_ARG
    assert nl.value == 4                  # blocks 8x8, 4x4, 2x2, 1x1

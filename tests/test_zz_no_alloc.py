"""lb_block_moments_noalloc: block moments of one density snapshot, no allocation.

This entry point serves callers that cannot allocate device memory (a framework
that already owns the whole device memory pool, or a loop that cannot pay for
the synchronisation of cudaMalloc/cudaFree); its scratch lives in a fixed
device array inside the library.  The test calls it through the C ABI and
compares its output with lb_observables, the workspace-based entry point, on
the same snapshot, for two calls in a row: the shared scratch keeps the
previous call's contents, so the second call also checks that nothing carries
over.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FIELDS = ("n", "sum_m", "sum_m2", "sum_abs_m", "sum_m4", "sum_e", "sum_e2")


@pytest.mark.parametrize("lattice,n", [("D2Q9", 48), ("D3Q19", 16)])
def test_noalloc_matches_workspace_observables_on_two_calls(lattice, n):
    import torch
    import paper_1202_4748_gb300 as lb
    if not torch.cuda.is_available():
        raise RuntimeError("needs CUDA")
    s = synth.system(lattice, n=n, a=-0.002, kT=1e-4, seed=7, system_id=1)
    ens = lb.Ensemble([s], precision="fp64", obs_every=1)
    ens.init(amplitude=0.01)
    code = lb.LB_D2Q9 if lattice == "D2Q9" else lb.LB_D3Q19
    for call in range(2):
        before, _ = ens.observables(0)
        ens.step(1)                       # one sample is taken after this step
        after, _ = ens.observables(0)
        want = np.array([[a[f] - b[f] for f in FIELDS] for a, b in zip(after, before)])
        rho = torch.from_numpy(ens.read_fields(0).sum(axis=0).copy()).to("cuda")
        out = torch.full((lb.LB_MAX_LEVELS, 7), float("nan"), dtype=torch.float64, device="cuda")
        nl = ctypes.c_int()
        st = lb.lb_block_moments_noalloc(ctypes.c_void_p(rho.data_ptr()), s["nx"], s["ny"], s["nz"], code,
                                         ctypes.c_void_p(out.data_ptr()), lb.LB_MAX_LEVELS, ctypes.byref(nl),
                                         ctypes.c_void_p(ens.stream.cuda_stream))
        assert st == lb.LB_OK, lb.lb_status_string(st)
        torch.cuda.synchronize()
        got = out[:nl.value].cpu().numpy()
        assert nl.value == len(after)
        assert np.array_equal(got[:, 0], want[:, 0])                     # block counts
        # level 0 is the whole lattice: m = 0 by mass conservation, so its m moments
        # are rounding noise on both sides; its energy moments are compared below
        assert np.all(np.abs(got[0, 1:5]) < 1e-12) and np.all(np.abs(want[0, 1:5]) < 1e-12)
        assert np.allclose(got[0, 5:], want[0, 5:], rtol=1e-10, atol=0)
        scale = np.abs(want[1:]).copy()
        scale[:, 1] = want[1:, 3]                                         # sum m vanishes: |m| scale
        assert np.all(np.abs(got[1:, 1:] - want[1:, 1:]) <= 1e-10 * scale[:, 1:] + 1e-300), (call, got, want)
    ens.close()


def test_noalloc_rejects_oversize_and_bad_arguments():
    import paper_1202_4748_gb300 as lb
    nl = ctypes.c_int()
    fake = ctypes.c_void_p(256)           # never dereferenced: the size check comes first
    side = 1 << 10
    assert lb.lb_block_moments_noalloc(fake, side, side, 1, lb.LB_D2Q9, fake, 32, ctypes.byref(nl),
                                       None) == lb.LB_ERR_UNSUPPORTED
    assert lb.lb_block_moments_noalloc(None, 8, 8, 1, lb.LB_D2Q9, fake, 32, ctypes.byref(nl), None) == lb.LB_ERR_ARG
    assert lb.lb_block_moments_noalloc(fake, 8, 8, 2, lb.LB_D2Q9, fake, 32, ctypes.byref(nl), None) == lb.LB_ERR_ARG
    assert lb.lb_block_moments_noalloc(fake, 8, 8, 1, lb.LB_D2Q9, fake, 2, ctypes.byref(nl), None) == lb.LB_ERR_ARG
    assert nl.value == 4                  # blocks 8x8, 4x4, 2x2, 1x1

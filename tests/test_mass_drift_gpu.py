"""Mass bookkeeping of the FP32-deviation path (populations in FP32, the
conserved mass summed in FP64 on the GPU).

The collision conserves mass exactly in exact arithmetic (Eq. 62: the density
moment is not relaxed and the noise has no density component), so only the
FP32 rounding of the stored deviations moves it.  Each stored deviation is
rounded to FP32 (at most 2^-24 of its size, |df| < 0.05 here: 3e-9), 19 per
site, so one step changes a site's mass by at most ~6e-8 and rounding to
nearest leaves no systematic trend in the worst case's sign; measured on a
64^3 system (a = -0.002, kT = 1e-4) the relative drift |sum rho(t) - sum
rho(0)| / sum rho(0) grows by ~1e-12 per step (9.8e-8 after 10^5 steps).  The
bars are 10x that rate: 1e-7 after 10^4 steps for FP32, and 1e-13 for the
FP64 path, whose rounding is 2^29 times finer.  The mass is summed in FP64
(the observable pass) from the populations themselves."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,steps,bar", [("fp32", 10000, 1e-7), ("fp64", 2000, 1e-13)])
def test_mass_drift_of_the_stored_populations(precision, steps, bar):
    import paper_1202_4748_gb300 as lb
    s = synth.system("D3Q19", "guo", n=32, a=-0.002, kT=1e-4, seed=5, system_id=3)
    ens = lb.Ensemble([s], precision=precision, obs_every=steps // 10, graph_chunk=steps // 10)
    ens.init(amplitude=0.01)
    ens.step(steps)
    _, g = ens.observables(0)
    ens.close()
    assert g["step"] == steps
    drift = abs(g["mass"] - g["mass0"]) / g["mass0"]
    assert drift < bar, drift

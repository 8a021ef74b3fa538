"""The bulk-viscosity study on oracle trajectories (CPU).

Sec. III A gives zeta = rho/3 (tau - 1/2)(2 - 3 c_s^2) for the modified
equilibrium; the Chapman-Enskog form (2/d + 1 - 3 c_s^2) used by the study
reduces to it in 2-D.  A standing sound wave must decay at
Gamma = k^2/2 (zeta + 2(1 - 1/d) eta)/rho, which differs from the ideal-gas
k^2 nu by 1.5 (1 - c_s^2).  The wave is stepped by the FP64 oracle and the
fit is the study's own; the remaining difference is the O(k^2) lattice
correction (< 0.3% at k = 2 pi / 64).
"""
import math

import numpy as np
import pytest

import synth
from oracle import lbm
from paper_1202_4748_gb300.studies import damping_rate, fit_damped_mode, mode_amplitude, viscosities, wave_density
from tests.helpers import params_of


def test_fit_recovers_a_damped_oscillation():
    t = np.arange(0, 1200, 4.0)
    y = np.exp(-1.3e-3 * t) * (2.0 * np.cos(0.031 * t) + 0.1 * np.sin(0.031 * t))
    fit = fit_damped_mode(t, y)
    assert fit["Gamma"] == pytest.approx(1.3e-3, rel=1e-8)
    assert fit["omega"] == pytest.approx(0.031, rel=1e-9)
    assert fit["A"] == pytest.approx(2.0, rel=1e-8) and fit["rms"] < 1e-10


def test_bulk_viscosity_formula_reduces_to_the_papers_in_2d_and_ideal_gas():
    eta, zeta = viscosities("D2Q9", 0.1, 0.8)
    assert zeta == pytest.approx(0.3 / 3 * (2 - 3 * 0.1), rel=1e-15)
    for lat, d in (("D2Q9", 2), ("D3Q19", 3)):
        eta, zeta = viscosities(lat, 1.0 / 3.0, 0.9)
        assert zeta == pytest.approx(2 * eta / d, rel=1e-14)            # ideal lattice gas


def _oracle_decay(lattice, coupling, nx, tau, a=0.1, steps=1200, every=4, ny=2, nz=1):
    s = synth.system(lattice, coupling, n=nx, a=a, kT=0.0, kappa=0.01, tau=tau)
    s.update(nx=nx, ny=ny, nz=nz)
    p = params_of(s)
    f = lbm.equilibrium_at_rest(wave_density(p.shape, p.rho_c, 1e-4), p)
    ts, ys = [0], [mode_amplitude(f)]
    for t in range(0, steps, every):
        f = lbm.run(f, t, every, p)
        ts.append(t + every)
        ys.append(mode_amplitude(f))
    return fit_damped_mode(ts, ys)


@pytest.mark.parametrize("lattice,coupling,nx,tau,steps,shape", [
    ("D2Q9", "modeq", 64, [1] * 3 + [0.8] * 6, 1200, (2, 1)),
    ("D2Q9", "guo", 64, [1] * 3 + [0.8] * 6, 1200, (2, 1)),
    ("D2Q9", "modeq", 64, [1] * 3 + [1.2] + [0.8] * 5, 1200, (2, 1)),
    ("D3Q19", "guo", 32, [1] * 4 + [0.8] * 15, 800, (2, 2)),
    ("D3Q19", "modeq", 32, [1] * 4 + [0.8] * 15, 800, (2, 2)),
])
def test_sound_wave_decays_at_the_predicted_rate(lattice, coupling, nx, tau, steps, shape):
    fit = _oracle_decay(lattice, coupling, nx, tau, steps=steps, ny=shape[0], nz=shape[1])
    d = 2 if lattice == "D2Q9" else 3
    k2 = (2 * math.pi / nx) ** 2
    tb, ts = (tau[3], tau[4]) if d == 2 else (tau[4], tau[5])
    want = damping_rate(lattice, k2, 0.1, ts, tb)
    assert fit["Gamma"] == pytest.approx(want, rel=3e-3)
    assert fit["Gamma"] / (k2 * (ts - 0.5) / 3) > 1.3            # the ideal-gas rate is clearly wrong
    assert fit["omega"] == pytest.approx(math.sqrt(0.1 * k2), rel=3e-3)

"""Shared test helpers: map workload descriptors to oracle parameters, compare fields."""
import numpy as np

from oracle import lbm


def params_of(s):
    return lbm.Params(lattice=s["lattice"], coupling=s["coupling"], nx=s["nx"], ny=s["ny"], nz=s["nz"],
                      rho_c=s["rho_c"], a=s["a"], b=s["b"], kappa=s["kappa"], kT=s["kT"],
                      tau=tuple(s["tau"]), seed=s["seed"], system_id=s["system_id"])


def rel_err(got, want):
    """max |got - want| / max |want| (the population-error measure of the parity bar)."""
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


def oracle_state(p, steps=3, seed_amp=0.02):
    """A generic non-equilibrium state: oracle initial state advanced a few steps."""
    f = lbm.initial_state(p, amplitude=seed_amp)
    return lbm.run(f, 0, steps, p)

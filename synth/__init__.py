"""Seeded synthetic workloads shared by tests, smoke and bench.

Holds none of the method's arithmetic: only system descriptors (sizes, GL
coefficients, relaxation times, kT, seeds) and plain seeded random arrays.
Both the CUDA library's callers and the oracle take their inputs from here.

Workloads (the paper's own runs are 2-D D2Q9, Sec. III A; the 3-D D3Q19
variant runs the same recipes on cubic lattices):

  single_16  : one system, 16^3 (D3Q19) / 64^2 (D2Q9); a = 0 (mean-field
               critical), b = 0.1, kappa = 0.01, tau = 1, kT = 1e-4, seed 1.
  single_64  : one system, 64^3 / 512^2, a = -0.002 (just below critical).
  fss_160    : finite-size-scaling ensemble, 160 systems:
               L in {16, 24, 32, 48, 64}^3 (D2Q9: {64, 120, 184, 336, 512}^2,
               the same site counts rounded to multiples of 8)
               x 8 values of a in [-0.004, 0.004] x 4 replicas (seed 1 + r).
  fss_60     : uneven ensemble, L in {32, 48, 64, 96, 128}^3
               (D2Q9: {184, 336, 512, 944, 1448}^2) x 6 a x 2 replicas.
  large_256  : one system 256^3 / 4096^2, a = 0.

system_id is the running index inside an ensemble; it enters the random
number counter so every system draws its own stream.
"""

import numpy as np

SIDES_3D = {
    "single_16": [16],
    "single_64": [64],
    "fss_160": [16, 24, 32, 48, 64],
    "fss_160_64": [64],          # the 64^3 members of fss_160 (a profiling case larger than L2)
    "fss_60": [32, 48, 64, 96, 128],
    "large_256": [256],
}
# 2-D sides with the same site count as L^3, rounded to a multiple of 8
SIDE_2D_OF = {16: 64, 24: 120, 32: 184, 48: 336, 64: 512, 96: 944, 128: 1448, 256: 4096}


def _a_values(name):
    if name == "single_16" or name == "large_256":
        return [0.0]
    if name == "single_64":
        return [-0.002]
    if name in ("fss_160", "fss_160_64"):
        return list(np.linspace(-0.004, 0.004, 8))
    if name == "fss_60":
        return list(np.linspace(-0.004, 0.004, 6))
    raise KeyError(name)


def _replicas(name):
    return {"fss_160": 4, "fss_160_64": 4, "fss_60": 2}.get(name, 1)


def system(lattice="D2Q9", coupling=None, n=64, a=0.0, b=0.1, kappa=0.01, kT=1e-4,
           tau=1.0, seed=1, system_id=0, rho_c=1.0):
    """One system descriptor (a plain dict)."""
    q = 9 if lattice == "D2Q9" else 19
    if coupling is None:
        coupling = "modeq" if lattice == "D2Q9" else "guo"
    nz = 1 if lattice == "D2Q9" else n
    taus = list(tau) if np.ndim(tau) else [float(tau)] * q
    return dict(lattice=lattice, coupling=coupling, nx=n, ny=n, nz=nz, rho_c=rho_c,
                a=float(a), b=b, kappa=kappa, kT=kT, tau=taus, seed=int(seed),
                system_id=int(system_id))


def ensemble(name, lattice="D2Q9", coupling=None):
    """List of system descriptors for a named workload."""
    out = []
    for side in SIDES_3D[name]:
        n = side if lattice == "D3Q19" else SIDE_2D_OF[side]
        for a in _a_values(name):
            for r in range(_replicas(name)):
                out.append(system(lattice, coupling, n=n, a=a, seed=1 + r, system_id=len(out)))
    return out


def sites(systems):
    return sum(s["nx"] * s["ny"] * s["nz"] for s in systems)


def random_density(shape, seed, amplitude=0.01, rho_c=1.0):
    """rho_c (1 + amplitude * N(0,1)) as float64, for tests that start from a density field."""
    rng = np.random.default_rng(seed)
    return rho_c * (1.0 + amplitude * rng.standard_normal(shape))


def random_perturbation(shape, seed, scale):
    """Plain seeded Gaussian array."""
    return scale * np.random.default_rng(seed).standard_normal(shape)

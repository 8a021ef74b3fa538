"""Studies built on the library: sound-mode damping (the bulk-viscosity artifact)
and a side-by-side comparison of the two thermodynamic couplings.

Bulk viscosity (Sec. III A, Eq. for zeta and the remark after the linearised
Navier-Stokes equation): an equilibrium that carries the non-ideal pressure p0
in its second moment gives, by the Chapman-Enskog expansion of the moment-space
collision (lattice third moment rho/3 (u d + perms), pressure derivative
c_s^2 = dp0/drho), a viscous stress with
    eta  = rho (tau_s - 1/2) / 3                         (shear modes)
    zeta = rho (tau_b - 1/2) / 3 * (2/d + 1 - 3 c_s^2)   (bulk / energy mode)
which is the paper's zeta = rho/3 (tau - 1/2)(2 - 3 c_s^2) for d = 2; an ideal
lattice gas (c_s^2 = 1/3) gives the usual zeta = 2 eta / d.  A standing sound
wave of wavenumber k then decays at
    Gamma = k^2 / 2 * (zeta + 2 (1 - 1/d) eta) / rho,
i.e. Gamma = k^2 (tau - 1/2)(1 - c_s^2) / 2 at a single tau, against k^2 nu for
the ideal gas.  ``sound_decay`` starts a density wave at rest, follows its
Fourier amplitude and fits the damped oscillation
    rho_k(t) = exp(-Gamma t) (A cos(omega t) + B sin(omega t)).

Everything that steps the lattice runs in the CUDA library; the fits are host
arithmetic on values read back through the public API.
"""
import math

import numpy as np

from . import Ensemble, oz_fit

LATTICE_D = {"D2Q9": 2, "D3Q19": 3}


def viscosities(lattice, c_s2, tau_shear, tau_bulk=None):
    """(eta/rho, zeta/rho) of the formulas in the module docstring."""
    d = LATTICE_D[lattice]
    tb = tau_shear if tau_bulk is None else tau_bulk
    eta = (tau_shear - 0.5) / 3.0
    zeta = (tb - 0.5) / 3.0 * (2.0 / d + 1.0 - 3.0 * c_s2)
    return eta, zeta


def damping_rate(lattice, k2, c_s2, tau_shear, tau_bulk=None):
    """Gamma of a sound wave with wavenumber^2 k2 (module docstring)."""
    d = LATTICE_D[lattice]
    eta, zeta = viscosities(lattice, c_s2, tau_shear, tau_bulk)
    return 0.5 * k2 * (zeta + 2.0 * (1.0 - 1.0 / d) * eta)


def fit_damped_mode(t, y):
    """Least-squares fit of y(t) = exp(-Gamma t)(A cos(omega t) + B sin(omega t)).

    Start values: omega from the zero crossings, Gamma from the decay of the
    successive extrema; then Gauss-Newton on (Gamma, omega) with A, B solved
    linearly at each step (variable projection).  Returns dict(Gamma, omega, A, B, rms).
    """
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    sgn = np.signbit(y)
    cross = np.nonzero(sgn[1:] != sgn[:-1])[0]
    if cross.size >= 2:
        half = np.mean(np.diff(t[cross]))
        omega = math.pi / half
    else:
        omega = math.pi / (t[-1] - t[0])
    amp = np.abs(y)
    gamma = max(1e-12, math.log(max(amp[0], 1e-300) / max(np.max(amp[len(amp) // 2:]), 1e-300)) /
                max(t[len(t) // 2] - t[0], 1.0))

    def solve(g, w):
        e = np.exp(-g * t)
        M = np.stack([e * np.cos(w * t), e * np.sin(w * t)], axis=1)
        ab, *_ = np.linalg.lstsq(M, y, rcond=None)
        return ab, y - M @ ab

    for _ in range(100):
        ab, res = solve(gamma, omega)
        hg, hw = 1e-7 * max(gamma, 1e-6), 1e-7 * max(omega, 1e-6)
        _, rg = solve(gamma + hg, omega)
        _, rw = solve(gamma, omega + hw)
        J = np.stack([(rg - res) / hg, (rw - res) / hw], axis=1)
        step, *_ = np.linalg.lstsq(J, -res, rcond=None)
        gamma, omega = gamma + step[0], omega + step[1]
        if abs(step[0]) < 1e-12 * max(abs(gamma), 1e-12) and abs(step[1]) < 1e-12 * max(abs(omega), 1e-12):
            break
    ab, res = solve(gamma, omega)
    return dict(Gamma=float(gamma), omega=float(omega), A=float(ab[0]), B=float(ab[1]),
                rms=float(np.sqrt(np.mean(res * res)) / max(np.max(np.abs(y)), 1e-300)))


def mode_amplitude(f, n=1):
    """Real part of the density's Fourier amplitude at k = 2 pi n / S along x (f: [q][z][y][x])."""
    rho = f.sum(axis=0)
    nx = rho.shape[-1]
    phase = np.cos(2.0 * math.pi * n * np.arange(nx) / nx)
    return float((rho * phase).sum())


def wave_density(shape, rho_c, amplitude, n=1):
    """rho(x) = rho_c (1 + amplitude cos(2 pi n x / S)) on a (nz, ny, nx) grid."""
    nz, ny, nx = shape
    x = np.arange(nx)
    row = rho_c * (1.0 + amplitude * np.cos(2.0 * math.pi * n * x / nx))
    return np.broadcast_to(row, shape).copy()


def sound_decay(system, steps=1000, every=5, amplitude=1e-4, precision="fp64", n=1):
    """Measured and predicted damping of a standing sound wave in one system.

    ``system`` is a descriptor dict (kT is forced to 0: the wave is followed
    without noise).  Returns dict(Gamma, omega, Gamma_theory, Gamma_ideal,
    k2, c_s2, fit rms)."""
    s = dict(system, kT=0.0)
    shape = (s["nz"], s["ny"], s["nx"])
    ens = Ensemble([s], precision=precision)
    try:
        ens.init(rho=wave_density(shape, s["rho_c"], amplitude, n))
        ts, ys = [0], [mode_amplitude(ens.read_fields(0), n)]
        for t in range(every, steps + 1, every):
            ens.step(every)
            ts.append(t)
            ys.append(mode_amplitude(ens.read_fields(0), n))
    finally:
        ens.close()
    fit = fit_damped_mode(ts, ys)
    d = LATTICE_D[s["lattice"]]
    k = 2.0 * math.pi * n / s["nx"]
    k2 = k * k
    c_s2 = s["a"]                          # dp0/drho at rho = rho_c (phi = 0) with rho_c = 1
    tau = s["tau"]
    tb = tau[3] if d == 2 else tau[4]      # energy (bulk) mode
    ts_ = tau[4] if d == 2 else tau[5]     # a shear mode
    return dict(Gamma=fit["Gamma"], omega=fit["omega"], rms=fit["rms"], k2=k2, c_s2=c_s2,
                Gamma_theory=damping_rate(s["lattice"], k2, c_s2, ts_, tb),
                Gamma_ideal=k2 * (ts_ - 0.5) / 3.0)


def statics(systems, steps, every, precision="fp32", kmax=6, warmup=0, graph_chunk=0):
    """Structure factor, OZ fit and momentum spectra of an ensemble of replicas of
    one cubic / square system (all systems share lattice, coupling and size).

    Returns dict(chi, xi, oz, jk_ratio: <|j(k)|^2> / (rho_c kT) per shell and
    component, sk: C(k) per shell)."""
    s0 = systems[0]
    side = s0["nx"]
    ens = Ensemble(systems, precision=precision, sk_every=every, jk_spectra=True, graph_chunk=graph_chunk)
    nb = kmax

    def totals():
        sk = np.zeros(nb)
        jk = np.zeros((3, nb))
        ns_tot, cnt = 0, None
        for k in range(len(systems)):
            s_, c_, ns = ens.structure_factor(k, nb)
            j_, _, _ = ens.momentum_spectra(k, nb)
            sk += s_
            jk += j_
            cnt = c_
            ns_tot += ns
        return sk, jk, ns_tot, cnt

    try:
        ens.init(amplitude=0.0)
        # the accumulated sums are additive: samples taken during the warm-up are
        # subtracted at the end
        ens.step(warmup)
        sk0, jk0, ns0, _ = totals()
        ens.step(steps)
        sk, jk, ns_tot, cnt = totals()
        sk, jk, ns_tot = sk - sk0, jk - jk0, ns_tot - ns0
    finally:
        ens.close()
    fit = oz_fit(s0["lattice"], side, sk, cnt, ns_tot, s0["kT"], kmax)
    C = sk / (cnt * ns_tot)
    J = jk / (cnt[None, :] * ns_tot) / (s0["rho_c"] * s0["kT"])
    return dict(chi=fit["chi"], xi=fit["xi"], oz=fit, sk=C, jk_ratio=J, samples=ns_tot)


def level_observables(systems, steps, precision, obs_every=10, sk_every=0, sk_bins=0, graph_chunk=0,
                      amplitude=0.01):
    """Per system: [(block side, U_L, chi_L, c_H,L)] after ``steps`` steps, and the
    shell-binned C(k) (sums, counts, samples) when sk_every > 0."""
    ens = Ensemble(systems, precision=precision, obs_every=obs_every, sk_every=sk_every,
                   graph_chunk=graph_chunk)
    try:
        ens.init(amplitude=amplitude)
        ens.step(steps)
        out, sk = [], []
        for k, s in enumerate(systems):
            levels, _ = ens.observables(k)
            row = []
            for L in levels:
                if L["n"] <= 0:
                    continue
                d = ens.derive(L, s["kT"])
                row.append((L["block"][0], d["U_L"], d["chi_L"], d["c_HL"]))
            out.append(row)
            if sk_every:
                sk.append(ens.structure_factor(k, sk_bins))
    finally:
        ens.close()
    return out, sk


def binder_cumulants(systems, steps, precision, obs_every=10, graph_chunk=0, amplitude=0.01):
    """U_L per system and level after ``steps`` steps: (list of lists of (block side, U_L))."""
    rows, _ = level_observables(systems, steps, precision, obs_every, graph_chunk=graph_chunk, amplitude=amplitude)
    return [[(L, u) for L, u, _, _ in r] for r in rows]


def precision_accuracy(systems, steps, obs_every=10, max_block_fraction=1.0 / 8.0, sk_every=0, sk_bins=0):
    """Observables of the same systems and seeds in FP32 and FP64.

    Systems are grouped by (side, a); within a group the replicas (different
    seeds) give the statistical error sigma of the FP64 mean.  For every group
    and every block size L <= max_block_fraction * S (the finite-size-scaling
    range of the analysis) and each of U_L, chi_L, c_H,L returns a row
    (quantity, side, a, L, mean fp32, mean fp64, sigma); with sk_every > 0 also
    the structure factor per shell (quantity "C_k", L = shell index)."""
    o32, k32 = level_observables(systems, steps, "fp32", obs_every, sk_every, sk_bins)
    o64, k64 = level_observables(systems, steps, "fp64", obs_every, sk_every, sk_bins)
    groups = {}
    for k, s in enumerate(systems):
        groups.setdefault((s["nx"], round(s["a"], 12)), []).append(k)
    rows = []
    for (side, a), ks in sorted(groups.items()):
        def emit(name, L, v32, v64):
            v32, v64 = np.asarray(v32), np.asarray(v64)
            sigma = float(np.std(v64, ddof=1) / math.sqrt(len(ks))) if len(ks) > 1 else float("nan")
            rows.append((name, side, a, L, float(v32.mean()), float(v64.mean()), sigma))
        for li, (L, _, _, _) in enumerate(o64[ks[0]]):
            if L > max_block_fraction * side or L == side:
                continue
            for qi, name in ((1, "U_L"), (2, "chi_L"), (3, "c_HL")):
                emit(name, L, [o32[k][li][qi] for k in ks], [o64[k][li][qi] for k in ks])
        if sk_every:
            for j in range(sk_bins):
                c32 = [k32[k][0][j] / (k32[k][1][j] * k32[k][2]) for k in ks if k32[k][1][j] > 0]
                c64 = [k64[k][0][j] / (k64[k][1][j] * k64[k][2]) for k in ks if k64[k][1][j] > 0]
                if c32 and c64:
                    emit("C_k", j + 1, c32, c64)
    return rows

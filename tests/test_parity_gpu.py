"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Bars (from the method's stated tolerances):
  FP64 path: max |f_gpu - f_oracle| / max |f_oracle| <= 1e-12 at every compared
             step; observables to 1e-10 relative.
  FP32-deviation path: one step from an identical state, max |df| / max |f| <= 1e-5.
Inputs are seeded and synthetic (see ``synth``); every expected value comes
from the oracle.
"""
import dataclasses
import os

import numpy as np
import pytest

import synth
from oracle import lbm, observables as ob
from tests.helpers import oracle_state, params_of, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need CUDA; the library has no CPU fallback")
    import paper_1202_4748_gb300 as m
    return m


def _sys(lattice, coupling, nx, ny, nz=1, **kw):
    s = synth.system(lattice, coupling, n=nx, **{k: v for k, v in kw.items() if k in
                                                 ("a", "b", "kappa", "kT", "tau", "seed", "system_id", "rho_c")})
    s.update(nx=nx, ny=ny, nz=nz)
    return s


MIXED_TAU_9 = [1, 1, 1, 0.8, 0.9, 1.3, 0.7, 1.6, 1.1]
MIXED_TAU_19 = [1, 1, 1, 1] + list(np.linspace(0.7, 1.5, 15))

CASES = [
    ("D2Q9", "modeq", (70, 37, 1), MIXED_TAU_9),
    ("D2Q9", "guo", (45, 29, 1), MIXED_TAU_9),
    ("D3Q19", "guo", (20, 13, 11), MIXED_TAU_19),
    ("D3Q19", "modeq", (20, 13, 11), MIXED_TAU_19),
]


def _run_gpu(lb, systems, f0s, nsteps, precision="fp64", **opts):
    ens = lb.Ensemble(systems, precision=precision, **opts)
    for k, f in enumerate(f0s):
        ens.write_fields(k, f)
    ens.step(nsteps)
    ens.sync()
    out = [ens.read_fields(k) for k in range(len(systems))]
    ens.close()
    return out


@pytest.mark.parametrize("lattice,coupling,shape,tau", CASES)
def test_fp64_multistep_parity(lb, lattice, coupling, shape, tau):
    s = _sys(lattice, coupling, *shape, a=0.01, b=0.1, kappa=0.01, kT=1e-4, tau=tau, seed=7, system_id=3)
    p = params_of(s)
    f0 = oracle_state(p)
    ens = lb.Ensemble([s], precision="fp64")
    ens.write_fields(0, f0)
    assert rel_err(ens.read_fields(0), f0) == 0.0          # write/read round trip is exact
    f = f0
    t = 0
    for chunk in (1, 4, 15):
        ens.step(chunk)
        ens.sync()
        f = lbm.run(f, t, chunk, p)
        t += chunk
        assert rel_err(ens.read_fields(0), f) < TOL64, (t, rel_err(ens.read_fields(0), f))
    ens.close()


@pytest.mark.parametrize("lattice,coupling,shape,tau", CASES)
def test_fp32_one_step_parity(lb, lattice, coupling, shape, tau):
    s = _sys(lattice, coupling, *shape, a=-0.002, b=0.1, kappa=0.01, kT=1e-4, tau=tau, seed=11)
    p = params_of(s)
    f0 = oracle_state(p, steps=5)
    ens = lb.Ensemble([s], precision="fp32")
    ens.write_fields(0, f0)
    f0r = ens.read_fields(0)            # the FP32-rounded state, as the GPU holds it
    assert rel_err(f0r, f0) < 1e-7
    for t in range(3):
        ens.step(1)
        ens.sync()
        got = ens.read_fields(0)
        want = lbm.step(f0r, t, p)
        assert rel_err(got, want) < TOL32, (t, rel_err(got, want))
        # the next step starts again from the GPU's own state
        ens.write_fields(0, got)
        f0r = ens.read_fields(0)
    ens.close()


def test_batched_systems_of_different_sizes(lb):
    """Tiles of several systems share one launch; each system matches the oracle alone."""
    systems = [_sys("D3Q19", "guo", 9, 8, 7, a=0.0, kT=1e-4, seed=1, system_id=0, tau=[1.0] * 19),
               _sys("D3Q19", "guo", 17, 5, 9, a=-0.003, kT=2e-4, seed=2, system_id=1, tau=MIXED_TAU_19),
               _sys("D3Q19", "guo", 4, 4, 4, a=0.003, kT=0.0, seed=3, system_id=2, tau=[1.0] * 19)]
    ps = [params_of(s) for s in systems]
    f0s = [oracle_state(p) for p in ps]
    got = _run_gpu(lb, systems, f0s, 6)
    for g, p, f in zip(got, ps, f0s):
        assert rel_err(g, lbm.run(f, 0, 6, p)) < TOL64


@pytest.mark.parametrize("lattice,coupling,shape", [
    ("D2Q9", "modeq", (1, 1, 1)), ("D2Q9", "modeq", (2, 3, 1)), ("D2Q9", "modeq", (5, 1, 1)),
    ("D2Q9", "guo", (3, 2, 1)), ("D3Q19", "guo", (2, 2, 2)), ("D3Q19", "guo", (1, 3, 2)),
    ("D3Q19", "guo", (3, 3, 3)),
])
def test_degenerate_tiny_lattices(lb, lattice, coupling, shape):
    """Sides shorter than the stencil: sites are their own periodic neighbours."""
    q = 9 if lattice == "D2Q9" else 19
    s = _sys(lattice, coupling, *shape, a=0.02, kT=1e-4, tau=[1.0] * q, seed=5)
    p = params_of(s)
    rng = np.random.default_rng(0)
    rho = 1 + 0.01 * rng.standard_normal(p.shape)
    f0 = lbm.equilibrium_at_rest(rho, p) + 1e-4 * rng.standard_normal((q,) + p.shape)
    got = _run_gpu(lb, [s], [f0], 5)[0]
    assert rel_err(got, lbm.run(f0, 0, 5, p)) < TOL64


@pytest.mark.parametrize("lattice,coupling", [("D2Q9", "modeq"), ("D2Q9", "guo"), ("D3Q19", "guo"),
                                              ("D3Q19", "modeq")])
def test_init_matches_oracle(lb, lattice, coupling):
    s = synth.system(lattice, coupling, n=24 if lattice == "D2Q9" else 10, seed=9, system_id=5)
    s["ny"] = s["nx"] - 3 if lattice == "D2Q9" else s["ny"]
    p = params_of(s)
    # FP32 deviations hold the initial mass to the float rounding of each population
    for prec, tol, mtol in (("fp64", 1e-14, 1e-14), ("fp32", 1e-7, 1e-9)):
        ens = lb.Ensemble([s], precision=prec)
        ens.init(amplitude=0.01)
        got = ens.read_fields(0)
        want = lbm.initial_state(p, amplitude=0.01)
        assert rel_err(got, want) < tol
        _, glob = ens.observables(0)
        assert abs(glob["mass0"] / p.n_sites - p.rho_c) < mtol
        ens.close()
    rho = synth.random_density(p.shape, seed=4)
    ens = lb.Ensemble([s], precision="fp64")
    ens.init(rho=rho)
    assert rel_err(ens.read_fields(0), lbm.equilibrium_at_rest(rho, p)) < 1e-14
    ens.close()


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_single_16_thousand_step_trajectory(lb, lattice):
    """The 16^3 / 64^2 FP64 workload (a = 0, b = 0.1, kappa = 0.01, tau = 1, kT = 1e-4,
    seed 1): trajectory parity at 1e-12 over 1000 steps, and observables every 10."""
    s = synth.ensemble("single_16", lattice)[0]
    p = params_of(s)
    ens = lb.Ensemble([s], precision="fp64", obs_every=10)
    ens.init(amplitude=0.01)
    rec = ob.Recorder(p, every=10)
    f = lbm.initial_state(p)
    t = 0
    for chunk in (10, 90, 400, 500):
        ens.step(chunk)
        f = lbm.run(f, t, chunk, p, callback=rec)
        t += chunk
        assert rel_err(ens.read_fields(0), f) < TOL64, (t, rel_err(ens.read_fields(0), f))
    levels, glob = ens.observables(0)
    assert glob["n_samples"] == 100 and glob["step"] == 1000
    assert len(levels) == len(rec.lv)
    for L, blk, row in zip(levels, rec.lv, rec.acc):
        assert L["block"] == blk
        got = np.array([L["n"], L["sum_m"], L["sum_m2"], L["sum_abs_m"], L["sum_m4"], L["sum_e"], L["sum_e2"]])
        scale = np.maximum(np.abs(row), 1e-300)
        if blk == (p.nx, p.ny, p.nz if lattice == "D3Q19" else 1):
            # whole-system level: m = 0 up to rounding (mass conservation)
            assert abs(got[1]) < 1e-12 * got[0] and got[0] == row[0]
            continue
        # sum_m vanishes at every level (mass conservation): compare it on the |m| scale
        scale[1] = row[3]
        assert np.all(np.abs(got - row) <= 1e-10 * scale), (blk, got, row)
    assert abs(glob["mass"] - rec.mass[-1]) < 1e-12 * rec.mass[-1]
    assert np.allclose(glob["momentum"], rec.mom[-1], atol=1e-12)
    ens.close()


@pytest.mark.parametrize("workload,lattice,coupling", [("fss_160", "D3Q19", None), ("fss_60", "D3Q19", None),
                                                       ("fss_160", "D2Q9", None), ("fss_160", "D3Q19", "modeq")])
def test_full_size_ensembles_sampled_parity(lb, workload, lattice, coupling):
    """The batched FP32 ensembles in the launch configuration the benchmark times
    (160 systems of 16^3..64^3, the uneven 60 systems of 32^3..128^3, the
    paper's D2Q9 lattice at 64^2..512^2, and the 160 systems with the modified
    equilibrium carried to D3Q19): after one step, three systems (smallest, a
    middle one, largest) are compared with the oracle stepping each from the
    same state."""
    systems = synth.ensemble(workload, lattice, coupling)
    ens = lb.Ensemble(systems, precision="fp32", obs_every=100, graph_chunk=100)
    ens.init(amplitude=0.01)
    picks = [0, len(systems) // 2, len(systems) - 1]
    before = {k: ens.read_fields(k) for k in picks}
    ens.step(1)
    ens.sync()
    for k in picks:
        p = params_of(systems[k])
        want = lbm.step(before[k], 0, p)
        assert rel_err(ens.read_fields(k), want) < TOL32, k
    ens.close()


def test_large_256_sampled_parity_and_observables(lb):
    """The one-system 256^3 FP32 workload (the largest single lattice) in the
    benchmark's launch configuration: after one step, sampled sites (corners,
    edges, faces, interior) match the oracle's update of each site from the same
    state (its radius-3 cut-out, noise keyed by the global site index), and the
    block observables of that step match the oracle's block moments of the
    GPU's own state to 1e-10."""
    s = synth.ensemble("large_256", "D3Q19")[0]
    p = params_of(s)
    n = p.nx
    ens = lb.Ensemble([s], precision="fp32", obs_every=1)
    ens.init(amplitude=0.01)
    before = ens.read_fields(0)
    ens.step(1)
    ens.sync()
    after = ens.read_fields(0)
    fmax = np.abs(before).max()
    c = p.lat.c
    picks = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 17), (n - 1, 0, 0), (128, 0, 200), (77, 131, 0),
             (15, 16, 17), (16, 15, 255), (200, 201, 202), (255, 100, 1)]
    for (x, y, z) in picks:
        ix, iy, iz = [(np.arange(-3, 4) + v) % n for v in (x, y, z)]
        blk = before[:, iz][:, :, iy][:, :, :, ix]
        gid = (iz[:, None, None] * n + iy[None, :, None]) * n + ix[None, None, :]
        fs = lbm.collide(blk, 0, dataclasses.replace(p, nx=7, ny=7, nz=7), sites=gid.ravel())
        want = np.array([fs[i, 3 - c[i, 2], 3 - c[i, 1], 3 - c[i, 0]] for i in range(p.lat.q)])
        assert np.abs(after[:, z, y, x] - want).max() < TOL32 * fmax, (x, y, z)
    levels, glob = ens.observables(0)
    assert glob["n_samples"] == 1
    lv = ob.levels(p)
    row_all = ob.sample(ob.order_parameter(after), lv)
    assert len(levels) == len(lv)
    for L, blk, row in zip(levels, lv, row_all):
        assert L["block"] == blk
        got = np.array([L["n"], L["sum_m"], L["sum_m2"], L["sum_abs_m"], L["sum_m4"], L["sum_e"], L["sum_e2"]])
        if blk == (n, n, n):
            assert abs(got[1]) < 1e-12 * got[0] and got[0] == row[0]
            continue
        scale = np.maximum(np.abs(row), 1e-300)
        scale[1] = row[3]
        assert np.all(np.abs(got - row) <= 1e-10 * scale), (blk, got, row)
    ens.close()


def test_large_256_d2q9_sampled_parity(lb):
    """The one-system 4096^2 D2Q9 FP32 workload (the paper's lattice, modified
    equilibrium) in the benchmark's launch configuration (the paired row
    strips): after one step, sampled sites on the corners, the edges, the
    strip seams (x = 63, 64, 4095) and the interior match the oracle's update
    of each site from the same state (its radius-3 cut-out, noise keyed by the
    global site index)."""
    s = synth.ensemble("large_256", "D2Q9")[0]
    p = params_of(s)
    n = p.nx
    ens = lb.Ensemble([s], precision="fp32", graph_chunk=0)
    assert lb.kernel_variants("D2Q9")[ens.kernel_variant()][6] == 2
    ens.init(amplitude=0.01)
    before = ens.read_fields(0)
    ens.step(1)
    ens.sync()
    after = ens.read_fields(0)
    ens.close()
    fmax = np.abs(before).max()
    c = p.lat.c
    picks = [(0, 0), (n - 1, n - 1), (63, 31), (64, 32), (4095, 17), (0, 4095), (2048, 2047), (127, 1000),
             (128, 33), (3001, 64)]
    for (x, y) in picks:
        ix, iy = [(np.arange(-3, 4) + v) % n for v in (x, y)]
        blk = before[:, :1][:, :, iy][:, :, :, ix]
        gid = iy[:, None] * n + ix[None, :]
        fs = lbm.collide(blk, 0, dataclasses.replace(p, nx=7, ny=7, nz=1), sites=gid.ravel())
        want = np.array([fs[i, 0, 3 - c[i, 1], 3 - c[i, 0]] for i in range(p.lat.q)])
        assert np.abs(after[:, 0, y, x] - want).max() < TOL32 * fmax, (x, y)


@pytest.mark.parametrize("lattice,coupling", [("D2Q9", "modeq"), ("D3Q19", "guo")])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tanh_stripe_init_is_the_stripe_density(lb, lattice, coupling, precision):
    """LB_INIT_TANH_STRIPE starts every system from lb_stripe_density's profile:
    the same state, bit for bit, as LB_INIT_FROM_RHO with that density, whose
    populations sum to it."""
    n = 32 if lattice == "D2Q9" else 12
    systems = [synth.system(lattice, coupling, n=n, a=-0.01, b=0.1, kappa=0.05, kT=0.0, system_id=0),
               synth.system(lattice, coupling, n=n + 4, a=-0.004, b=0.1, kappa=0.02, kT=0.0, system_id=1)]
    rho = lb.stripe_density(systems)
    ea = lb.Ensemble(systems, precision=precision)
    ea.init(mode=lb.LB_INIT_TANH_STRIPE)
    eb = lb.Ensemble(systems, precision=precision)
    eb.init(rho=rho)
    tol = 1e-13 if precision == "fp64" else 2e-6
    off = 0
    for k, s in enumerate(systems):
        fa, fb = ea.read_fields(k), eb.read_fields(k)
        assert np.array_equal(fa, fb)
        m = s["nx"] * s["ny"] * s["nz"]
        want = rho[off:off + m].reshape(s["nz"], s["ny"], s["nx"])
        assert np.abs(fa.sum(axis=0) - want).max() < tol
        off += m
    ea.step(3)
    eb.step(3)
    for k in range(len(systems)):
        assert np.array_equal(ea.read_fields(k), eb.read_fields(k))
    ea.close()
    eb.close()


@pytest.mark.parametrize("lattice,coupling", [("D2Q9", "modeq"), ("D3Q19", "guo"), ("D3Q19", "modeq")])
def test_fp32_default_kernels_report_device_errors(lb, lattice, coupling):
    """The FP32 default kernels (paired strips on D2Q9, the paired warp-specialised
    kernel on D3Q19, the radius-1 kernel of the D3Q19 modified equilibrium) set
    the status bits themselves: a non-positive density and an indefinite noise
    covariance (c_s^2 = rho a = 0.7) are reported by lb_sync."""
    nz = 1 if lattice == "D2Q9" else 16
    q = 9 if lattice == "D2Q9" else 19
    s = _sys(lattice, coupling, 16, 16, nz, kT=1e-4, tau=[1.0] * q)
    p = params_of(s)
    f = lbm.equilibrium_at_rest(np.ones(p.shape), p)
    f[0, 0, 5, 6] = -5.0
    ens = lb.Ensemble([s], precision="fp32")
    ens.write_fields(0, f)
    ens.step(1)
    with pytest.raises(lb.LBError) as e:
        ens.sync()
    assert e.value.status == lb.LB_ERR_NONPOSITIVE_DENSITY
    ens.close()
    s2 = _sys(lattice, coupling, 16, 16, nz, a=0.7, b=0.0, kT=1e-4, tau=[1.0] * q)
    ens = lb.Ensemble([s2], precision="fp32")
    ens.init(amplitude=0.0)
    ens.step(1)
    with pytest.raises(lb.LBError) as e:
        ens.sync()
    assert e.value.status == lb.LB_ERR_NOISE_NOT_PD
    ens.close()


def test_errors_are_reported_and_sticky(lb):
    s = _sys("D2Q9", "modeq", 16, 16, kT=1e-4, tau=[1.0] * 9)
    p = params_of(s)
    f = lbm.equilibrium_at_rest(np.ones(p.shape), p)
    f[0, 0, 3, 3] = -5.0
    ens = lb.Ensemble([s], precision="fp64")
    ens.write_fields(0, f)
    ens.step(1)
    with pytest.raises(lb.LBError) as e:
        ens.sync()
    assert e.value.status == lb.LB_ERR_NONPOSITIVE_DENSITY
    with pytest.raises(lb.LBError) as e:
        ens.step(1)
    assert e.value.status == lb.LB_ERR_STATE
    ens.write_fields(0, lbm.equilibrium_at_rest(np.ones(p.shape), p))     # restores a state
    ens.step(2)
    ens.sync()
    ens.close()
    # c_s^2 = rho a >= 0.6 makes the covariance of Eq. 68 indefinite
    s2 = _sys("D2Q9", "modeq", 8, 8, a=0.7, b=0.0, kT=1e-4, tau=[1.0] * 9)
    ens = lb.Ensemble([s2], precision="fp64")
    ens.init(amplitude=0.0)
    ens.step(1)
    with pytest.raises(lb.LBError) as e:
        ens.sync()
    assert e.value.status == lb.LB_ERR_NOISE_NOT_PD
    ens.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_is_bit_identical(lb, tmp_path, precision):
    systems = synth.ensemble("single_16", "D3Q19") + [synth.system("D3Q19", n=8, system_id=1, seed=3)]
    a = lb.Ensemble(systems, precision=precision, obs_every=5)
    a.init()
    a.step(12)
    path = os.path.join(tmp_path, "ck.bin")
    a.save(path)
    a.step(13)
    ref = [a.read_fields(k) for k in range(2)]
    ref_obs = a.observables(0)
    b = lb.Ensemble(systems, precision=precision, obs_every=5)
    b.load(path)
    assert b.get_step() == 12
    b.step(13)
    for k in range(2):
        assert np.array_equal(b.read_fields(k), ref[k])
    assert b.observables(0) == ref_obs
    a.close()
    b.close()


def test_graph_replay_equals_plain_launches_and_is_deterministic(lb):
    systems = synth.ensemble("fss_160", "D2Q9")[:6]
    runs = []
    for chunk in (0, 10, 10):
        e = lb.Ensemble(systems, precision="fp32", obs_every=5, graph_chunk=chunk)
        e.init()
        e.step(3)        # unaligned start: plain launches to the chunk boundary
        e.step(37)
        runs.append(([e.read_fields(k) for k in range(len(systems))], e.observables(2)))
        if chunk:        # a new start on the same context replays the graphs it has cached
            e.init()
            e.step(3)
            e.step(37)
            runs.append(([e.read_fields(k) for k in range(len(systems))], e.observables(2)))
        e.close()
    for r in runs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(runs[0][0], r[0]))
        assert r[1] == runs[0][1]


def test_a_system_evolves_the_same_alone_or_in_a_batch(lb):
    systems = synth.ensemble("fss_160", "D3Q19")[:5]
    e = lb.Ensemble(systems, precision="fp32")
    e.init()
    e.step(4)
    batch = e.read_fields(3)
    e.close()
    e = lb.Ensemble([systems[3]], precision="fp32")
    e.init()
    e.step(4)
    assert np.array_equal(e.read_fields(0), batch)
    e.close()


@pytest.mark.parametrize("lattice,n,obs_every", [("D2Q9", 24, 3), ("D3Q19", 8, 0), ("D3Q19", 48, 0),
                                                 ("D2Q9", 20, 0), ("D3Q19", 10, 0)])
def test_structure_factor_matches_oracle(lb, lattice, n, obs_every):
    """C(k) of Eq. 80 accumulated every 2 steps, binned in shells, against the
    oracle's FFT-based spectrum (and C(0) = 0 is excluded by the shell rule).
    Sides 2^a 3^b go through the library's line FFTs (radices 4, 2 and 3 all
    appear: 24 = 4 2 3, 48 = 4 4 3), the others (20, 10) through its direct
    sums."""
    s = synth.system(lattice, n=n, a=0.01, kT=1e-4, seed=4, system_id=2)
    p = params_of(s)
    ens = lb.Ensemble([s], precision="fp64", sk_every=2, obs_every=obs_every)
    ens.init(amplitude=0.01)
    ens.step(10)
    nb = int(np.ceil(np.sqrt(p.lat.d) * n / 2))
    sums, counts, ns = ens.structure_factor(0, nb)
    rec = ob.Recorder(p, every=obs_every or 10 ** 9, sk_every=2)
    lbm.run(lbm.initial_state(p), 0, 10, p, callback=rec)
    want_s, want_c = ob.bin_shells(rec.ck, p.shape, nb)
    assert ns == rec.n_sk == 5
    assert np.array_equal(counts, want_c)
    assert np.allclose(sums, want_s, rtol=1e-10, atol=1e-14 * want_s.max())
    ens.close()


@pytest.mark.parametrize("lattice,coupling,shape", [("D2Q9", "modeq", (33, 18, 1)), ("D2Q9", "guo", (21, 30, 1)),
                                                     ("D3Q19", "guo", (18, 11, 35)), ("D3Q19", "modeq", (18, 11, 35))])
@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_single_rate_collision_paths(lb, lattice, coupling, shape, tau):
    """One relaxation rate for every non-conserved mode (the paper's BGK form):
    the population-space (tau != 1) and fully relaxed (tau = 1) code paths."""
    q = 9 if lattice == "D2Q9" else 19
    s = _sys(lattice, coupling, *shape, a=-0.001, b=0.1, kappa=0.01, kT=1e-4, tau=[tau] * q, seed=3)
    p = params_of(s)
    f0 = oracle_state(p)
    for prec, tol, n in (("fp64", TOL64, 7), ("fp32", TOL32, 1)):
        ens = lb.Ensemble([s], precision=prec)
        ens.write_fields(0, f0)
        start = ens.read_fields(0)
        ens.step(n)
        assert rel_err(ens.read_fields(0), lbm.run(start, 0, n, p)) < tol, prec
        ens.close()


def test_autotuner_times_every_variant_and_caches(lb, tmp_path):
    from paper_1202_4748_gb300 import autotune
    systems = synth.ensemble("fss_160", "D3Q19")[:8]
    rows = autotune.variants("D3Q19")
    cache = os.path.join(tmp_path, "tiles.json")
    best, ms = autotune.tune(systems, "fp32", cache=cache, steps=4, warmup=2)
    assert set(ms) == set(rows) and best in ms
    assert all(v > 0 for v in ms.values())
    best2, ms2 = autotune.tune(systems, "fp32", cache=cache)
    assert best2 == best and ms2 == ms
    # every variant gives the same trajectory (it only changes the schedule)
    runs = []
    for i in range(len(rows)):
        e = lb.Ensemble(systems[:3], precision="fp32", variant=i + 1)
        e.init()
        e.step(3)
        runs.append([e.read_fields(k) for k in range(3)])
        e.close()
    for r in runs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(runs[0], r))


def test_observables_of_all_systems_in_one_read(lb):
    systems = synth.ensemble("fss_160", "D3Q19")[::16]
    ens = lb.Ensemble(systems, precision="fp32", obs_every=5)
    ens.init()
    ens.step(20)
    both = ens.observables_all()
    assert len(both) == len(systems)
    for k in range(len(systems)):
        assert both[k] == ens.observables(k)
    # a level array shorter than the total is rejected, the counts still come back
    import ctypes
    first = (ctypes.c_int * (len(systems) + 1))()
    short = (lb.lb_obs_level * 1)()
    assert lb.lb_observables_all(ens.ctx, short, 1, first, None) == lb.LB_ERR_ARG
    assert first[len(systems)] == sum(len(b[0]) for b in both)
    ens.close()


def test_bounded_wait_reports_timeout_and_context_survives(lb):
    """The warp-specialised kernel's waits are bounded: a wait on a barrier that
    nothing arrives at gives up (about 0.3 s), reports LB_ERR_TIMEOUT through the
    status word, and the context keeps working afterwards."""
    import torch
    d = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    assert lb.lb_selftest_wait_timeout(d.data_ptr(), st.cuda_stream) == lb.LB_ERR_TIMEOUT
    s = synth.ensemble("single_16", "D3Q19")
    e = lb.Ensemble(s, precision="fp32")
    e.init()
    e.step(3)
    e.sync()
    assert e.get_step() == 3
    e.close()


@pytest.mark.parametrize("coupling", ["guo", "modeq"])
def test_fp32_fully_relaxed_path_on_odd_and_tiny_shapes(lb, coupling):
    """The FP32 tau = 1 path (the warp-specialised default kernel; the radius-1
    z-marching kernel for the modified equilibrium) on systems with sides
    shorter than the stencil, ragged tiles and several z-chunks, batched in one
    launch: each step matches the oracle stepped from the GPU's own FP32 state,
    and every compiled step-kernel variant gives the same bits."""
    shapes = [(20, 13, 11), (9, 8, 7), (4, 4, 4), (2, 2, 2), (1, 3, 2), (17, 5, 70)]
    systems = [_sys("D3Q19", coupling, *sh, a=-0.002 + 0.001 * k, b=0.1, kappa=0.01, kT=1e-4, tau=[1.0] * 19,
                    seed=20 + k, system_id=k) for k, sh in enumerate(shapes)]
    ps = [params_of(s) for s in systems]
    f0s = [oracle_state(p, steps=2) for p in ps]
    ens = lb.Ensemble(systems, precision="fp32")
    for k, f in enumerate(f0s):
        ens.write_fields(k, f)
    cur = [ens.read_fields(k) for k in range(len(systems))]
    for t in range(2):
        ens.step(1)
        ens.sync()
        for k, p in enumerate(ps):
            got = ens.read_fields(k)
            assert rel_err(got, lbm.step(cur[k], t, p)) < TOL32, (shapes[k], t)
            cur[k] = got
    ens.close()
    runs = []
    for v in range(len(lb.kernel_variants("D3Q19"))):
        e = lb.Ensemble(systems, precision="fp32", variant=v + 1)
        for k, f in enumerate(f0s):
            e.write_fields(k, f)
        e.step(3)
        runs.append([e.read_fields(k) for k in range(len(systems))])
        e.close()
    for r in runs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(runs[0], r))


@pytest.mark.parametrize("coupling", ["guo", "modeq"])
def test_fp32_paired_kernel_on_even_shapes(lb, coupling):
    """The paired-site kernel (two x-adjacent sites per consumer thread, paired
    FP32 arithmetic, producers pulling aligned quads of sites) runs when every
    nx is a multiple of 4, for the Guo form and for the modified equilibrium:
    ragged tiles in x and y, several z-chunks, sides shorter than the stencil,
    batched in one launch.  Each FP32 step matches the oracle stepped from the
    GPU's own state, the achieved one-step error is far inside the bar (FP32
    rounding of the stored deviations and of the collision: a few 1e-8 of
    max |f|), and every compiled D3Q19 variant (one-site kernels included)
    gives the same bits."""
    shapes = [(20, 13, 11), (8, 8, 7), (4, 4, 4), (4, 2, 2), (4, 3, 2), (12, 5, 70), (48, 24, 6), (36, 40, 3)]
    systems = [_sys("D3Q19", coupling, *sh, a=-0.002 + 0.001 * k, b=0.1, kappa=0.01, kT=1e-4, tau=[1.0] * 19,
                    seed=60 + k, system_id=k) for k, sh in enumerate(shapes)]
    rows = lb.kernel_variants("D3Q19")
    assert rows[0][6] == 2                               # the default pairs sites
    ps = [params_of(s) for s in systems]
    f0s = [oracle_state(p, steps=2) for p in ps]
    ens = lb.Ensemble(systems, precision="fp32")
    for k, f in enumerate(f0s):
        ens.write_fields(k, f)
    cur = [ens.read_fields(k) for k in range(len(systems))]
    worst = 0.0
    for t in range(2):
        ens.step(1)
        ens.sync()
        for k, p in enumerate(ps):
            got = ens.read_fields(k)
            e = rel_err(got, lbm.step(cur[k], t, p))
            assert e < TOL32, (shapes[k], t, e)
            worst = max(worst, e)
            cur[k] = got
    ens.close()
    assert worst < 2e-7, worst                        # measured 4.8e-8 on GB300
    runs = []
    for v in range(len(rows)):
        e = lb.Ensemble(systems, precision="fp32", variant=v + 1)
        for k, f in enumerate(f0s):
            e.write_fields(k, f)
        e.step(3)
        runs.append([e.read_fields(k) for k in range(len(systems))])
        e.close()
    for r in runs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(runs[0], r))


@pytest.mark.parametrize("tau", [[1.0] * 9, [0.8] * 9, [1.0] * 3 + [0.8, 0.9, 1.1, 0.7, 0.8, 0.85]])
def test_d2q9_strips_and_tiles_on_odd_and_tiny_shapes(lb, tau):
    """The D2Q9 modified-equilibrium step on sides that are not multiples of the
    32-site strips or the row chunks, and on sides shorter than the stencil,
    batched in one launch: each FP32 step matches the oracle stepped from the
    GPU's own state, and the row-marching strips and the CTA tiles (every
    compiled D2Q9 variant) give the same bits, for tau = 1, one rate and
    per-mode rates."""
    shapes = [(64, 40), (37, 21), (33, 18), (5, 3), (2, 2), (1, 4), (96, 7)]
    systems = [_sys("D2Q9", "modeq", nx, ny, 1, a=-0.002 + 0.001 * k, b=0.1, kappa=0.01, kT=1e-4, tau=tau,
                    seed=40 + k, system_id=k) for k, (nx, ny) in enumerate(shapes)]
    ps = [params_of(s) for s in systems]
    f0s = [oracle_state(p, steps=2) for p in ps]
    ens = lb.Ensemble(systems, precision="fp32")
    for k, f in enumerate(f0s):
        ens.write_fields(k, f)
    cur = [ens.read_fields(k) for k in range(len(systems))]
    for t in range(2):
        ens.step(1)
        ens.sync()
        for k, p in enumerate(ps):
            got = ens.read_fields(k)
            assert rel_err(got, lbm.step(cur[k], t, p)) < TOL32, (shapes[k], t)
            cur[k] = got
    ens.close()
    rows = lb.kernel_variants("D2Q9")
    assert any(r[5] == 2 for r in rows) and any(r[5] == 0 for r in rows)
    for precision in ("fp32", "fp64"):
        runs = []
        for v in range(len(rows)):
            e = lb.Ensemble(systems, precision=precision, variant=v + 1)
            for k, f in enumerate(f0s):
                e.write_fields(k, f)
            e.step(3)
            runs.append([e.read_fields(k) for k in range(len(systems))])
            e.close()
        for r in runs[1:]:
            assert all(np.array_equal(a, b) for a, b in zip(runs[0], r))


def test_init_from_device_density_equals_host_density(lb):
    """LB_INIT_FROM_DEVICE_RHO reads the same float64 densities from device
    memory (stream-ordered) and gives the bits of LB_INIT_FROM_RHO."""
    import torch
    systems = [synth.system("D3Q19", "guo", n=n, seed=3 + k, system_id=k) for k, n in enumerate((12, 16))]
    rho = np.concatenate([synth.random_density((s["nz"], s["ny"], s["nx"]), seed=9 + k).ravel()
                          for k, s in enumerate(systems)])
    a = lb.Ensemble(systems, precision="fp32")
    a.init(rho=rho)
    a.step(3)
    b = lb.Ensemble(systems, precision="fp32")
    b.init(rho_device=torch.from_numpy(rho).cuda())
    b.step(3)
    for k in range(len(systems)):
        assert np.array_equal(a.read_fields(k), b.read_fields(k))
    with pytest.raises(ValueError):
        b.init(rho_device=torch.from_numpy(rho[:-1]).cuda())
    a.close()
    b.close()


def test_default_z_chunk_adapts_to_the_ensemble(lb):
    """With no variant, tile or occupancy given, the default D3Q19 kernel takes
    the longer z-chunk only when the ensemble keeps at least two waves of
    resident CTAs (row 1 differs from row 0 only in the chunk)."""
    import torch
    rows = lb.kernel_variants("D3Q19")
    assert rows[1][2] > rows[0][2] and rows[1][:2] == rows[0][:2] and rows[1][3:] == rows[0][3:]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    few = [synth.system("D3Q19", "guo", n=64, seed=1 + k, system_id=k) for k in range(32)]
    many = [synth.system("D3Q19", "guo", n=32, seed=1 + k, system_id=k) for k in range(8 * sms // 4 + 4)]
    for systems, want in ((few, 0), (many, 1)):
        tiles = sum(-(-s["nx"] // rows[1][0]) * -(-s["ny"] // rows[1][1]) * -(-s["nz"] // rows[1][2])
                    for s in systems)
        assert (tiles >= 2 * rows[1][3] * sms) == (want == 1)
        e = lb.Ensemble(systems, precision="fp32")
        assert e.kernel_variant() == want
        e.close()
        e = lb.Ensemble(systems, precision="fp32", variant=1)
        assert e.kernel_variant() == 0
        e.close()


def test_d2q9_paired_strips_on_even_shapes(lb):
    """The two-site row strips (lane pairs of x-adjacent sites, paired FP32,
    64-site strips) run when every nx is a multiple of 4 and every mode is at
    tau = 1: strips ragged in x (a last strip of 4 sites, systems narrower
    than one strip) and in y, sides shorter than the stencil, batched in one
    launch.  Each FP32 step matches the oracle stepped from the GPU's own
    state, far inside the bar, and every compiled D2Q9 variant (one-site
    strips and CTA tiles included) gives the same bits in FP32 and in FP64."""
    shapes = [(64, 40), (68, 21), (8, 3), (4, 2), (4, 1), (136, 7), (200, 33), (12, 70)]
    systems = [_sys("D2Q9", "modeq", nx, ny, 1, a=-0.002 + 0.001 * k, b=0.1, kappa=0.01, kT=1e-4, tau=[1.0] * 9,
                    seed=80 + k, system_id=k) for k, (nx, ny) in enumerate(shapes)]
    rows = lb.kernel_variants("D2Q9")
    assert rows[0][6] == 2 and rows[0][5] == 2           # the default pairs sites in row strips
    ps = [params_of(s) for s in systems]
    f0s = [oracle_state(p, steps=2) for p in ps]
    ens = lb.Ensemble(systems, precision="fp32")
    for k, f in enumerate(f0s):
        ens.write_fields(k, f)
    cur = [ens.read_fields(k) for k in range(len(systems))]
    worst = 0.0
    for t in range(2):
        ens.step(1)
        ens.sync()
        for k, p in enumerate(ps):
            got = ens.read_fields(k)
            e = rel_err(got, lbm.step(cur[k], t, p))
            assert e < TOL32, (shapes[k], t, e)
            worst = max(worst, e)
            cur[k] = got
    ens.close()
    assert worst < 2e-7, worst
    for precision in ("fp32", "fp64"):
        runs = []
        for v in range(len(rows)):
            e = lb.Ensemble(systems, precision=precision, variant=v + 1)
            for k, f in enumerate(f0s):
                e.write_fields(k, f)
            e.step(3)
            runs.append([e.read_fields(k) for k in range(len(systems))])
            e.close()
        for v, r in enumerate(runs[1:]):
            assert all(np.array_equal(a, b) for a, b in zip(runs[0], r)), (precision, v + 1)


@pytest.mark.parametrize("kind,code", [("DENSITY", "NONPOSITIVE_DENSITY"), ("NOISE", "NOISE_NOT_PD"),
                                       ("NONFINITE", "NONFINITE"), ("TIMEOUT", "TIMEOUT")])
def test_injected_device_errors_are_reported_sticky_and_cleared(lb, tmp_path, kind, code):
    """Failure detection without a GPU fault: a host-armed fault sets the status bit
    a kernel would set; lb_sync reports it, later steps are refused, and a
    checkpoint load clears it and the run continues as if nothing happened."""
    systems = synth.ensemble("single_16", "D3Q19")
    ens = lb.Ensemble(systems, precision="fp32", obs_every=5, graph_chunk=10)
    ens.init()
    ens.step(10)
    path = os.path.join(tmp_path, "ck.bin")
    ens.save(path)
    ref = lb.Ensemble(systems, precision="fp32", obs_every=5, graph_chunk=10)
    ref.init()
    ref.step(30)
    want = ref.read_fields(0)
    ref.close()
    assert lb.lb_inject_fault(ens.ctx, getattr(lb, "LB_FAULT_" + kind), 17) == lb.LB_OK
    ens.step(10)                                  # the fault fires after the step ending at 17
    with pytest.raises(lb.LBError) as e:
        ens.sync()
    assert e.value.status == getattr(lb, "LB_ERR_" + code)
    with pytest.raises(lb.LBError) as e:
        ens.step(1)
    assert e.value.status == lb.LB_ERR_STATE
    ens.load(path)                                # clears the sticky error
    ens.step(20)
    ens.sync()
    assert np.array_equal(ens.read_fields(0), want)
    ens.close()


def test_injected_launch_failure_leaves_a_consistent_context(lb):
    systems = synth.ensemble("single_16", "D2Q9")
    ens = lb.Ensemble(systems, precision="fp32", graph_chunk=10)
    ens.init()
    assert lb.lb_inject_fault(ens.ctx, lb.LB_FAULT_LAUNCH, 7) == lb.LB_OK
    assert lb.lb_inject_fault(ens.ctx, lb.LB_FAULT_LAUNCH, 0) == lb.LB_ERR_ARG     # not in the future
    with pytest.raises(lb.LBError) as e:
        ens.step(20)
    assert e.value.status == lb.LB_ERR_CUDA
    assert ens.get_step() == 6                    # the steps before the failed one ran
    ens.step(14)                                  # the fault fired once; the run carries on
    ens.sync()
    ref = lb.Ensemble(systems, precision="fp32", graph_chunk=10)
    ref.init()
    ref.step(20)
    assert np.array_equal(ens.read_fields(0), ref.read_fields(0))
    ref.close()
    ens.close()

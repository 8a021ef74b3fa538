"""The C ABI: library loads, exports every declared entry point, validates arguments.

Runs without a GPU: nothing here reaches a CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbfluct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    import paper_1202_4748_gb300 as lb
    lib = ctypes.CDLL(lb.LIB_PATH)
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lb.EXPORTED) == names


def test_header_constants_match_the_binding():
    """Every numeric #define of the header has the same value in the binding."""
    import paper_1202_4748_gb300 as lb
    src = open(os.path.join(ROOT, "include", "lbfluct.h")).read()
    defs = re.findall(r"^#define (LB_[A-Z0-9_]+) (.+)$", src, flags=re.M)
    assert len(defs) >= 5
    for name, expr in defs:
        value = eval(expr.strip(), {})
        assert getattr(lb, name) == value, name
    assert len(lb.HIST_EST_FIELDS) == lb.LB_HIST_EST


def test_observables_all_rejects_missing_arguments():
    import paper_1202_4748_gb300 as lb
    assert lb.lb_observables_all(None, None, 0, None, None) == lb.LB_ERR_ARG


def test_status_strings_and_version():
    import paper_1202_4748_gb300 as lb
    assert lb.lb_status_string(0) == b"ok"
    for code in range(-11, 0):
        assert lb.lb_status_string(code) != b"unknown status"
    assert b"sm_103a" in lb.lb_version()


def _one(**kw):
    s = synth.system("D2Q9", n=16)
    s.update(kw)
    return s


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(nz=2), dict(kT=-1.0), dict(rho_c=0.0), dict(kappa=-1e-3),
    dict(tau=[1.0] * 3 + [0.5] + [1.0] * 5), dict(system_id=1 << 24), dict(coupling=7),
    dict(a=float("nan")),
])
def test_invalid_descriptors_rejected(bad):
    import paper_1202_4748_gb300 as lb
    s = _one(**bad)
    if s["lattice"] == "D3Q19":
        s["tau"] = [1.0] * 19
    with pytest.raises(lb.LBError) as e:
        lb.workspace_bytes([s])
    assert e.value.status == lb.LB_ERR_ARG


def test_mixed_lattices_and_bad_options_rejected():
    import paper_1202_4748_gb300 as lb
    a = _one()
    b = synth.system("D3Q19", n=8)
    with pytest.raises(lb.LBError):
        lb.workspace_bytes([a, b])
    with pytest.raises(lb.LBError):
        lb.workspace_bytes([a], graph_chunk=3)
    with pytest.raises(lb.LBError):
        lb.workspace_bytes([a], precision=7)
    with pytest.raises(lb.LBError) as e:
        lb.workspace_bytes([a], tile=(7, 7, 1))
    assert e.value.status == lb.LB_ERR_UNSUPPORTED


def test_workspace_grows_with_sites_and_precision():
    import paper_1202_4748_gb300 as lb
    e = synth.ensemble("fss_160", "D3Q19")
    b32 = lb.workspace_bytes(e, precision="fp32", obs_every=100)
    b64 = lb.workspace_bytes(e, precision="fp64", obs_every=100)
    pops32 = 2 * 19 * 4 * synth.sites(e)
    assert pops32 < b32 < pops32 * 1.6
    assert b64 == b32 + pops32      # same bookkeeping, twice the population bytes


def test_create_rejects_bad_workspace_without_touching_the_device():
    import paper_1202_4748_gb300 as lb
    desc = lb.make_desc([_one()])
    o = lb.make_opts()
    ctx = ctypes.c_void_p()
    st = lb.lb_create(desc, 1, ctypes.byref(o), None, 1 << 20, None, ctypes.byref(ctx))
    assert st == lb.LB_ERR_WORKSPACE and not ctx.value
    st = lb.lb_create(desc, 1, ctypes.byref(o), ctypes.c_void_p(4096 + 8), 1 << 40, None, ctypes.byref(ctx))
    assert st == lb.LB_ERR_WORKSPACE


def test_null_context_calls_fail_cleanly():
    import paper_1202_4748_gb300 as lb
    assert lb.lb_step(None, 1) == lb.LB_ERR_ARG
    assert lb.lb_sync(None) == lb.LB_ERR_ARG
    assert lb.lb_init(None, 0, 0.01, None) == lb.LB_ERR_ARG
    lb.lb_destroy(None)


def test_derive_matches_oracle_formulas():
    """lb_derive (host arithmetic in the library) against the oracle's Eqs. 47-50."""
    import paper_1202_4748_gb300 as lb
    from oracle import observables as ob
    rng = np.random.default_rng(3)
    acc = np.abs(rng.standard_normal((1, 7)))
    acc[0, 0] = 1234.0
    kT = 2e-4
    want = ob.derived(acc, [(4, 2, 1)], kT)[0]
    L = lb.lb_obs_level()
    L.bx, L.by, L.bz = 4, 2, 1
    L.n, L.sum_m, L.sum_m2, L.sum_abs_m, L.sum_m4, L.sum_e, L.sum_e2 = acc[0]
    out = (ctypes.c_double * 6)()
    assert lb.lb_derive(ctypes.byref(L), kT, out) == 0
    assert np.isclose(out[0], want["M_L"], rtol=1e-15)
    assert np.isclose(out[1], want["chi_L"], rtol=1e-13)
    assert np.isclose(out[2], want["chi_L_lowT"], rtol=1e-13)
    assert np.isclose(out[3], want["c_HL"], rtol=1e-13)
    assert np.isclose(out[4], want["U_L"], rtol=1e-13)
    L.n = 0
    assert lb.lb_derive(ctypes.byref(L), kT, out) == lb.LB_ERR_ARG


def test_strip_variants_are_refused_for_the_guo_form():
    """Row-marching strips are compiled for the modified equilibrium only: a Guo
    ensemble that asks for one is refused at plan time, and its default is the
    first tile row."""
    import paper_1202_4748_gb300 as lb
    s = synth.system("D2Q9", "guo", n=16)
    rows = lb.kernel_variants("D2Q9")
    strip = [i for i, r in enumerate(rows) if r[5] == 2]
    assert strip and strip[0] == 0                      # the modified equilibrium's default
    with pytest.raises(lb.LBError) as e:
        lb.workspace_bytes([s], precision="fp32", variant=strip[0] + 1)
    assert e.value.status == lb.LB_ERR_UNSUPPORTED
    assert lb.workspace_bytes([s], precision="fp32") > 0
    assert lb.workspace_bytes([synth.system("D2Q9", "modeq", n=16)], precision="fp32", variant=1) > 0


def test_kernel_variant_table():
    import paper_1202_4748_gb300 as lb
    for lat in ("D2Q9", "D3Q19"):
        rows = lb.kernel_variants(lat)
        assert len(rows) >= 3 and len(set(rows)) == len(rows)
        for x, y, z, occ, pw, stg, spt in rows:
            assert x > 0 and y > 0 and z > 0 and occ >= 0 and pw >= 0 and stg in (0, 1, 2, 3) and spt in (1, 2)
            assert x % 16 == 0
            assert stg != 1 or pw > 0                    # bulk staging is done by producer warps
            if spt == 2 and lat == "D3Q19":              # paired sites: the warp-specialised kernel
                assert pw > 0 and stg in (0, 3) and (x * y // 2) % 32 == 0
            if spt == 2 and lat == "D2Q9":               # paired sites: two-site row strips
                assert stg == 2
            assert stg != 3 or spt == 2                  # cp.async staging: the paired kernel's producers
            if stg == 2:                                 # row strips: one warp per 32 sites x spt of a row
                assert lat == "D2Q9" and x == 32 * spt and pw == 0
            else:
                assert x * y // spt + 32 * pw <= 1024
                assert x * y + 32 * pw <= 1024           # the one-site fallback of the same tile
            if lat == "D2Q9":
                assert pw == 0                           # producer warps only on the 3-D kernel
        if lat == "D2Q9":
            assert all(r[2] == 1 for r in rows)
    assert lb.lb_kernel_variants(7, None, 0) == lb.LB_ERR_ARG
    # a variant index past the table is rejected at plan time
    s = synth.system("D3Q19", n=16)
    n = len(lb.kernel_variants("D3Q19"))
    with pytest.raises(lb.LBError) as e:
        lb.workspace_bytes([s], precision="fp32", variant=n + 1)
    assert e.value.status == lb.LB_ERR_UNSUPPORTED
    assert lb.workspace_bytes([s], precision="fp32", variant=n) > 0


def _mixture_counts(lo, hi, nb, parts, n_total):
    from scipy.special import ndtr
    edges = lo + (hi - lo) * np.arange(nb + 1) / nb
    cdf = sum(wt * ndtr((edges - mu) / sg) for wt, mu, sg in parts)
    c = np.rint(n_total * np.diff(cdf)).astype(np.int64)
    return np.concatenate([[17], c, [5]]).astype(np.uint64)


@pytest.mark.parametrize("case", ["two", "one", "cut", "flat"])
def test_histogram_estimates_match_oracle(case):
    import paper_1202_4748_gb300 as lb
    from oracle import observables as ob
    lo, hi = -0.4, 0.4
    if case == "two":
        c = _mixture_counts(lo, hi, 640, [(0.5, 0.21, 0.01), (0.5, -0.21, 0.012)], 10 ** 9)
        kw = dict(vol=64.0, kT=1e-4)
    elif case == "one":
        c = _mixture_counts(lo, hi, 801, [(1.0, 0.001, 0.05)], 10 ** 8)
        kw = dict(vol=1.0, kT=2e-4)
    elif case == "cut":
        c = _mixture_counts(lo, hi, 640, [(0.45, 0.2, 0.01), (0.45, -0.2, 0.01), (0.1, 0.0, 0.2)], 10 ** 9)
        kw = dict(vol=8.0, kT=1e-4, m_cut=0.1, frac=0.3)
    else:
        c = np.ones(66, dtype=np.uint64)
        kw = dict(vol=8.0, kT=1e-4)
    got = lb.histogram_estimates(c, lo, hi, **kw)
    want = ob.histogram_estimates(c.astype(np.int64), lo, hi, **kw)
    for k in lb.HIST_EST_FIELDS:
        g, w = got[k], want[k]
        if isinstance(w, float) and np.isnan(w):
            assert np.isnan(g), k
        else:
            assert g == pytest.approx(w, rel=1e-9, abs=1e-12), k


def test_histogram_estimates_and_options_rejected():
    import paper_1202_4748_gb300 as lb
    c = np.ones(10, dtype=np.uint64)
    for args in [(-0.5, 0.6, 1.0, 1e-4), (-0.5, 0.5, 0.0, 1e-4), (-0.5, 0.5, 1.0, 0.0)]:
        with pytest.raises(lb.LBError):
            lb.histogram_estimates(c, *args)
    with pytest.raises(lb.LBError):
        lb.histogram_estimates(c, -0.5, 0.5, 1.0, 1e-4, frac=1.5)
    s = synth.system("D2Q9", n=16)
    for kw in [dict(hist_bins=lb.LB_MAX_HIST_BINS + 1, hist_range=0.5), dict(hist_bins=8, hist_range=0.0),
               dict(hist_bins=-1, hist_range=0.5), dict(hist_bins=8, hist_range=float("inf"))]:
        with pytest.raises(lb.LBError) as e:
            lb.workspace_bytes([s], **kw)
        assert e.value.status == lb.LB_ERR_ARG
    base = lb.workspace_bytes([s])
    # 5 levels (16, 8, 4, 2, 1) of 102 64-bit counts, up to one alignment unit of slack
    assert lb.workspace_bytes([s], hist_bins=100, hist_range=0.5) >= base + 8 * 102 * 5 - 256


@pytest.mark.parametrize("lattice,side,xi", [("D3Q19", 24, 1.2), ("D2Q9", 48, 2.0), ("D3Q19", 16, 0.0)])
def test_oz_fit_matches_oracle(lattice, side, xi):
    import paper_1202_4748_gb300 as lb
    from oracle import observables as ob
    from oracle.lattice import d2q9, d3q19
    lat = d3q19() if lattice == "D3Q19" else d2q9()
    shape = (side, side, side) if lattice == "D3Q19" else (1, side, side)
    kT, chi, kmax, ns = 1e-4, 9.0, 7, 4
    C = kT * chi / (1.0 + xi * xi * ob.laplacian_symbol(shape, lat))
    sums, counts = ob.bin_shells(ns * C, shape, kmax + 2)
    got = lb.oz_fit(lattice, side, sums, counts, ns, kT, kmax)
    want = ob.oz_fit(sums, counts, ns, shape, lat, kT, kmax)
    assert got["shells"] == want["shells"] == kmax
    for k in ("chi", "a"):
        assert got[k] == pytest.approx(want[k], rel=1e-9), k
    # b is a difference of large sums: compare it on the scale of a
    assert abs(got["b"] - want["b"]) <= 1e-9 * abs(want["a"])
    if xi > 0:
        assert got["xi"] == pytest.approx(want["xi"], rel=1e-6)
    else:                        # b = 0 up to rounding: xi is 0 or NaN (b slightly negative)
        assert all(np.isnan(v) or v < 1e-5 for v in (got["xi"], want["xi"]))
    bad = counts.copy()
    bad[2] += 1
    with pytest.raises(lb.LBError):
        lb.oz_fit(lattice, side, sums, bad, ns, kT, kmax)


def test_momentum_spectra_option_needs_structure_factor():
    import paper_1202_4748_gb300 as lb
    s = synth.system("D2Q9", n=16)
    with pytest.raises(lb.LBError) as e:
        lb.workspace_bytes([s], jk_spectra=True)
    assert e.value.status == lb.LB_ERR_ARG
    a = lb.workspace_bytes([s], sk_every=5)
    b = lb.workspace_bytes([s], sk_every=5, jk_spectra=True)
    assert b >= a + 13 * 8 * 256 - 4 * 256        # j, Laplacian, three transforms, three accumulators


def test_pt_workspace_sizes_and_validation():
    import paper_1202_4748_gb300 as lb
    n = ctypes.c_size_t()
    assert lb.lb_pt_workspace_bytes(lb.LB_D3Q19, 16, ctypes.byref(n)) == lb.LB_OK
    assert n.value >= 8 * 5 * 16 ** 3                 # G plus two complex transform buffers
    assert lb.lb_pt_workspace_bytes(lb.LB_D2Q9, 64, ctypes.byref(n)) == lb.LB_OK
    assert n.value >= 8 * 5 * 64 ** 2
    for lat, side in [(lb.LB_D3Q19, 1), (5, 16), (lb.LB_D3Q19, 1024)]:
        assert lb.lb_pt_workspace_bytes(lat, side, ctypes.byref(n)) == lb.LB_ERR_ARG
    out = (ctypes.c_double * 7)()
    # argument checks come before any device work
    assert lb.lb_pt_broken(lb.LB_D2Q9, 8, 1e-3, 0.1, 0.01, 1e-4, None, 0, None, out) == lb.LB_ERR_ARG
    assert lb.lb_pt_symmetric(lb.LB_D2Q9, 8, 1e-3, -0.1, 0.01, 1e-4, None, 0, None, out) == lb.LB_ERR_ARG
    assert lb.lb_pt_sums(lb.LB_D2Q9, 8, 0.0, 0.01, None, 0, None, out) == lb.LB_ERR_ARG
    assert lb.lb_pt_sums(lb.LB_D2Q9, 8, 1.0, 0.01, None, 0, None, out) == lb.LB_ERR_WORKSPACE


def test_stripe_density_is_the_mean_field_profile():
    """lb_stripe_density (host only): coexistence plateaus rho_c +- sqrt(-a/b)
    (Eq. 20) joined by tanh interfaces of width sqrt(-2 kappa/a) (Eqs. 22-23) at
    x = nx/4 and 3nx/4, every system in descriptor order."""
    import paper_1202_4748_gb300 as lb
    systems = [synth.system("D2Q9", "modeq", n=64, a=-0.01, b=0.1, kappa=0.1),
               dict(synth.system("D3Q19", "guo", n=12, a=-0.004, b=0.1, kappa=0.0, rho_c=1.3), ny=5, nz=3)]
    rho = lb.stripe_density(systems)
    assert rho.shape == (64 * 64 + 12 * 5 * 3,)
    a = rho[:64 * 64].reshape(64, 64)
    x = np.arange(64.0)
    phi0, w = np.sqrt(0.1), np.sqrt(20.0)
    want = 1.0 + phi0 * (np.tanh((x - 16) / w) - np.tanh((x - 48) / w) - 1)
    assert np.allclose(a, want[None, :], rtol=0, atol=1e-14)
    assert abs(a[:, 32].mean() - (1 + phi0)) < 2e-3 and abs(a[:, 0].mean() - (1 - phi0)) < 2e-3
    b = rho[64 * 64:].reshape(3, 5, 12)                    # kappa = 0: the sharp step
    phi1 = np.sqrt(0.04)
    step = np.where((np.arange(12) >= 3) & (np.arange(12) < 9), 1.3 + phi1, 1.3 - phi1)
    assert np.array_equal(b, np.broadcast_to(step, b.shape))
    for bad in (dict(a=0.001), dict(a=-0.01, b=-0.1), dict(a=-0.01, kappa=-1.0)):
        with pytest.raises(lb.LBError) as e:
            lb.stripe_density([dict(systems[0], **bad)])
        assert e.value.status == lb.LB_ERR_ARG
    assert lb.lb_stripe_density(None, 1, None) == lb.LB_ERR_ARG

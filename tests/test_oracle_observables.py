"""Pins for the block observables (Eqs. 46-50) and the structure factor (Eq. 80)."""
import numpy as np
import pytest

from oracle import lbm, observables as ob


@pytest.mark.parametrize("shape,d,want", [
    ((64, 64, 1), 2, [(64, 64, 1), (32, 32, 1), (16, 16, 1), (8, 8, 1), (4, 4, 1), (2, 2, 1), (1, 1, 1)]),
    ((120, 120, 1), 2, [(120, 120, 1), (60, 60, 1), (30, 30, 1), (15, 15, 1), (1, 1, 1)]),
    ((24, 24, 24), 3, [(24, 24, 24), (12, 12, 12), (6, 6, 6), (3, 3, 3), (1, 1, 1)]),
    ((16, 8, 1), 2, [(16, 8, 1), (8, 4, 1), (4, 2, 1), (2, 1, 1), (1, 1, 1)]),
    ((5, 7, 1), 2, [(5, 7, 1), (1, 1, 1)]),
])
def test_levels(shape, d, want):
    p = lbm.Params(lattice="D2Q9" if d == 2 else "D3Q19", nx=shape[0], ny=shape[1], nz=shape[2])
    assert ob.levels(p) == want


def test_block_sums_brute_force():
    rng = np.random.default_rng(0)
    p = lbm.Params(nx=8, ny=8)
    phi = rng.standard_normal((1, 8, 8)) * 0.01
    lv = ob.levels(p)
    acc = ob.sample(phi, lv)
    for row, (bx, by, bz) in zip(acc, lv):
        ms, es = [], []
        for y0 in range(0, 8, by):
            for x0 in range(0, 8, bx):
                s = 0.0
                s2 = 0.0
                for y in range(y0, y0 + by):
                    for x in range(x0, x0 + bx):
                        s += phi[0, y, x]
                        s2 += phi[0, y, x] ** 2
                ms.append(s / (bx * by))
                es.append(s2 / (2 * bx * by))
        ms, es = np.array(ms), np.array(es)
        want = [len(ms), ms.sum(), (ms ** 2).sum(), np.abs(ms).sum(), (ms ** 4).sum(), es.sum(), (es ** 2).sum()]
        assert np.allclose(row, want, rtol=1e-13, atol=1e-20)


def test_whole_system_level_vanishes_by_conservation():
    """m at L = S is zero: phi is measured from the global mean (Eq. 1, text above Eq. 46)."""
    p = lbm.Params(nx=16, ny=16)
    f = lbm.initial_state(p)
    phi = ob.order_parameter(f)
    acc = ob.sample(phi, ob.levels(p))
    assert abs(acc[0, 1]) < 1e-15 and acc[0, 2] < 1e-30


def test_derived_quantities_gaussian_limit():
    """For iid Gaussian phi: chi_1 = var/kT, U_L = 0 (Gaussian), M_L = sqrt(2/pi) sigma_L."""
    rng = np.random.default_rng(1)
    p = lbm.Params(nx=32, ny=32, kT=1e-4)
    lv = ob.levels(p)
    acc = np.zeros((len(lv), 7))
    sig = 0.01
    for _ in range(400):
        phi = sig * rng.standard_normal((1, 32, 32))
        phi -= phi.mean()
        acc += ob.sample(phi, lv)
    d = {r["block"]: r for r in ob.derived(acc, lv, p.kT)}
    one = d[(1, 1, 1)]
    assert abs(one["chi_L"] * p.kT / sig ** 2 - 1) < 0.02
    assert abs(one["U_L"]) < 0.02
    assert abs(one["M_L"] / (np.sqrt(2 / np.pi) * sig) - 1) < 0.01
    four = d[(4, 4, 1)]
    # block of 16 iid sites (with the global mean removed): var = sig^2/16 (1 - 16/1024)
    assert abs(four["chi_L"] * p.kT / (sig ** 2 * (1 - 16 / 1024)) - 1) < 0.03


def test_structure_factor_against_naive_dft():
    rng = np.random.default_rng(2)
    for shape in [(1, 8, 8), (4, 4, 4), (1, 6, 6)]:
        phi = rng.standard_normal(shape)
        phi -= phi.mean()
        nz, ny, nx = shape
        ck = ob.structure_factor(phi)
        for kz in range(nz):
            for ky in range(ny):
                for kx in range(nx):
                    s = 0j
                    for z in range(nz):
                        for y in range(ny):
                            for x in range(nx):
                                s += phi[z, y, x] * np.exp(-2j * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz))
                    assert np.isclose(ck[kz, ky, kx], abs(s) ** 2 / phi.size, rtol=1e-10, atol=1e-12)
        assert abs(ck[0, 0, 0]) < 1e-20          # C(0) = 0 by mass conservation


def test_shell_index_is_nearest_integer_radius():
    for shape in [(1, 16, 16), (8, 8, 8), (1, 9, 9)]:
        j = ob.shell_index(shape)
        nz, ny, nx = shape
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    n = [v if 2 * v < s else v - s for v, s in ((x, nx), (y, ny), (z, nz))]
                    r = np.sqrt(sum(v * v for v in n))
                    assert j[z, y, x] == int(np.floor(r + 0.5))


def test_recorder_schedule():
    p = lbm.Params(nx=8, ny=8, kT=1e-5, a=0.05)
    rec = ob.Recorder(p, every=3, sk_every=5)
    f = lbm.initial_state(p)
    lbm.run(f, 0, 10, p, callback=rec)
    assert rec.acc[0, 0] == 3                  # samples at t = 3, 6, 9
    assert rec.n_sk == 2                       # t = 5, 10
    assert len(rec.mass) == 3 and np.allclose(rec.mass, 64.0, rtol=1e-14)

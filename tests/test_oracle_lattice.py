"""Pins for velocity sets, weights and moment bases."""
import os

import numpy as np
import pytest

from oracle import lattice


def _golden(golden_dir):
    out = {}
    with open(os.path.join(golden_dir, "d2q9_paper_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                out[k] = np.array([float(x) for x in v])
    return out


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_isotropy(name):
    lat = lattice.get(name)
    c = lat.c.astype(float)
    t = lat.t
    assert np.isclose(t.sum(), 1.0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia->a", t, c), 0, atol=1e-15)
    d = np.eye(3)
    d[lat.d:, lat.d:] = 0
    assert np.allclose(np.einsum("i,ia,ib->ab", t, c, c), d / 3, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", t, c, c, c), 0, atol=1e-15)
    four = np.einsum("i,ia,ib,ic,id->abcd", t, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(four, iso, atol=1e-15)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_basis_orthogonal_brute_force(name):
    lat = lattice.get(name)
    q = lat.q
    for a in range(q):
        for b in range(q):
            s = 0.0
            for i in range(q):
                s += lat.t[i] * lat.T[a, i] * lat.T[b, i]
            if a == b:
                assert s > 0 and np.isclose(s, lat.N[a], rtol=1e-14)
            else:
                assert abs(s) < 1e-14


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_round_trip_and_conserved_rows(name):
    lat = lattice.get(name)
    rng = np.random.default_rng(5)
    f = rng.random((lat.q, 2, 2, 2))
    assert np.allclose(lat.populations(lat.moments(f)), f, rtol=1e-13, atol=1e-14)
    m = lat.moments(f)
    assert np.allclose(m[0], f.sum(0), rtol=1e-14)
    for a in range(lat.d):
        assert np.allclose(m[1 + a], np.tensordot(lat.c[:, a].astype(float), f, 1), atol=1e-14)


def test_d2q9_norms_match_eq68_diagonal(golden_dir):
    g = _golden(golden_dir)
    lat = lattice.d2q9()
    assert np.allclose(lat.N[:3], [1, 1 / 3, 1 / 3], rtol=1e-14)
    assert np.allclose(lat.N[3:], g["noise_diag_cs2_third"], rtol=1e-14)


def test_pooley_weights_as_printed(golden_dir):
    g = _golden(golden_dir)
    assert np.allclose(lattice.POOLEY_W[1:], g["w"])
    assert np.allclose(lattice.POOLEY_WXX[1:], g["wxx"])
    assert np.allclose(lattice.POOLEY_WYY[1:], g["wyy"])
    assert np.allclose(lattice.POOLEY_WXY[1:], g["wxy"])
    # the weights are 3 t_i, which makes them carry the second moment exactly
    lat = lattice.d2q9()
    assert np.allclose(lattice.POOLEY_W[1:], 3 * lat.t[1:])

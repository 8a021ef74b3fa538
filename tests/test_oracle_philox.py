"""Pins for the oracle's Philox4x32-10 and Box-Muller normals."""
import os

import numpy as np

from oracle import philox


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


def test_known_answer_vectors(golden_dir):
    for r in _kat(golden_dir):
        out = philox.philox4x32_10(*r[:6])
        assert [int(v) for v in out] == r[6:]


def test_vectorised_matches_scalar():
    c0 = np.arange(50, dtype=np.uint64) * 977 + 3
    vec = philox.philox4x32_10(c0, 7, 0, (5 << 8) | 1, 12345, 678)
    for k in range(50):
        sc = philox.philox4x32_10(int(c0[k]), 7, 0, (5 << 8) | 1, 12345, 678)
        assert [int(v[k]) for v in vec] == [int(s) for s in sc]


def test_uniform_open_interval():
    w = np.array([0, 1, 2 ** 31, 2 ** 32 - 1], dtype=np.uint32)
    u = philox.uniform01(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert u[0] == 0.5 * 2.0 ** -32


def test_normals_moments_and_independence():
    sites = np.arange(200_000, dtype=np.uint64)
    n = philox.site_normals(sites, 3, 2, 99, 6)
    flat = n.ravel()
    se = 1.0 / np.sqrt(flat.size)
    assert abs(flat.mean()) < 5 * se
    assert abs(flat.var() - 1.0) < 5 * np.sqrt(2.0) * se
    assert abs((flat ** 4).mean() - 3.0) < 5 * np.sqrt(96.0) * se
    c = np.corrcoef(n)
    off = c[~np.eye(6, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / np.sqrt(sites.size)
    # different steps / systems / seeds give uncorrelated streams
    for args in ((4, 2, 99), (3, 3, 99), (3, 2, 100)):
        m = philox.site_normals(sites, *args, 6)
        assert abs(np.corrcoef(n[0], m[0])[0, 1]) < 5 / np.sqrt(sites.size)


def test_draw_order():
    w0 = philox.site_words([11], 5, 3, 0, 42)
    w1 = philox.site_words([11], 5, 3, 1, 42)
    n = philox.site_normals([11], 5, 3, 42, 6)
    a, b = philox.box_muller(w0[0], w0[1])
    c, d = philox.box_muller(w0[2], w0[3])
    e, f = philox.box_muller(w1[0], w1[1])
    assert np.allclose(n[:, 0], [a[0], b[0], c[0], d[0], e[0], f[0]], rtol=0, atol=0)

"""Philox4x32-10 and Box-Muller normals (oracle side; test infrastructure).

The paper asks for Gaussian random variables for the noise (Sec. III A, text
around Eq. 67) without naming a generator.  Both sides of this project use the
counter-based Philox4x32 generator with 10 rounds, as published by Salmon,
Moraes, Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC'11).
Each side implements it independently from that definition; this file is the
oracle's copy.

One round maps the counter (c0, c1, c2, c3) with key (k0, k1) to
    (hi(B*c2) ^ c1 ^ k0,  lo(B*c2),  hi(A*c0) ^ c3 ^ k1,  lo(A*c0))
with the multipliers A = 0xD2511F53, B = 0xCD9E8D57; between rounds the key is
bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).

Counter layout used by the method (a convention of this project -- parity
unpinned by the paper, identical on both sides by construction):
    c0 = linear site index x + nx*(y + ny*z)
    c1 = time step, low 32 bits;  c2 = time step, high 32 bits
    c3 = (system_id << 8) | draw
    key = (seed & 0xffffffff, seed >> 32)
"""

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_A = np.uint64(0xD2511F53)
_B = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)

# Draw index reserved for the initial density perturbation.
INIT_DRAW = 0xFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds.  Arguments broadcast; returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p_a = _A * c0          # < 2**64, exact in uint64
        p_b = _B * c2
        c0, c1, c2, c3 = ((p_b >> np.uint64(32)) ^ c1 ^ k0, p_b & _MASK,
                          (p_a >> np.uint64(32)) ^ c3 ^ k1, p_a & _MASK)
    return tuple(np.asarray(v, dtype=np.uint32) for v in (c0, c1, c2, c3))


def uniform01(word):
    """Map a uint32 word to (0, 1): U = (x + 1/2) * 2**-32 (exact in float64)."""
    return (np.asarray(word, dtype=np.float64) + 0.5) * 2.0 ** -32


def box_muller(w_a, w_b):
    """Two independent N(0,1) variates from two uint32 words (textbook form).

    R = sqrt(-2 ln U_a);  n0 = R cos(2 pi U_b);  n1 = R sin(2 pi U_b).
    """
    ua = uniform01(w_a)
    ub = uniform01(w_b)
    r = np.sqrt(-2.0 * np.log(ua))
    ang = 2.0 * np.pi * ub
    return r * np.cos(ang), r * np.sin(ang)


def site_words(sites, step, system_id, draw, seed):
    """Four Philox words per site for (site, step, system_id, draw) under ``seed``."""
    sites = np.asarray(sites, dtype=np.uint64)
    step = int(step)
    seed = int(seed)
    c3 = (int(system_id) << 8) | int(draw)
    return philox4x32_10(sites, step & 0xFFFFFFFF, (step >> 32) & 0xFFFFFFFF, c3,
                         seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def site_normals(sites, step, system_id, seed, count):
    """``count`` standard normals per site, shape (count, n_sites).

    Normals are produced in draw order: draw 0 gives words w0..w3 and the
    Box-Muller pairs (w0, w1) -> (n0, n1), (w2, w3) -> (n2, n3); draw 1 gives
    n4..n7, and so on.  Unused normals of the last draw are discarded.
    """
    out = []
    draw = 0
    while len(out) < count:
        w = site_words(sites, step, system_id, draw, seed)
        out.extend(box_muller(w[0], w[1]))
        out.extend(box_muller(w[2], w[3]))
        draw += 1
    return np.stack(out[:count])

"""Perturbation-theory comparator in plain FP64 (test infrastructure).

Sec. II C (perturbation theory).  On a periodic lattice of side S (d = 2 or 3,
V = N = S^d sites) the momentum integrals become sums over the permissible
wavevectors except the zero mode (the text after Eq. 32), with the propagator

    G(q) = 1 / (m + kappa q^2)         for q != 0,

where q^2 is the symbol of the lattice Laplacian of the simulated model,
6 sum_i t_i (1 - cos q.c_i) (the cut-off is the lattice; reading recorded in
the design notes), and m the mass of the propagator.

Lattice sums (all over q != 0):
    S1(m)  = V^-1 sum_q G(q)                              (Eq. 31 / kT, Eq. 40)
    S2(m)  = V^-2 sum_{q1, q2} G(q1) G(q2) G(q1 + q2)     (Eq. 32 at k = 0 / kT^2)
             with terms whose q1 + q2 is the zero mode dropped: every
             propagator at the zero mode vanishes, because the order parameter
             is conserved (reading recorded in the design notes)
    S1sq(m) = V^-1 sum_q G(q)^2                           (first term of Eq. 42 at k = 0)

Symmetric phase, Eq. 36:  r' = r + 3 u kT S1(r') - 6 u^2 kT^2 S2(r'),
solved for r' > 0; then chi = 1 / r', xi = sqrt(kappa / r').

Broken phase, Eqs. 40, 42, 43 (r < 0): with r_s = r + 3 u v^2,
    0 = r + u v^2 + 3 u kT S1(r_s)            (Eq. 40 divided by v != 0)
    r'_s = r_s + kT (-18 u^2 v^2 kT S1sq(r_s) + 3 u S1(r_s))
and chi' = 1 / r'_s, xi' = sqrt(kappa / r'_s).  The root v^2 taken is the one
next below the mean-field value -r/u, where fluctuations lower the order
parameter; none exists when fluctuations destroy the order.

Root finding: bisection on a sign-changing bracket (steps below), the plain
method; scipy's brentq would serve equally as a library primitive.
"""

import numpy as np

from .lattice import d2q9, d3q19


def lattice_of(name):
    return d3q19() if name == "D3Q19" else d2q9()


def symbol(side, lat):
    """q^2 of the lattice Laplacian on the S^d grid (shape (S,)*d, numpy FFT order)."""
    d = lat.d
    k = 2.0 * np.pi * np.fft.fftfreq(side) * 1.0          # 2 pi n / S with n wrapped
    grids = np.meshgrid(*([k] * d), indexing="ij")       # axis order irrelevant: the symbol is symmetric
    out = np.zeros((side,) * d)
    for i in range(1, lat.q):
        kc = sum(grids[a] * float(lat.c[i][a]) for a in range(d))
        out += 6.0 * lat.t[i] * (1.0 - np.cos(kc))
    return out


def propagator(side, lat, m, kappa):
    """G(q) with G at the zero mode set to 0."""
    q2 = symbol(side, lat)
    G = 1.0 / (m + kappa * q2)
    G.flat[0] = 0.0
    return G


def s1(G):
    return float(G.sum() / G.size)


def s1sq(G):
    return float((G * G).sum() / G.size)


def s2_brute(G):
    """V^-2 sum over q1, q2 of G(q1) G(q2) G(q1 + q2), as the definition reads (O(N^2))."""
    N = G.size
    d = G.ndim
    total = 0.0
    for idx in np.ndindex(*G.shape):
        g1 = G[idx]
        if g1 == 0.0:
            continue
        # G(q1 + q2) for every q2: the grid shifted by -q1 (periodic)
        shifted = np.roll(G, shift=tuple(-i for i in idx), axis=tuple(range(d)))
        total += g1 * float((G * shifted).sum())
    return total / (N * N)


def s2_fft(G):
    """The same sum through the convolution identity: sum_r g(r)^3 with g = inverse DFT of G."""
    g = np.fft.ifftn(G).real
    return float((g ** 3).sum())


def _bisect(fn, lo, hi, iters=200):
    flo = fn(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        fm = fn(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def symmetric(lattice, side, r, u, kappa, kT, s2=s2_fft):
    """Eq. 36 solved for r' with F(m) = r + 3 u kT S1(m) - 6 u^2 kT^2 S2(m) - m.

    The root taken is the largest one, the branch that tends to r as u -> 0.
    Since S1(m) < 1/m and the two-loop term is negative, F(m) < 0 for
    m > m_up = (max(r, 0) + sqrt(r^2 + 12 u kT)) / 2; from hi = 1.01 m_up the
    bracket end lo is halved until F(lo) > 0 (no root if F stays <= 0 or
    stops being finite), then bisection on [lo, 2 lo]."""
    lat = lattice_of(lattice)

    def F(m):
        G = propagator(side, lat, m, kappa)
        return r + 3.0 * u * kT * s1(G) - 6.0 * u * u * kT * kT * s2(G) - m

    hi = 1.01 * 0.5 * (max(r, 0.0) + np.sqrt(r * r + 12.0 * u * kT))
    if not hi > 0:
        raise ArithmeticError("no root with r' > 0")
    lo = hi
    while True:
        lo *= 0.5
        f = F(lo)
        if not np.isfinite(f) or lo < 1e-300:
            raise ArithmeticError("no root with r' > 0")
        if f > 0:
            break
        hi = lo
    rp = _bisect(F, lo, hi)
    G = propagator(side, lat, rp, kappa)
    return dict(r_prime=rp, chi=1.0 / rp, xi=float(np.sqrt(kappa / rp)), S1=s1(G), S2=s2(G))


def broken(lattice, side, r, u, kappa, kT):
    """Eqs. 40, 42, 43 solved for v (r < 0).  h(w) = r + u w + 3 u kT S1(r + 3 u w)
    for w = v^2: h(-r/u) > 0; w steps down from -r/u by halving its distance to
    the lowest admissible w (where r + 3 u w + kappa q^2_min = 0) until h < 0,
    then bisection on [w_neg, w_pos]."""
    if not (r < 0 and u > 0):
        raise ValueError("the broken phase needs r < 0 and u > 0")
    lat = lattice_of(lattice)
    q2 = symbol(side, lat)
    q2min = float(np.min(q2.flat[1:]))

    def h(w):
        G = propagator(side, lat, r + 3.0 * u * w, kappa)
        return r + u * w + 3.0 * u * kT * s1(G)

    w_mf = -r / u
    w_low = max(0.0, (-r - kappa * q2min) / (3.0 * u))
    w_pos, w_neg = w_mf, None
    w = w_mf
    for _ in range(200):
        w = w_low + 0.5 * (w - w_low)
        if h(w) < 0:
            w_neg = w
            break
        w_pos = w
    if w_neg is None:
        raise ArithmeticError("no ordered solution: fluctuations destroy the order")
    w = _bisect(lambda x: h(x), w_neg, w_pos)
    v = float(np.sqrt(w))
    rs = r + 3.0 * u * w
    G = propagator(side, lat, rs, kappa)
    rps = rs + kT * (-18.0 * u * u * w * kT * s1sq(G) + 3.0 * u * s1(G))
    return dict(v=v, r_sigma=rs, r_prime_sigma=rps, chi=1.0 / rps, xi=float(np.sqrt(kappa / rps)),
                S1=s1(G), S1sq=s1sq(G))

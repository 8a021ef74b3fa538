"""Block observables and structure factor in plain FP64 (test infrastructure).

Sec. II B (Eqs. 46-50): the lattice of side S is divided into blocks of side
L = S/2^i (i = 0, 1, ...; the paper allows powers of two, footnote there) and
  m_L^(b) = L^-d sum_{i in b} phi_i                      (Eq. 46)
  M_L = <|m_L|>                                          (Eq. 47)
  chi_L = L^d/kT (<m_L^2> - <m_L>^2)        (theta > 0)  (Eq. 48)
  chi_L = L^d/kT (<m_L^2> - <|m_L|>^2)      (theta < 0)  (Eq. 49)
  c_H,L = L^d/kT (<E_L^2> - <E_L>^2),  E_L^(b) = (2 L^d)^-1 sum phi_i^2  (Eq. 50)
averaged over all blocks of a level and over samples in time.  phi is the
order parameter of Eq. 1 with rho_0 the global mean density.  U_L =
1 - <m^4>/(3 <m^2>^2) is Binder's cumulant (the paper does not use it; it is
reported as a numerical-accuracy figure).

Levels: block dims (nx/2^i, ny/2^i[, nz/2^i]) for i = 0, 1, ... while every
division is exact, then the single-site level (1, 1, 1) if not yet reached.
For a 2-D lattice the z extent of a block is 1.  Level i = 0 is the whole
system, where m = 0 by mass conservation (kept as a check).

Order-parameter distribution (Sec. II D): P_L(m) is the histogram of the
block values m_L^(b) of a level over all blocks and samples.  Bins (a
convention of this project): nbins equal bins on [lo, hi); a value goes to bin
floor(t) with t = (m - lo) * (nbins / (hi - lo)) evaluated in FP64, below lo to
an underflow count and at or above hi (or NaN) to an overflow count.  From a
histogram symmetric about m = 0 the estimators of Sec. IV (order-parameter
distribution results) are: M_L as the position of the maximum of P_L, chi_L
from the peak height through the Gaussian forms of P_L (Eqs. 57 and 58; one central peak:
chi_L = L^d / (2 pi kT P_max^2); two displaced peaks, each carrying half the
weight: chi_L = L^d / (8 pi kT P_max^2)), and chi_L from the variance of a
Gaussian fitted to the peak (chi_L = L^d sigma^2 / kT), after an optional
central region |m| < m_cut is set to zero (also in the normalisation).

Momentum spectra (Sec. III D, equilibration of momentum, and Eq. 69): the fluid
momentum j = rho u of the collision (j = sum_i c_i f_i with the modified
equilibrium; j + F/2 with the Guo force F = kappa rho grad lap rho), its DFT
J_a(k) = sum_r j_a(r) e^{-i k.r}, and per k the three spectra |J_x|^2 / N,
|khat . J|^2 / N (longitudinal) and (|J|^2 - |khat . J|^2) / (N (d - 1))
(transverse, per component), with khat = n / |n| for k = 2 pi n / S (n wrapped
as below; both projections are 0 at k = 0).  In equilibrium each equals
rho_0 kT (Eq. 69).  They are accumulated on the structure-factor schedule and
binned in the same shells.

Ornstein-Zernike fit (Eq. 25 with the lattice Laplacian's symbol for k^2, as
Sec. IV requires): on shells 1..kmax, 1 / C_j = a + b k2_j by weighted least
squares, with C_j the shell mean of C, k2_j the shell mean of the symbol
6 sum_i t_i (1 - cos k.c_i), and weights (points in shell) x C_j^2 (the inverse
variance of 1 / C_j when C_j has relative error ~ 1/sqrt(points)); then
chi = 1 / (kT a) and xi = sqrt(b / a).

Structure factor (Eq. 80): C(k) = N^-1 |sum_r phi(r) exp(-i k.r)|^2, with the
discrete Fourier transform taken by numpy's FFT (a library primitive).  Shell
binning (a convention of this project): on an S^d lattice, k = 2 pi n / S with
n_a wrapped to [-S/2, S/2), and the point goes to shell j with
j (j - 1) < |n|^2 <= j (j + 1), i.e. the integer nearest to |n|.  Shell 0
(k = 0, where C = 0 by mass conservation) is not reported.
"""

import numpy as np

from . import lbm

ACC_FIELDS = ("n", "sum_m", "sum_m2", "sum_abs_m", "sum_m4", "sum_e", "sum_e2")


def levels(p):
    dims = [p.nx, p.ny] + ([p.nz] if p.nz > 1 or p.lattice == "D3Q19" else [])
    out = []
    i = 0
    while all(n % (1 << i) == 0 and (n >> i) >= 1 for n in dims):
        blk = [n >> i for n in dims]
        if p.nz == 1 and len(blk) == 2:
            blk.append(1)
        out.append(tuple(blk))
        if all(b == 1 for b in blk):
            break
        i += 1
    if out[-1] != (1, 1, 1):
        out.append((1, 1, 1))
    return out


def order_parameter(f):
    """phi = (rho - rho_bar)/rho_bar with rho_bar the global mean (Eq. 1)."""
    rho = lbm.density(f)
    rbar = rho.mean()
    return (rho - rbar) / rbar


def block_means(x, blk):
    """Mean of ``x`` (shape (nz, ny, nx)) over blocks of dims (bx, by, bz)."""
    bx, by, bz = blk
    nz, ny, nx = x.shape
    return x.reshape(nz // bz, bz, ny // by, by, nx // bx, bx).mean(axis=(1, 3, 5))


def sample(phi, lv):
    """Per-level increments of the accumulators for one snapshot of phi."""
    rows = []
    for blk in lv:
        m = block_means(phi, blk).ravel()
        e = 0.5 * block_means(phi * phi, blk).ravel()
        rows.append([m.size, m.sum(), (m * m).sum(), np.abs(m).sum(), (m ** 4).sum(),
                     e.sum(), (e * e).sum()])
    return np.asarray(rows, dtype=np.float64)


def derived(acc, lv, kT):
    """M_L, chi_L (Eqs. 48 and 49), c_H,L (Eq. 50), U_L from accumulated sums."""
    out = []
    for row, blk in zip(acc, lv):
        n = row[0]
        vol = float(blk[0] * blk[1] * blk[2])
        mean_m, m2, am, m4, e, e2 = (row[1:] / n) if n > 0 else (np.nan,) * 6
        out.append({
            "block": blk,
            "M_L": am,
            "m2": m2,
            "m4": m4,
            "chi_L": vol / kT * (m2 - mean_m ** 2),
            "chi_L_lowT": vol / kT * (m2 - am ** 2),
            "c_HL": vol / kT * (e2 - e ** 2),
            "U_L": 1.0 - m4 / (3.0 * m2 * m2) if m2 > 0 else np.nan,
        })
    return out


def structure_factor(phi):
    """C(k) = |sum_r phi(r) e^{-i k.r}|^2 / N over the full k grid (Eq. 80)."""
    F = np.fft.fftn(phi)
    return (F.real ** 2 + F.imag ** 2) / phi.size


def shell_index(shape):
    """Shell j of every k point of a cubic / square lattice (see module docstring)."""
    nz, ny, nx = shape
    sides = [n for n in (nx, ny, nz) if n > 1]
    if len(set(sides)) != 1:
        raise ValueError("shell binning needs equal sides")
    n2 = np.zeros(shape, dtype=np.int64)
    for ax, n in zip((0, 1, 2), (nz, ny, nx)):
        if n == 1:
            continue
        idx = np.arange(n)
        idx = np.where(2 * idx < n, idx, idx - n)             # wrap to [-S/2, S/2)
        shp = [1, 1, 1]
        shp[ax] = n
        n2 = n2 + (idx.reshape(shp) ** 2)
    j = np.floor(np.sqrt(n2.astype(np.float64))).astype(np.int64)
    # exact integer rule j(j-1) < n2 <= j(j+1)
    j = np.where(j * (j + 1) < n2, j + 1, j)
    j = np.where(j * (j - 1) >= n2, j - 1, j)
    j = np.where(n2 == 0, 0, j)
    return j


def bin_shells(ck_sum, shape, nbins):
    """(sum of C over each shell j = 1..nbins, number of k points per shell)."""
    j = shell_index(shape).ravel()
    vals = np.asarray(ck_sum).ravel()
    sums = np.zeros(nbins)
    counts = np.zeros(nbins, dtype=np.int64)
    for b in range(1, nbins + 1):
        sel = j == b
        sums[b - 1] = vals[sel].sum()
        counts[b - 1] = sel.sum()
    return sums, counts


def histogram(m, lo, hi, nbins):
    """[underflow, bin 0 .. nbins-1, overflow] counts of the values ``m``."""
    m = np.asarray(m, dtype=np.float64).ravel()
    inv_w = float(nbins) / (hi - lo)
    t = (m - lo) * inv_w
    out = np.zeros(nbins + 2, dtype=np.int64)
    under = t < 0
    inside = (t >= 0) & (t < nbins)
    out[0] = under.sum()
    out[-1] = m.size - under.sum() - inside.sum()        # t >= nbins or NaN
    np.add.at(out, 1 + np.floor(t[inside]).astype(np.int64), 1)
    return out


def sample_histograms(phi, lv, lo, hi, nbins):
    """Per-level histogram increments of one snapshot of phi."""
    return np.stack([histogram(block_means(phi, blk), lo, hi, nbins) for blk in lv])


def histogram_estimates(counts, lo, hi, vol, kT, m_cut=0.0, frac=0.2):
    """Estimators of M_L and chi_L from one level's histogram (see module docstring).

    The range must be symmetric (lo = -hi).  Steps: bin centres m_k; bins with
    |m_k| < m_cut zeroed; N = kept bins + underflow + overflow; the histogram
    symmetrised, P_s(k) = (c_k + c_{nbins-1-k}) / 2; the peak k* = the first
    maximum of P_s over the upper half m_k >= 0; P_max = P_s(k*) / (N w); the
    peak is central when k* is the innermost upper bin.  The Gaussian fit is a
    least-squares fit of log P_s = alpha + beta m + gamma m^2, weighted by the
    counts, over the contiguous bins around k* with P_s >= frac P_s(k*) (for a
    central peak on both sides of m = 0, else in the upper half);
    sigma^2 = -1 / (2 gamma), centre -beta / (2 gamma).
    """
    counts = np.asarray(counts, dtype=np.float64)
    nb = counts.size - 2
    if not (lo == -hi and hi > 0 and nb >= 2 and vol > 0 and kT > 0):
        raise ValueError("need a symmetric range, >= 2 bins, vol > 0 and kT > 0")
    w = (hi - lo) / nb
    centres = lo + (np.arange(nb) + 0.5) * w
    c = counts[1:-1].copy()
    c[np.abs(centres) < m_cut] = 0.0
    n_all = c.sum() + counts[0] + counts[-1]
    ps = 0.5 * (c + c[::-1])
    k_in = nb // 2                          # innermost bin with centre >= 0
    upper = ps[k_in:]
    nan = float("nan")
    out = dict(m_max=nan, P_max=nan, chi_peak=nan, M_fit=nan, sigma2_fit=nan, chi_fit=nan, n_fit=0,
               central=True, hist_abs_m=nan, hist_m2=nan, n_total=n_all)
    if n_all <= 0 or upper.max() <= 0:
        return out
    ks = k_in + int(np.argmax(upper))
    out["m_max"] = centres[ks]
    out["P_max"] = ps[ks] / (n_all * w)
    central = ks == k_in
    out["central"] = bool(central)
    out["chi_peak"] = vol / ((2.0 if central else 8.0) * np.pi * kT * out["P_max"] ** 2)
    lo_k = ks
    floor = frac * ps[ks]
    kmin = 0 if central else k_in
    while lo_k - 1 >= kmin and ps[lo_k - 1] >= floor:
        lo_k -= 1
    hi_k = ks
    while hi_k + 1 < nb and ps[hi_k + 1] >= floor:
        hi_k += 1
    sel = np.arange(lo_k, hi_k + 1)
    if sel.size >= 3:
        x = centres[sel]
        y = np.log(ps[sel])
        wt = ps[sel]
        A = np.stack([np.ones_like(x), x, x * x], axis=1)
        coef = np.linalg.solve(A.T @ (wt[:, None] * A), A.T @ (wt * y))
        if coef[2] < 0:
            out["sigma2_fit"] = -0.5 / coef[2]
            out["M_fit"] = -coef[1] / (2.0 * coef[2])
            out["chi_fit"] = vol * out["sigma2_fit"] / kT
        out["n_fit"] = int(sel.size)
    kept = c.sum()
    if kept > 0:
        out["hist_abs_m"] = float((np.abs(centres) * c).sum() / kept)
        out["hist_m2"] = float((centres * centres * c).sum() / kept)
    return out


def fluid_momentum(f, p):
    """rho u as the collision defines it (see module docstring); shape (3, nz, ny, nx)."""
    j = lbm.momentum(f, p.lat)
    if p.coupling == "guo":
        rho = lbm.density(f)
        j = j + 0.5 * p.kappa * rho * lbm.gradient(lbm.laplacian(rho, p.lat), p.lat)
    return j


def wavevectors(shape):
    """Integer wavevector components (n_x, n_y, n_z), each wrapped to [-S/2, S/2), on a (nz, ny, nx) grid."""
    nz, ny, nx = shape
    out = []
    for ax, n in ((2, nx), (1, ny), (0, nz)):
        idx = np.arange(n)
        idx = np.where(2 * idx < n, idx, idx - n)
        shp = [1, 1, 1]
        shp[ax] = n
        out.append(np.broadcast_to(idx.reshape(shp), shape).astype(np.float64))
    return out


def momentum_spectra(f, p):
    """(3, nz, ny, nx): |J_x|^2 / N, longitudinal and transverse spectra per k (module docstring)."""
    return spectra_of_momentum(fluid_momentum(f, p), p.lat.d)


def spectra_of_momentum(j, d):
    """The three spectra of a momentum field j (shape (3, nz, ny, nx)) in d dimensions."""
    shape = j.shape[1:]
    N = float(np.prod(shape))
    J = [np.fft.fftn(j[a]) for a in range(d)]
    nvec = wavevectors(shape)[:d]
    nn = np.sqrt(sum(n * n for n in nvec))
    safe = np.where(nn > 0, nn, 1.0)
    par = sum((n / safe) * Ja for n, Ja in zip(nvec, J))
    tot = sum(np.abs(Ja) ** 2 for Ja in J)
    p2 = np.abs(par) ** 2
    out = np.zeros((3,) + shape)
    out[0] = np.abs(J[0]) ** 2 / N
    out[1] = np.where(nn > 0, p2 / N, 0.0)
    out[2] = np.where(nn > 0, (tot - p2) / (N * (d - 1)), 0.0)
    return out


def laplacian_symbol(shape, lat):
    """k^2 of the lattice Laplacian: 6 sum_i t_i (1 - cos k.c_i), k = 2 pi n / S."""
    nz, ny, nx = shape
    nvec = wavevectors(shape)
    k = [2.0 * np.pi * n / s for n, s in zip(nvec, (nx, ny, nz))]
    out = np.zeros(shape)
    for i in range(1, lat.q):
        kc = sum(k[a] * float(lat.c[i][a]) for a in range(3))
        out += 6.0 * lat.t[i] * (1.0 - np.cos(kc))
    return out


def oz_fit(sk_sum, counts, n_samples, shape, lat, kT, kmax):
    """Ornstein-Zernike fit of a shell-binned C(k) (module docstring): dict(chi, xi, a, b, shells)."""
    k2sum, k2cnt = bin_shells(laplacian_symbol(shape, lat), shape, kmax)
    sk_sum = np.asarray(sk_sum, dtype=np.float64)[:kmax]
    counts = np.asarray(counts, dtype=np.float64)[:kmax]
    if not np.array_equal(counts, k2cnt):
        raise ValueError("shell counts do not belong to this lattice")
    use = counts > 0
    C = sk_sum[use] / (counts[use] * n_samples)
    x = k2sum[use] / counts[use]
    y = 1.0 / C
    wt = counts[use] * C * C
    A = np.stack([np.ones_like(x), x], axis=1)
    a, b = np.linalg.solve(A.T @ (wt[:, None] * A), A.T @ (wt * y))
    xi = float(np.sqrt(b / a)) if a > 0 and b >= 0 else float("nan")
    return dict(chi=1.0 / (kT * a), xi=xi, a=float(a), b=float(b), shells=int(use.sum()))


class Recorder:
    """Accumulates block observables (and optionally C(k)) every ``every`` steps.

    A sample is taken at times t > 0 with t % every == 0, from the state f(., t).
    Also records the FP64 mass sum rho and momentum sum j at each sample.
    """

    def __init__(self, p, every, sk_every=0, hist=None, jk=False):
        self.p = p
        self.lv = levels(p)
        self.every = every
        self.sk_every = sk_every
        self.hist_cfg = hist                    # (nbins, lo, hi) or None
        self.hist = np.zeros((len(self.lv), hist[0] + 2), dtype=np.int64) if hist else None
        self.acc = np.zeros((len(self.lv), len(ACC_FIELDS)))
        self.ck = np.zeros(p.shape)
        self.jk = np.zeros((3,) + p.shape) if jk else None
        self.n_sk = 0
        self.mass = []
        self.mom = []

    def __call__(self, f, t):
        if self.every > 0 and t > 0 and t % self.every == 0:
            phi = order_parameter(f)
            self.acc += sample(phi, self.lv)
            if self.hist is not None:
                nb, lo, hi = self.hist_cfg
                self.hist += sample_histograms(phi, self.lv, lo, hi, nb)
            self.mass.append(lbm.density(f).sum())
            self.mom.append(lbm.momentum(f, self.p.lat).reshape(3, -1).sum(axis=1))
        if self.sk_every > 0 and t > 0 and t % self.sk_every == 0:
            self.ck += structure_factor(order_parameter(f))
            if self.jk is not None:
                self.jk += momentum_spectra(f, self.p)
            self.n_sk += 1

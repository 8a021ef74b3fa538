"""One fluctuating lattice Boltzmann time step in plain FP64 (test infrastructure).

Follows Sec. III A of Gross & Varnik (arXiv:1202.4748):

  Eq. 61  f_i(r + c_i, t+1) = f_i - (f_i - f_i^eq)/tau + theta_i      (LBE)
  Eq. 62  rho = sum_i f_i,  rho u = sum_i f_i c_i                     (moments)
  Eq. 63  second moment of f^eq = P + rho u u + nu(u d rho + ...)      (Holdych term)
  Eq. 64  P = (p0 - kappa rho lap rho - kappa/2 |grad rho|^2) 1 + kappa grad rho grad rho
  Eq. 65  explicit modified equilibrium on D2Q9 with weights w, w^xx, w^yy, w^xy
  Eq. 66  f_i = T_ai t_i m_a / N_a                                    (moment basis)
  Eq. 68  covariance of the moment-space noise, local in rho and c_s^2(r)

State convention: ``f`` has shape (q, nz, ny, nx) and holds f_i(r, t) -- the
populations at site r at time t before the collision of step t (i.e. after the
streaming of step t-1).  One step = collide every site, then stream.

Two couplings of the non-ideal thermodynamics:

* ``modeq`` (the paper): the pressure tensor enters through the modified
  equilibrium of Eq. 65; no force.  Readings of printing errors in Eq. 65
  (each forced by the moment condition Eq. 63, pinned in the tests):
    g1  "p0 - rho lap rho"       -> p0 - kappa rho lap rho   (as in Eq. 64)
    g2  missing "+" before u_gamma d_gamma rho delta_ab restored
    g3  "w^xx kappa (d_x rho d_y rho)" -> w^xx kappa (d_x rho)^2
  The printed square-gradient weights are one rotation-invariant expression,
  kappa t_i [(9/2)(c_i . g)^2 + A c_i^2 |g|^2 + B |g|^2], g = grad rho, with
  (A, B) = (-9/2, 3); in d dimensions the second-moment condition of Eq. 63
  (these terms must contribute kappa (g_a g_b - |g|^2 delta_ab / 2)) fixes only
  A (d + 2)/9 + B/3 = -1.  On D3Q19 (the paper prints D2Q9 only) this project
  keeps A = -9/2, the printed set's -(9/2)|c_i x g|^2 structure, so B = 9/2;
  the other terms of Eq. 65 carry over with the isotropic weights 3 t_i, and
  nu is taken from the c_y^2 - c_z^2 shear mode.
* ``guo`` (variant for the 3-D workloads; D2Q9 and D3Q19): the GL force
  -rho grad mu, mu = f0'(phi)/rho_0 - kappa lap rho, is split by the identity
  rho grad(f0'/rho_0) = grad p0.  The bulk part enters as the isotropic
  pressure p0 of the equilibrium (second moment p0 1 + rho u u, made by
  shifting the second-order equilibrium by 3 t_i (p0 - rho/3) on i >= 1 and
  restoring mass on f_0 -- the structure of Eq. 65, whose isotropic weights are
  3 t_i); the square-gradient part is a Guo body force F = kappa rho grad lap rho
  (Guo, Zheng & Shi 2002), u = (j + F/2)/rho, source (1 - lambda_a/2)(T F)_a.
  Two literal all-force readings were rejected on measured grounds: cancelling
  the ideal pressure rho/3 with a force leaves an O(1/12) lattice stiffness
  that adds to kappa; a zero-pressure equilibrium with the whole force leaves
  the density mode at k = pi unrestrained (the force stencil has symbol sin k).

Relaxation is done in moment space with a rate lambda_a = 1/tau_a per mode.
With all tau_a equal this is exactly the single-tau BGK form of Eq. 61,
because T is a complete orthogonal basis.

Noise (Eq. 68): xi = s L n on the non-conserved modes, s^2 = 3 rho kT
(Delta V = Delta t = 1), L the lower Cholesky factor of the bracketed matrix
times the per-mode factor g_ab = 1 - gamma_a gamma_b, gamma_a = 1 - lambda_a,
n the site's normals in draw order.  With equal rates g = (1/tau)(2 - 1/tau),
the prefactor printed in Eq. 68.  For ``guo`` the matrix is the lattice-
general form diag(N_a) + (1 - 3 c_s^2) v v^T, v_a = T_a(c = 0) the basis at the
rest velocity: the conditional covariance of the non-conserved moments under
the exact kappa = 0 stationary state (derived for this project; on D2Q9 it is
Eq. 68 entry by entry, which a test checks).

Gradients (the paper defers the discrete operators to its Ref.
[gross_flb_2010]; parity unpinned by the paper, identical on both sides by
construction):  d_a rho = 3 sum_i t_i c_ia rho(r + c_i),
lap rho = 6 sum_i t_i (rho(r + c_i) - rho(r)).
"""

from dataclasses import dataclass, field

import numpy as np

from . import lattice as _lat
from . import philox


class NonPositiveDensity(ValueError):
    pass


class NoiseNotPositiveDefinite(ValueError):
    pass


@dataclass
class Params:
    lattice: str = "D2Q9"
    coupling: str = "modeq"
    nx: int = 16
    ny: int = 16
    nz: int = 1
    rho_c: float = 1.0     # reference density rho_0 of Eq. 1
    a: float = 0.0         # quadratic Landau coefficient (the paper's r, Eq. 3)
    b: float = 0.1         # quartic Landau coefficient (the paper's u, Eq. 3)
    kappa: float = 0.01    # square-gradient coefficient (Eq. 2)
    kT: float = 1e-4       # noise temperature k_B T
    tau: tuple = field(default_factory=tuple)   # per-mode tau_a (len q); empty -> all 1
    seed: int = 1
    system_id: int = 0

    @property
    def lat(self):
        return _lat.get(self.lattice)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_sites(self):
        return self.nx * self.ny * self.nz

    def taus(self):
        q = self.lat.q
        if len(self.tau) == 0:
            return np.ones(q)
        t = np.asarray(self.tau, dtype=np.float64)
        if t.shape != (q,):
            raise ValueError("tau must have one entry per mode")
        return t


# --------------------------------------------------------------------------
# lattice operators
# --------------------------------------------------------------------------

def shift(field_, c):
    """Value of ``field_`` at r + c on the periodic lattice (last three axes z, y, x)."""
    return np.roll(field_, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(-3, -2, -1))


def density(f):
    """rho = sum_i f_i (Eq. 62)."""
    return f.sum(axis=0)


def momentum(f, lat):
    """j = rho u = sum_i f_i c_i (Eq. 62); shape (3, nz, ny, nx)."""
    return np.tensordot(lat.c.T.astype(np.float64), f, axes=(1, 0))


def gradient(s, lat):
    """d_a s = 3 sum_i t_i c_ia s(r + c_i)."""
    g = np.zeros((3,) + s.shape)
    for i in range(1, lat.q):
        g += 3.0 * lat.t[i] * lat.c[i].astype(np.float64)[:, None, None, None] * shift(s, lat.c[i])
    return g


def laplacian(s, lat):
    """lap s = 6 sum_i t_i (s(r + c_i) - s(r))."""
    out = np.zeros_like(s)
    for i in range(1, lat.q):
        out += 6.0 * lat.t[i] * (shift(s, lat.c[i]) - s)
    return out


def stream(fstar, lat):
    """f_i(r + c_i, t+1) = f*_i(r, t) on the periodic lattice (Eq. 61)."""
    out = np.empty_like(fstar)
    for i in range(lat.q):
        c = lat.c[i]
        out[i] = np.roll(fstar[i], shift=(int(c[2]), int(c[1]), int(c[0])), axis=(0, 1, 2))
    return out


# --------------------------------------------------------------------------
# thermodynamics (Sec. II A, Eqs. 1-3; pressure below Eq. 64)
# --------------------------------------------------------------------------

def landau(rho, p):
    """phi = (rho - rho_0)/rho_0 (Eq. 1), f0 (Eq. 3), d f0/d phi, p0, c_s^2.

    p0 = (rho/rho_0) d_phi f0 - f0 (defined below Eq. 64);
    c_s^2 = d p0 / d rho = (rho/rho_0^2)(r + 3 u phi^2).
    """
    phi = (rho - p.rho_c) / p.rho_c
    f0 = 0.5 * p.a * phi ** 2 + 0.25 * p.b * phi ** 4
    df0 = p.a * phi + p.b * phi ** 3
    p0 = rho / p.rho_c * df0 - f0
    cs2 = rho / p.rho_c ** 2 * (p.a + 3.0 * p.b * phi ** 2)
    return phi, f0, df0, p0, cs2


def kinematic_viscosity(p):
    """nu = (tau - 1/2)/3 (below Eq. 63), tau of a shear mode: c_x^2 - c_y^2 (index 4)
    on D2Q9, c_y^2 - c_z^2 (index 6) on D3Q19."""
    return (p.taus()[4 if p.lattice == "D2Q9" else 6] - 0.5) / 3.0


def modeq_gradient_coefficients(d):
    """(A, B) of the square-gradient terms kappa t_i [(9/2)(c.g)^2 + A c^2 |g|^2 + B |g|^2]:
    the printed D2Q9 values in 2-D, A = -9/2 and B from the second-moment
    condition A (d + 2)/9 + B/3 = -1 in 3-D."""
    if d == 2:
        return -4.5, 3.0
    A = -4.5
    return A, -3.0 * (1.0 + A * (d + 2) / 9.0)


def feq_modeq_d3q19(rho, u, grad, lap, p):
    """Modified equilibrium on D3Q19: Eq. 65's structure with the isotropic
    weights 3 t_i and the rotation-invariant square-gradient terms (module
    docstring), shape (19, ...)."""
    lat = _lat.d3q19()
    nu = kinematic_viscosity(p)
    _, _, _, p0, _ = landau(rho, p)
    iso = p0 - p.kappa * rho * lap
    udg = u[0] * grad[0] + u[1] * grad[1] + u[2] * grad[2]
    g2 = grad[0] ** 2 + grad[1] ** 2 + grad[2] ** 2
    X = [[rho * u[a] * u[b] + nu * (u[a] * grad[b] + u[b] * grad[a] + udg * (a == b)) for b in range(3)]
         for a in range(3)]
    A, B = modeq_gradient_coefficients(3)
    feq = np.empty((19,) + rho.shape)
    for i in range(1, 19):
        c = lat.c[i].astype(np.float64)
        cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
        cg = c[0] * grad[0] + c[1] * grad[1] + c[2] * grad[2]
        c2 = float(c @ c)
        xcc = sum((c[a] * c[b] - (a == b) / 3.0) * X[a][b] for a in range(3) for b in range(3))
        feq[i] = (3.0 * lat.t[i] * (iso + rho * cu + 1.5 * xcc)
                  + p.kappa * lat.t[i] * (4.5 * cg * cg + A * c2 * g2 + B * g2))
    feq[0] = rho - feq[1:].sum(axis=0)
    return feq


def feq_modeq(rho, u, grad, lap, p):
    """Modified equilibrium (Eq. 65, readings g1-g3): the printed D2Q9 form,
    shape (9, ...); on D3Q19 feq_modeq_d3q19."""
    if p.lattice == "D3Q19":
        return feq_modeq_d3q19(rho, u, grad, lap, p)
    lat = _lat.d2q9()
    nu = kinematic_viscosity(p)
    _, _, _, p0, _ = landau(rho, p)
    iso = p0 - p.kappa * rho * lap                                  # reading g1
    ux, uy = u[0], u[1]
    gx, gy = grad[0], grad[1]
    udg = ux * gx + uy * gy
    # X_ab = rho u_a u_b + nu (u_a d_b rho + u_b d_a rho + u.grad rho delta_ab)  (reading g2)
    Xxx = rho * ux * ux + nu * (2 * ux * gx + udg)
    Xyy = rho * uy * uy + nu * (2 * uy * gy + udg)
    Xxy = rho * ux * uy + nu * (ux * gy + uy * gx)
    feq = np.empty((9,) + rho.shape)
    for i in range(1, 9):
        cx, cy = float(lat.c[i, 0]), float(lat.c[i, 1])
        xcc = ((cx * cx - 1 / 3) * Xxx + (cy * cy - 1 / 3) * Xyy + 2 * cx * cy * Xxy)
        feq[i] = (_lat.POOLEY_W[i] * (iso + rho * (cx * ux + cy * uy) + 1.5 * xcc)
                  + p.kappa * (_lat.POOLEY_WXX[i] * gx * gx              # reading g3
                               + _lat.POOLEY_WYY[i] * gy * gy
                               + _lat.POOLEY_WXY[i] * gx * gy))
    feq[0] = rho - feq[1:].sum(axis=0)
    return feq


def feq_standard(rho, u, lat):
    """Second-order equilibrium t_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2)."""
    cu = np.tensordot(lat.c.astype(np.float64), u, axes=(1, 0))
    uu = (u * u).sum(axis=0)
    return lat.t.reshape((-1,) + (1,) * rho.ndim) * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)


def feq_landau_pressure(rho, u, p):
    """Second-order equilibrium whose isotropic pressure is p0 instead of rho/3.

    f_i = t_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2) + 3 t_i (p0 - rho/3), i >= 1;
    f_0 = rho - sum_{i>=1} f_i.  Moments: rho, rho u, p0 1 + rho u u."""
    lat = p.lat
    f = feq_standard(rho, u, lat)
    _, _, _, p0, _ = landau(rho, p)
    tb = lat.t.reshape((-1,) + (1,) * rho.ndim)
    f[1:] += (3.0 * tb * (p0 - rho / 3.0))[1:]
    f[0] = rho - f[1:].sum(axis=0)
    return f


def guo_population_force(u, F, lat):
    """F_i = t_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)] (Guo, Zheng & Shi 2002)."""
    c = lat.c.astype(np.float64)
    cu = np.tensordot(c, u, axes=(1, 0))
    cF = np.tensordot(c, F, axes=(1, 0))
    uF = (u * F).sum(axis=0)
    return lat.t.reshape((-1,) + (1,) * uF.ndim) * (3 * (cF - uF) + 9 * cu * cF)


# --------------------------------------------------------------------------
# noise (Eq. 68)
# --------------------------------------------------------------------------

def relaxation_rates(p):
    """lambda_a = 1/tau_a on non-conserved modes, 0 on the conserved ones."""
    lat = p.lat
    lam = 1.0 / p.taus()
    lam[: lat.n_conserved] = 0.0
    return lam


def noise_matrix(cs2, p):
    """Eq. 68 without the 3 rho kT prefactor, on the non-conserved modes.

    Returns an array (..., K, K), K = q - 1 - d, in mode order.  Entry (a, b)
    is the printed matrix element times g_ab = 1 - gamma_a gamma_b.
    """
    lat = p.lat
    nc = lat.n_conserved
    gamma = 1.0 - relaxation_rates(p)[nc:]
    g = 1.0 - gamma[:, None] * gamma[None, :]
    K = lat.q - nc
    if p.coupling == "modeq" and lat.name == "D2Q9":
        cs2 = np.asarray(cs2, dtype=np.float64)
        M = np.zeros(cs2.shape + (K, K))
        # printed rows/columns 4..9 of Eq. 68 -> our modes 3..8 -> local 0..5
        M[..., 0, 0] = 4.0 * (2.0 - 3.0 * cs2)
        M[..., 0, 5] = 12.0 * (cs2 - 1.0 / 3.0)
        M[..., 5, 0] = 12.0 * (cs2 - 1.0 / 3.0)
        M[..., 1, 1] = 4.0 / 9.0
        M[..., 2, 2] = 1.0 / 9.0
        M[..., 3, 3] = 2.0 / 3.0
        M[..., 4, 4] = 2.0 / 3.0
        M[..., 5, 5] = 16.0 * (5.0 / 4.0 - 0.75 * cs2)
        return M * g
    # lattice-general form; equals the printed Eq. 68 on D2Q9
    v = lat.T[nc:, 0]
    cs2 = np.asarray(cs2, dtype=np.float64)
    M = np.diag(lat.N[nc:]) + (1.0 - 3.0 * cs2)[..., None, None] * np.outer(v, v)
    return M * g


def noise(rho, cs2, t, p, sites=None):
    """Moment-space noise xi on the non-conserved modes, shape (K, nz, ny, nx).

    ``sites``: the global site index (x + nx (y + ny z) in the whole system) of
    every site of ``rho`` in its (z, y, x) order, when ``rho`` is a cut-out;
    default: the sites of the whole system ``p`` in order."""
    lat = p.lat
    K = lat.q - lat.n_conserved
    M = noise_matrix(cs2, p)
    if M.ndim == 2:
        M = np.broadcast_to(M, rho.shape + M.shape)
    flatM = M.reshape((-1, K, K))
    try:
        L = np.linalg.cholesky(flatM)
    except np.linalg.LinAlgError as exc:
        raise NoiseNotPositiveDefinite(str(exc)) from exc
    if sites is None:
        sites = np.arange(p.n_sites, dtype=np.uint64)
    sites = np.asarray(sites, dtype=np.uint64).reshape(-1)
    n = philox.site_normals(sites, t, p.system_id, p.seed, K)        # (K, nsites)
    s = np.sqrt(3.0 * rho.reshape(-1) * p.kT)
    xi = s[None, :] * np.einsum("sab,bs->as", L, n)
    return xi.reshape((K,) + rho.shape)


# --------------------------------------------------------------------------
# the step
# --------------------------------------------------------------------------

def collide(f, t, p, sites=None):
    """Post-collision populations f*_i(r, t) (right-hand side of Eq. 61).

    ``f`` may be a periodic cut-out of a larger system (``p`` then describes
    the cut-out's shape) with ``sites`` its global site indices for the noise
    keys; sites farther than the stencil from the cut-out's edge get the
    whole system's result."""
    lat = p.lat
    rho = density(f)
    if not np.all(rho > 0):
        raise NonPositiveDensity("rho <= 0 at step %d" % t)
    j = momentum(f, lat)
    grad = gradient(rho, lat)
    lap = laplacian(rho, lat)
    lam = relaxation_rates(p)
    lam_b = lam.reshape((-1,) + (1,) * rho.ndim)
    if p.coupling == "modeq":
        u = j / rho
        meq = lat.moments(feq_modeq(rho, u, grad, lap, p))
        src = 0.0
    elif p.coupling == "guo":
        F = p.kappa * rho * gradient(lap, lat)          # -rho grad(-kappa lap rho)
        u = (j + 0.5 * F) / rho
        meq = lat.moments(feq_landau_pressure(rho, u, p))
        src = (1.0 - 0.5 * lam_b) * lat.moments(guo_population_force(u, F, lat))
    else:
        raise ValueError(p.coupling)
    m = lat.moments(f)
    mp = m - lam_b * (m - meq) + src
    if p.kT > 0:
        _, _, _, _, cs2 = landau(rho, p)
        mp[lat.n_conserved:] += noise(rho, cs2, t, p, sites)
    return lat.populations(mp)


def step(f, t, p):
    """f(., t) -> f(., t+1)."""
    return stream(collide(f, t, p), p.lat)


def initial_density(p, amplitude=0.01):
    """rho = rho_c + amplitude (2U - 1), U from Philox draw 0xFF at step 0 (word 0),
    minus its mean so that the global average is rho_c (the paper quenches at
    the critical density; the perturbation recipe is a convention of this project)."""
    sites = np.arange(p.n_sites, dtype=np.uint64)
    w = philox.site_words(sites, 0, p.system_id, philox.INIT_DRAW, p.seed)
    d = amplitude * (2.0 * philox.uniform01(w[0]) - 1.0)
    d = d - d.mean()
    return p.rho_c + d.reshape(p.shape)


def equilibrium_at_rest(rho, p):
    """f = f^eq(rho, u = 0, grad rho) used to start from a density field."""
    lat = p.lat
    zero = np.zeros((3,) + rho.shape)
    if p.coupling == "modeq":
        return feq_modeq(rho, zero, gradient(rho, lat), laplacian(rho, lat), p)
    return feq_landau_pressure(rho, zero, p)


def initial_state(p, amplitude=0.01):
    return equilibrium_at_rest(initial_density(p, amplitude), p)


def run(f, t0, nsteps, p, callback=None):
    """Advance ``nsteps`` steps from time ``t0``; ``callback(f, t)`` after each."""
    for t in range(t0, t0 + nsteps):
        f = step(f, t, p)
        if callback is not None:
            callback(f, t + 1)
    return f

"""Velocity sets, weights and moment bases (oracle side; test infrastructure).

D2Q9 is the paper's lattice (Sec. III A: "simulations are performed on a D2Q9
lattice").  Velocities are stored with three components (c_z = 0 in 2D) so one
code path serves both lattices.

Ordering (a convention of this project, deduced from the printed equilibrium
weights of Eq. 65 -- w^xy = +1/4 on i=5,6 and -1/4 on i=7,8 fixes the
diagonal pairs): the paper's rest velocity (its 9th) is our index 0, then
    1:(1,0) 2:(-1,0) 3:(0,1) 4:(0,-1) 5:(1,1) 6:(-1,-1) 7:(1,-1) 8:(-1,1).

Moment basis (Eq. 66 expands f_i = T_ai t_i m_a / N_a).  The paper cites the
basis of its Ref. [gross_flb_2010] without printing it; it states only that
rows 1-3 give rho, rho u_x, rho u_y, rows 4-6 the stresses and 7-9 the ghost
modes, and the noise matrix of Eq. 68 reduces at c_s^2 = 1/3 to
diag(N_4..N_9) = (4, 4/9, 1/9, 2/3, 2/3, 16).  The rows below are the standard
orthogonal polynomial basis with exactly those squared lengths:
    1, c_x, c_y, 3c^2-2, c_x^2-c_y^2, c_x c_y, (3c^2-4)c_x, (3c^2-4)c_y,
    9c^4-15c^2+2.
Pinned by tests: orthogonality sum_i t_i T_ai T_bi = N_a delta_ab and the six
printed diagonal entries.

D3Q19 (literature variant for the 3-D workloads, not in the paper): rest,
6 face and 12 edge velocities with weights 1/3, 1/18, 1/36, and an orthogonal
19-row polynomial basis (density, momentum, six second-order stresses, nine
ghosts), orthogonality pinned by brute force in the tests.
"""

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Lattice:
    name: str
    d: int                 # spatial dimension
    c: np.ndarray          # (q, 3) integer velocities
    t: np.ndarray          # (q,) lattice weights (sum 1, second moment 1/3)
    T: np.ndarray          # (q, q) moment basis, row a = mode a
    N: np.ndarray          # (q,) squared lengths sum_i t_i T_ai^2

    @property
    def q(self):
        return len(self.t)

    @property
    def n_conserved(self):
        return 1 + self.d

    def moments(self, f):
        """m_a = sum_i T_ai f_i  (first axis of ``f`` is the population index)."""
        return np.tensordot(self.T, f, axes=(1, 0))

    def populations(self, m):
        """f_i = t_i sum_a T_ai m_a / N_a  (Eq. 66)."""
        tinv = (self.t[:, None] * self.T.T) / self.N[None, :]
        return np.tensordot(tinv, m, axes=(1, 0))


def _finish(name, d, c, t, rows):
    c = np.asarray(c, dtype=np.int64)
    t = np.asarray(t, dtype=np.float64)
    T = np.asarray(rows, dtype=np.float64)
    N = (T ** 2 * t[None, :]).sum(axis=1)
    return Lattice(name, d, c, t, T, N)


def d2q9():
    c = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
         (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0)]
    t = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    ca = np.asarray(c, dtype=np.float64)
    cx, cy = ca[:, 0], ca[:, 1]
    c2 = cx * cx + cy * cy
    rows = [np.ones(9), cx, cy,
            3 * c2 - 2, cx * cx - cy * cy, cx * cy,
            (3 * c2 - 4) * cx, (3 * c2 - 4) * cy,
            9 * c2 * c2 - 15 * c2 + 2]
    return _finish("D2Q9", 2, c, t, rows)


def d3q19():
    c = [(0, 0, 0),
         (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
         (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
         (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
         (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
    t = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
    ca = np.asarray(c, dtype=np.float64)
    cx, cy, cz = ca[:, 0], ca[:, 1], ca[:, 2]
    c2 = cx * cx + cy * cy + cz * cz
    rows = [np.ones(19), cx, cy, cz,
            c2 - 1, 3 * cx * cx - c2, cy * cy - cz * cz,
            cx * cy, cy * cz, cz * cx,
            (3 * c2 - 5) * cx, (3 * c2 - 5) * cy, (3 * c2 - 5) * cz,
            (cy * cy - cz * cz) * cx, (cz * cz - cx * cx) * cy, (cx * cx - cy * cy) * cz,
            3 * c2 * c2 - 6 * c2 + 1,
            (2 * c2 - 3) * (3 * cx * cx - c2), (2 * c2 - 3) * (cy * cy - cz * cz)]
    return _finish("D3Q19", 3, c, t, rows)


def get(name):
    return {"D2Q9": d2q9, "D3Q19": d3q19}[name]()


# Equilibrium weights of the modified equilibrium on D2Q9 (Eq. 65), indexed
# like the velocities above (entry 0 unused: f_0 follows from mass).
POOLEY_W = np.array([0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 1 / 12, 1 / 12, 1 / 12, 1 / 12])
POOLEY_WXX = np.array([0, 1 / 3, 1 / 3, -1 / 6, -1 / 6, -1 / 24, -1 / 24, -1 / 24, -1 / 24])
POOLEY_WYY = np.array([0, -1 / 6, -1 / 6, 1 / 3, 1 / 3, -1 / 24, -1 / 24, -1 / 24, -1 / 24])
POOLEY_WXY = np.array([0, 0, 0, 0, 0, 1 / 4, 1 / 4, -1 / 4, -1 / 4])

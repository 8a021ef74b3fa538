"""Exact stationary statics of the oracle's step, linearised about a uniform rest state.

Test helper (not part of the oracle).  The linearised step is translation
invariant, so in Fourier space it is one q x q matrix J_k per wave vector k.
J_k is built from the response of the oracle's deterministic step (kT = 0) to
a perturbation of each population at one site (central differences).  The
noise enters as the local covariance of Eq. 68 mapped to populations and
streamed, Q_k = D_k Q_loc D_k^H with D_k = diag(exp(-i k.c_i)).  The stationary
covariance per unit volume then solves the discrete Lyapunov equation
    S_k = J_k S_k J_k^H + Q_loc(k).
"""
import dataclasses

import numpy as np
import scipy.linalg

from oracle import lbm


def rest_state(p):
    rho = np.full(p.shape, p.rho_c)
    return lbm.equilibrium_at_rest(rho, p)


def site_response(p, eps=1e-5):
    """R[i, j, z, y, x] = d f_i(r, t+1) / d f_j(0, t) about the uniform rest state
    (central differences: the quadratic terms of the step cancel exactly, the
    cubic ones leave O(eps^2); eps = 1e-5 keeps the rounding error of the
    difference, O(1e-16 / eps), at the same few 1e-10)."""
    pd = dataclasses.replace(p, kT=0.0)
    f0 = rest_state(pd)
    q = p.lat.q
    R = np.empty((q, q) + p.shape)
    for j in range(q):
        e = np.zeros_like(f0)
        e[j, 0, 0, 0] = eps
        R[:, j] = (lbm.step(f0 + e, 0, pd) - lbm.step(f0 - e, 0, pd)) / (2 * eps)
    return R


def k_grid(p):
    kz = 2 * np.pi * np.fft.fftfreq(p.nz)
    ky = 2 * np.pi * np.fft.fftfreq(p.ny)
    kx = 2 * np.pi * np.fft.fftfreq(p.nx)
    return np.meshgrid(kz, ky, kx, indexing="ij")


def jk_all(R):
    """J_k[i, j] = sum_r R[i, j, r] exp(-i k.r) for every k of the lattice."""
    return np.fft.fftn(R, axes=(2, 3, 4))


def local_noise_population_cov(p):
    lat = p.lat
    nc = lat.n_conserved
    _, _, _, _, cs2 = lbm.landau(np.float64(p.rho_c), p)
    M = 3.0 * p.rho_c * p.kT * lbm.noise_matrix(cs2, p)
    tinv = (lat.t[:, None] * lat.T.T) / lat.N[None, :]
    A = tinv[:, nc:]
    return A @ M @ A.T


def stationary_covariances(p, R=None, skipped=None):
    """Dict k-index -> S_k for all k != 0 (per-site normalisation).

    Wave vectors whose J_k has an eigenvalue of modulus 1 carry a lattice
    invariant (e.g. the longitudinal momentum at k_a = pi, which streaming
    flips in sign and the collision conserves); the Lyapunov equation has no
    unique solution there, so they are left out and listed in ``skipped``."""
    if R is None:
        R = site_response(p)
    J = jk_all(R)
    Ql = local_noise_population_cov(p)
    KZ, KY, KX = k_grid(p)
    c = p.lat.c.astype(float)
    out = {}
    for idx in np.ndindex(*p.shape):
        if idx == (0, 0, 0):
            continue
        k = np.array([KX[idx], KY[idx], KZ[idx]])
        D = np.diag(np.exp(-1j * (c @ k)))
        Q = D @ Ql @ D.conj().T
        Jk = J[(slice(None), slice(None)) + idx]
        if np.max(np.abs(np.linalg.eigvals(Jk))) > 1 - 1e-9:
            if skipped is not None:
                skipped.append(idx)
            continue
        out[idx] = scipy.linalg.solve_discrete_lyapunov(Jk, Q)
    return out


def laplacian_symbol(p, idx):
    KZ, KY, KX = k_grid(p)
    k = np.array([KX[idx], KY[idx], KZ[idx]])
    lat = p.lat
    return -sum(6 * lat.t[i] * (np.cos(lat.c[i] @ k) - 1) for i in range(1, lat.q))

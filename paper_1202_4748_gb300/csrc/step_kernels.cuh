// Fused fluctuating LB time step (Eq. 61): pull-stream, moments (Eq. 62),
// density gradients from a shared-memory halo, equilibrium (Eq. 65 or the
// Landau-pressure form with a Guo body force), relaxation (Eq. 66), local
// Cholesky-factored noise (Eq. 68), aligned store.
//
// Storage: per system, SoA populations [q][z][y][x] holding deviations
// delta f_i = f_i - f^eq_i(rho_c, u = 0), i.e. f_0 - rho_c on the rest velocity
// and f_i elsewhere.  The buffer read by step t holds the post-collision
// populations of step t-1 at their origin sites, so the pre-collision value
// f_i(r, t) is pulled from r - c_i and every store is aligned.
//
// Relaxation: when every non-conserved mode relaxes at one rate (the paper's
// single-tau BGK form of Eq. 61, and tau = 1 in every workload) the update is
// done on the populations, f <- f - lam (f - f^eq) + (1 - lam/2) F_i + T^-1 xi,
// which equals the moment-space form because T is linear and invertible;
// otherwise each moment relaxes at its own rate in the basis of Eq. 66.
#pragma once

#include "collide_d2q9.cuh"
#include "collide_d3q19.cuh"
#include "lb_device.cuh"

namespace lbf {

template <class Real>
struct StepArgs {
    const SysDev* sys;
    const SysPhys<Real>* phys;   // per-system physics in the kernel's precision
    const int4* tiles;        // (system, x0, y0, z0) per CTA
    const Real* fin;
    Real* fout;
    const int64_t* step_ptr;  // device step counter at the start of the chunk
    int k;                    // offset of this step inside the chunk
    int* status;
};

template <class L, int CP>
struct HaloOf {
    static constexpr int H = CP == GUO ? 2 : 1;     // rho needed up to distance H
    static constexpr int HZ = L::D == 3 ? H : 0;
};

// Linear site index inside a system.
__device__ __forceinline__ int site_index(int x, int y, int z, int nx, int ny) { return x + nx * (y + ny * z); }

// Wrapped neighbour coordinates of a site inside its system, as index offsets:
// X[1 + d] = x + d, Y[1 + d] = (y + d) nx, Z[1 + d] = (z + d) nx ny  (d = -1, 0, 1).
struct Nbr {
    int X[3], Y[3], Z[3];
    __device__ __forceinline__ Nbr(int x, int y, int z, int nx, int ny, int nz, bool d3) {
        X[0] = x == 0 ? nx - 1 : x - 1;
        X[1] = x;
        X[2] = x == nx - 1 ? 0 : x + 1;
        Y[0] = (y == 0 ? ny - 1 : y - 1) * nx;
        Y[1] = y * nx;
        Y[2] = (y == ny - 1 ? 0 : y + 1) * nx;
        if (d3) {
            const int pl = nx * ny;
            Z[0] = (z == 0 ? nz - 1 : z - 1) * pl;
            Z[1] = z * pl;
            Z[2] = (z == nz - 1 ? 0 : z + 1) * pl;
        } else {
            Z[0] = Z[1] = Z[2] = 0;
        }
    }
    // index of r + c for a compile-time velocity c
    template <int CX, int CY, int CZ>
    __device__ __forceinline__ int at() const { return X[1 + CX] + Y[1 + CY] + Z[1 + CZ]; }
};

// Neighbourhood views of a shared-memory field around the collided site:
// at<cx, cy, cz>() is the value at r + c.
template <class Real, int PX, int PY>
struct TileView {          // one 3-D block with row pitch PX and plane pitch PX * PY
    const Real* p;
    int c;
    template <int CX, int CY, int CZ>
    __device__ __forceinline__ Real at() const { return p[c + CX + PX * (CY + PY * CZ)]; }
};
template <class Real, int PX>
struct RingView {          // three planes (z - 1, z, z + 1) at arbitrary offsets, row pitch PX
    const Real* p;
    int zm, z0, zp, c;
    template <int CX, int CY, int CZ>
    __device__ __forceinline__ Real at() const {
        return p[(CZ == 0 ? z0 : (CZ > 0 ? zp : zm)) + c + CX + PX * CY];
    }
};

// Pull all q populations of the site described by `nb` (f_i(r) = buf_i(r - c_i)).
template <class L, class Real>
__device__ __forceinline__ void pull_site(const Real* __restrict__ fb, int N, const Nbr& nb, Real (&f)[L::Q]) {
    sfor<0, L::Q>([&](auto I) {
        constexpr int i = I;
        f[i] = fb[i * N + nb.template at<-L::c(i, 0), -L::c(i, 1), -L::c(i, 2)>()];
    });
}

// Moment-space noise of Eq. 68 on the non-conserved modes: xi[a - NC].
// TAU1: every non-conserved mode fully relaxed (tau = 1), so g_ab = 1 and the
// amplitudes are the lattice constants sqrt(N_a); the per-system tables are
// not read.
template <class L, class Real, bool TAU1 = false>
__device__ __forceinline__ void noise_modes(const SysDev& S, const SysPhys<Real>& P, uint32_t site, int64_t step,
                                            Real rho, Real cs2, Real (&xi)[L::Q - L::NC], int* status) {
    constexpr int Q = L::Q;
    constexpr int K = Q - L::NC;
    constexpr int NDRAW = (K + 3) / 4;
    Real nrm[4 * NDRAW];
    sfor<0, NDRAW>([&](auto D) {
        constexpr int d = D;
        const uint4 w = site_draw(S, site, step, uint32_t(d));
        box_muller(w.x, w.y, nrm[4 * d + 0], nrm[4 * d + 1]);
        box_muller(w.z, w.w, nrm[4 * d + 2], nrm[4 * d + 3]);
    });
    const Real sc = fast_sqrt(Real(3) * (rho > Real(0) ? rho : Real(0)) * P.kT);
    // the coupled pair (MP, MR): M = [N + (1 - 3 c_s^2) v v^T] g, v_a = T_a(c = 0)
    constexpr int MP = L::PP, MR = L::PR;
    constexpr double vP = double(L::T(MP, 0)), vR = double(L::T(MR, 0));
    constexpr double NP = norm2<L>(MP), NR = norm2<L>(MR);
    const Real om = Real(1) - Real(3) * cs2;
    const Real gP = TAU1 ? Real(1) : P.g_diag[MP], gR = TAU1 ? Real(1) : P.g_diag[MR];
    const Real Mpp = (Real(NP) + om * Real(vP * vP)) * gP;
    const Real Mrr = (Real(NR) + om * Real(vR * vR)) * gR;
    const Real Mpr = om * Real(vP * vR) * (TAU1 ? Real(1) : P.g_pair);
    const Real det = Mpp * Mrr - Mpr * Mpr;
    if (Mpp > Real(0) && det > Real(0)) {
        const Real r = fast_rsqrt(Mpp);
        const Real l11 = Mpp * r;
        const Real l21 = Mpr * r;
        const Real l22 = fast_sqrt(det) * r;
        const Real nP = nrm[MP - L::NC], nR = nrm[MR - L::NC];
        xi[MP - L::NC] = sc * l11 * nP;
        xi[MR - L::NC] = sc * (l21 * nP + l22 * nR);
    } else {
        atomicOr(status, ST_NOISE);
        xi[MP - L::NC] = Real(0);
        xi[MR - L::NC] = Real(0);
    }
    sfor<L::NC, Q>([&](auto A) {
        constexpr int a = A;
        if constexpr (a != MP && a != MR) {
            const Real amp = TAU1 ? Real(sqrt(norm2<L>(a))) : P.namp[a];
            xi[a - L::NC] = sc * amp * nrm[a - L::NC];
        }
    });
}

// f_i = t_i sum_a T_ai w_a / N_a for a full moment vector w, using the pairs
// (i, i+1), i odd, of opposite velocities: f_i = E + O, f_{i+1} = E - O with E
// (O) the sum over modes even (odd) in c.
template <class L, class Real>
__device__ __forceinline__ void from_moments(const Real (&w)[L::Q], Real (&out)[L::Q]) {
    {
        Real s = Real(0);
        sfor<0, L::Q>([&](auto A) {
            constexpr int a = A;
            constexpr double coef = tinv<L>(0, a);
            if constexpr (coef != 0.0) s += Real(coef) * w[a];
        });
        out[0] = s;
    }
    sfor<0, (L::Q - 1) / 2>([&](auto P) {
        constexpr int i = 1 + 2 * int(P);
        Real e = Real(0), o = Real(0);
        sfor<0, L::Q>([&](auto A) {
            constexpr int a = A;
            constexpr double coef = tinv<L>(i, a);
            if constexpr (coef != 0.0) {
                if constexpr (mode_parity<L>(a) > 0) e += Real(coef) * w[a];
                else o += Real(coef) * w[a];
            }
        });
        out[i] = e + o;
        out[i + 1] = e - o;
    });
}

// Single-rate collision of the Landau-pressure / Guo form in moment space with
// closed-form moments (lattice-general, derived from the equilibrium of the
// population form):  for a non-conserved mode a,
//   m^eq_a - T_a(0) rho_c = T_a(0) (drho - 3 p0) + 9/2 rho u.M_a.u,
//   (T F_i)_a = 9 u.M_a.F,   M_a,bc = sum_i t_i T_ai c_ib c_ic,
// and f <- (1 - lam) f + T^-1 w with w = (lam drho, lam j + F, lam m^eq + (1 - lam/2) F^ + xi).
// j = sum_i c_i f_i (Eq. 62), summed in population order.
template <class L, class Real>
__device__ __forceinline__ void momentum_of(const Real (&f)[L::Q], Real (&j)[3]) {
    j[0] = j[1] = j[2] = Real(0);
    sfor<1, L::Q>([&](auto I) {
        constexpr int i = I;
        sfor<0, L::D>([&](auto A) {
            constexpr int a = A;
            if constexpr (L::c(i, a) == 1) j[a] += f[i];
            if constexpr (L::c(i, a) == -1) j[a] -= f[i];
        });
    });
}

// Single-rate Guo collision from the conserved moments (drho, j) of the site;
// f holds the pre-collision populations on entry unless TAU1 (fully relaxed:
// the update does not read them) and the post-collision ones on exit.
template <class L, class Real, bool TAU1, class LapV>
__device__ __forceinline__ void collide_guo_bgk_m(Real (&f)[L::Q], const Real drho, const Real (&j)[3], const LapV& lv,
                                                  const SysDev& S, const SysPhys<Real>& P, const uint32_t site,
                                                  const int64_t step, int* status) {
    constexpr int Q = L::Q;
    constexpr int K = Q - L::NC;
    const Real rho = P.rho_c + drho;
    if (!(rho > Real(0))) atomicOr(status, ST_RHO);
    const Real irc = P.inv_rho_c;
    const Real phi = drho * irc;
    const Real A_ = P.a, B_ = P.b, kap = P.kappa;
    const Real df0 = phi * (A_ + B_ * phi * phi);
    const Real f0 = phi * phi * (Real(0.5) * A_ + Real(0.25) * B_ * phi * phi);
    const Real p0 = rho * irc * df0 - f0;
    const Real cs2 = rho * irc * irc * (A_ + Real(3) * B_ * phi * phi);
    // Guo body force F = kappa rho grad(lap rho)
    Real gl[3] = {Real(0), Real(0), Real(0)};
    sfor<1, Q>([&](auto I) {
        constexpr int i = I;
        const Real ln = lv.template at<L::c(i, 0), L::c(i, 1), L::c(i, 2)>();
        sfor<0, L::D>([&](auto A) {
            constexpr int a = A;
            if constexpr (L::c(i, a) != 0) gl[a] += Real(3.0 * L::w(i) * L::c(i, a)) * ln;
        });
    });
    const Real ir = fast_rcp(rho);
    Real u[3] = {Real(0), Real(0), Real(0)}, F[3] = {Real(0), Real(0), Real(0)};
    sfor<0, L::D>([&](auto A) {
        constexpr int a = A;
        F[a] = kap * rho * gl[a];
        u[a] = (j[a] + Real(0.5) * F[a]) * ir;
    });
    Real xi[K];
    sfor<0, K>([&](auto A) { xi[decltype(A)::value] = Real(0); });
    if (P.kT > Real(0)) noise_modes<L, Real, TAU1>(S, P, site, step, rho, cs2, xi, status);

    const Real lam = TAU1 ? Real(1) : P.lam_bgk;
    const Real fs = Real(1) - Real(0.5) * lam;
    const Real iso = drho - Real(3) * p0;
    const Real r45 = Real(4.5) * rho;
    Real w[Q];
    w[0] = lam * drho;
    sfor<0, L::D>([&](auto A) {
        constexpr int a = A;
        w[1 + a] = lam * j[a] + F[a];
    });
    sfor<L::NC, Q>([&](auto A) {
        constexpr int a = A;
        Real uMu = Real(0), uMF = Real(0);
        sfor<0, L::D>([&](auto B) {
            constexpr int b = B;
            sfor<0, L::D>([&](auto C) {
                constexpr int c = C;
                constexpr double m = mproj<L>(a, b, c);
                if constexpr (m != 0.0) {
                    uMu += Real(m) * u[b] * u[c];
                    uMF += Real(m) * u[b] * F[c];
                }
            });
        });
        Real meq = r45 * uMu;
        if constexpr (L::T(a, 0) != 0) meq += Real(L::T(a, 0)) * iso;
        w[a] = lam * meq + fs * Real(9) * uMF + xi[a - L::NC];
    });
    if constexpr (TAU1) {
        from_moments<L, Real>(w, f);          // the pre-collision f is fully relaxed away
    } else {
        Real out[Q];
        from_moments<L, Real>(w, out);
        const Real keep = Real(1) - lam;
        sfor<0, Q>([&](auto I) {
            constexpr int i = I;
            f[i] = keep * f[i] + out[i];
        });
    }
}

template <class L, class Real, bool TAU1, class LapV>
__device__ __forceinline__ void collide_guo_bgk(Real (&f)[L::Q], const Real drho, const LapV& lv, const SysDev& S,
                                                const SysPhys<Real>& P, const uint32_t site, const int64_t step,
                                                int* status) {
    Real j[3];
    momentum_of<L, Real>(f, j);
    collide_guo_bgk_m<L, Real, TAU1>(f, drho, j, lv, S, P, site, step, status);
}

// Collision of one site given its pulled deviations f[], the density halo and
// (Guo) the Laplacian halo.  Returns post-collision deviations in f[].
// TAU1 (with BGK_ONLY): the single rate is 1, so f is replaced by the
// equilibrium (plus force) and the noise amplitudes are the lattice constants.
template <class L, int CP, class Real, bool BGK_ONLY, class RhoV, class LapV, bool TAU1 = false>
__device__ __forceinline__ void collide_site(Real (&f)[L::Q], const Real drho, const RhoV& rv, const LapV& lv,
                                             const SysDev& S, const SysPhys<Real>& P, const uint32_t site,
                                             const int64_t step, int* status) {
    constexpr int Q = L::Q;
    constexpr int K = Q - L::NC;
    const Real rho = P.rho_c + drho;
    if (!(rho > Real(0))) atomicOr(status, ST_RHO);

    // conserved moments j = sum_i c_i f_i
    Real j[3] = {Real(0), Real(0), Real(0)};
    sfor<1, Q>([&](auto I) {
        constexpr int i = I;
        sfor<0, L::D>([&](auto A) {
            constexpr int a = A;
            if constexpr (L::c(i, a) == 1) j[a] += f[i];
            if constexpr (L::c(i, a) == -1) j[a] -= f[i];
        });
    });

    // thermodynamics (Eqs. 1, 3 and below Eq. 64)
    const Real irc = P.inv_rho_c;
    const Real phi = drho * irc;
    const Real A_ = P.a, B_ = P.b, kap = P.kappa;
    const Real df0 = phi * (A_ + B_ * phi * phi);
    const Real f0 = phi * phi * (Real(0.5) * A_ + Real(0.25) * B_ * phi * phi);
    const Real p0 = rho * irc * df0 - f0;
    const Real cs2 = rho * irc * irc * (A_ + Real(3) * B_ * phi * phi);

    Real feq[BGK_ONLY ? 1 : Q];
    Real fsrc[BGK_ONLY ? 1 : Q];   // Guo population force
    Real F[3] = {Real(0), Real(0), Real(0)};
    // single-rate update f <- f - lam (f - f^eq) + (1 - lam/2) F_i done in the loops below
    const Real lam_b = P.lam_bgk;
    const Real fs_b = Real(1) - Real(0.5) * lam_b;
    if constexpr (CP == MODEQ) {
        // d_a rho = 3 sum_i t_i c_ia rho(r+c_i);  lap rho = 6 sum_i t_i (rho(r+c_i) - rho(r))
        Real g[2] = {Real(0), Real(0)};
        Real lap = Real(0);
        sfor<1, Q>([&](auto I) {
            constexpr int i = I;
            const Real rn = rv.template at<L::c(i, 0), L::c(i, 1), L::c(i, 2)>();
            if constexpr (L::c(i, 0) != 0) g[0] += Real(3.0 * L::w(i) * L::c(i, 0)) * rn;
            if constexpr (L::c(i, 1) != 0) g[1] += Real(3.0 * L::w(i) * L::c(i, 1)) * rn;
            lap += Real(6.0 * L::w(i)) * (rn - drho);
        });
        const Real ir = fast_rcp(rho);
        const Real ux = j[0] * ir, uy = j[1] * ir;
        const Real nu = P.nu;
        const Real iso = p0 - kap * rho * lap;                     // p0 - kappa rho lap rho
        const Real udg = ux * g[0] + uy * g[1];
        // X_ab = rho u_a u_b + nu (u_a d_b rho + u_b d_a rho + u.grad rho delta_ab)
        const Real Xxx = rho * ux * ux + nu * (Real(2) * ux * g[0] + udg);
        const Real Xyy = rho * uy * uy + nu * (Real(2) * uy * g[1] + udg);
        const Real Xxy = rho * ux * uy + nu * (ux * g[1] + uy * g[0]);
        const Real gxx = kap * g[0] * g[0], gyy = kap * g[1] * g[1], gxy = kap * g[0] * g[1];
        Real s = Real(0);
        sfor<1, Q>([&](auto I) {
            constexpr int i = I;
            constexpr int cx = L::c(i, 0), cy = L::c(i, 1);
            const Real xcc = Real(cx * cx - 1.0 / 3.0) * Xxx + Real(cy * cy - 1.0 / 3.0) * Xyy +
                             Real(2.0 * cx * cy) * Xxy;
            Real cu;
            if constexpr (cx == 0) cu = Real(cy) * uy;
            else if constexpr (cy == 0) cu = Real(cx) * ux;
            else cu = Real(cx) * ux + Real(cy) * uy;
            Real v = Real(pooley_w(i)) * (iso + rho * cu + Real(1.5) * xcc) + Real(pooley_wxx(i)) * gxx +
                     Real(pooley_wyy(i)) * gyy;
            if constexpr (pooley_wxy(i) != 0.0) v += Real(pooley_wxy(i)) * gxy;
            s += v;
            if constexpr (BGK_ONLY && TAU1) f[i] = v;
            else if constexpr (BGK_ONLY) f[i] -= lam_b * (f[i] - v);
            else feq[i] = v;
        });
        // deviation form of f_0 = rho - sum_{i>=1} f_i
        if constexpr (BGK_ONLY && TAU1) f[0] = drho - s;
        else if constexpr (BGK_ONLY) f[0] -= lam_b * (f[0] - (drho - s));
        else feq[0] = drho - s;
    } else {
        // Guo body force F = kappa rho grad(lap rho)
        Real gl[3] = {Real(0), Real(0), Real(0)};
        sfor<1, Q>([&](auto I) {
            constexpr int i = I;
            const Real ln = lv.template at<L::c(i, 0), L::c(i, 1), L::c(i, 2)>();
            sfor<0, L::D>([&](auto A) {
                constexpr int a = A;
                if constexpr (L::c(i, a) != 0) gl[a] += Real(3.0 * L::w(i) * L::c(i, a)) * ln;
            });
        });
        const Real ir = Real(1) / rho;
        Real u[3] = {Real(0), Real(0), Real(0)};
        sfor<0, L::D>([&](auto A) {
            constexpr int a = A;
            F[a] = kap * rho * gl[a];
            u[a] = (j[a] + Real(0.5) * F[a]) * ir;
        });
        const Real uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const Real uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
        const Real p3 = Real(3) * p0;
        Real s = Real(0);
        sfor<1, Q>([&](auto I) {
            constexpr int i = I;
            Real cu = Real(0), cF = Real(0);
            sfor<0, L::D>([&](auto A) {
                constexpr int a = A;
                if constexpr (L::c(i, a) == 1) {
                    cu += u[a];
                    cF += F[a];
                }
                if constexpr (L::c(i, a) == -1) {
                    cu -= u[a];
                    cF -= F[a];
                }
            });
            constexpr double wi = L::w(i);
            const Real v = Real(wi) * (p3 + rho * (Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * uu));
            const Real src = Real(wi) * (Real(3) * (cF - uF) + Real(9) * cu * cF);
            s += v;
            if constexpr (BGK_ONLY) {
                f[i] -= lam_b * (f[i] - v);
                f[i] += fs_b * src;
            } else {
                feq[i] = v;
                fsrc[i] = src;
            }
        });
        if constexpr (BGK_ONLY) {
            f[0] -= lam_b * (f[0] - (drho - s));
            f[0] += fs_b * Real(-3.0 * L::w(0)) * uF;
        } else {
            feq[0] = drho - s;
            fsrc[0] = Real(-3.0 * L::w(0)) * uF;
        }
    }

    Real xi[K];
    sfor<0, K>([&](auto A) { xi[decltype(A)::value] = Real(0); });
    if (P.kT > Real(0)) noise_modes<L, Real, BGK_ONLY && TAU1>(S, P, site, step, rho, cs2, xi, status);

    if constexpr (BGK_ONLY) {
        // f already relaxed and forced; add the noise through f_i += sum_a t_i T_ai xi_a / N_a
        sfor<0, Q>([&](auto I) {
            constexpr int i = I;
            Real v = f[i];
            sfor<L::NC, Q>([&](auto A) {
                constexpr int a = A;
                constexpr double coef = tinv<L>(i, a);
                if constexpr (coef != 0.0) v += Real(coef) * xi[a - L::NC];
            });
            f[i] = v;
        });
        return;
    } else {
    if (S.bgk) {
        // single relaxation rate: population-space update plus T^-1 xi
        const Real lam = P.lam_bgk;
        const Real fs = Real(1) - Real(0.5) * lam;
        sfor<0, Q>([&](auto I) {
            constexpr int i = I;
            Real v = f[i] - lam * (f[i] - feq[i]);
            if constexpr (CP == GUO) v += fs * fsrc[i];
            sfor<L::NC, Q>([&](auto A) {
                constexpr int a = A;
                constexpr double coef = tinv<L>(i, a);
                if constexpr (coef != 0.0) v += Real(coef) * xi[a - L::NC];
            });
            f[i] = v;
        });
        return;
    }

    // per-mode rates: moments of f (deviation), relaxation of the non-conserved ones
    Real m[Q];
    sfor<0, Q>([&](auto A) {
        constexpr int a = A;
        Real s = Real(0);
        sfor<0, Q>([&](auto I) {
            constexpr int i = I;
            constexpr int t = L::T(a, i);
            if constexpr (t == 1) s += f[i];
            else if constexpr (t == -1) s -= f[i];
            else if constexpr (t != 0) s += Real(t) * f[i];
        });
        m[a] = s;
    });
    sfor<L::NC, Q>([&](auto A) {
        constexpr int a = A;
        Real me = Real(0);
        sfor<0, Q>([&](auto I) {
            constexpr int i = I;
            constexpr int t = L::T(a, i);
            if constexpr (t == 1) me += feq[i];
            else if constexpr (t == -1) me -= feq[i];
            else if constexpr (t != 0) me += Real(t) * feq[i];
        });
        const Real lam = P.lam[a];
        m[a] -= lam * (m[a] - me);
        if constexpr (CP == GUO) {
            Real fh = Real(0);
            sfor<0, Q>([&](auto I) {
                constexpr int i = I;
                constexpr int t = L::T(a, i);
                if constexpr (t == 1) fh += fsrc[i];
                else if constexpr (t == -1) fh -= fsrc[i];
                else if constexpr (t != 0) fh += Real(t) * fsrc[i];
            });
            m[a] += (Real(1) - Real(0.5) * lam) * fh;
        }
        m[a] += xi[a - L::NC];
    });
    if constexpr (CP == GUO) {
        sfor<0, L::D>([&](auto A) {
            constexpr int a = A;
            m[1 + a] += F[a];   // (T F)_a = F_a on the momentum rows
        });
    }
    // back to populations: f_i = t_i sum_a T_ai m_a / N_a
    sfor<0, Q>([&](auto I) {
        constexpr int i = I;
        Real s = Real(0);
        sfor<0, Q>([&](auto A) {
            constexpr int a = A;
            constexpr double coef = tinv<L>(i, a);
            if constexpr (coef != 0.0) s += Real(coef) * m[a];
        });
        f[i] = s;
    });
    }
}

template <class L, int CP, class Real, int TX, int TY, int TZ, int MODE>
__global__ void __launch_bounds__(TX* TY* TZ)
    step_kernel(const StepArgs<Real> A) {
    constexpr bool BGK_ONLY = MODE >= 1;
    constexpr bool TAU1 = MODE == 2;
    constexpr int Q = L::Q;
    constexpr int H = HaloOf<L, CP>::H;
    constexpr int HZ = HaloOf<L, CP>::HZ;
    constexpr int SX = TX + 2 * H, SY = TY + 2 * H, SZ = TZ + 2 * HZ;
    constexpr int LX = TX + 2, LY = TY + 2, LZ = L::D == 3 ? TZ + 2 : TZ;   // Laplacian halo (Guo)
    constexpr int NT = TX * TY * TZ;
    __shared__ Real srho[SX * SY * SZ];
    __shared__ Real slap[CP == GUO ? LX * LY * LZ : 1];

    const int4 tl = A.tiles[blockIdx.x];
    const SysDev& S = A.sys[tl.x];
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const int N = S.ns;
    const Real* __restrict__ fb = A.fin + S.pop_offset;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
    const int x = tl.y + tx, y = tl.z + ty, z = tl.w + tz;
    const bool valid = x < nx && y < ny && z < nz;

    // ---- own site: pull f_i(r, t) = f*_i(r - c_i, t - 1) ----------------
    Real f[Q];
    Real drho = Real(0);
    if (valid) {
        const Nbr nb(x, y, z, nx, ny, nz, L::D == 3);
        pull_site<L, Real>(fb, N, nb, f);
        sfor<0, Q>([&](auto I) { drho += f[decltype(I)::value]; });
    }
    const int cidx = (tz + HZ) * SX * SY + (ty + H) * SX + (tx + H);

    // ---- density deviation on tile + halo --------------------------------
    // Slots of valid tile sites are written by their owner; the loop fills the
    // halo and the tile slots that lie beyond the system (needed when a tile
    // overhangs a short side: they hold the periodic images).
    if (valid) srho[cidx] = drho;
    for (int idx = tid; idx < SX * SY * SZ; idx += NT) {
        const int px = idx % SX, py = (idx / SX) % SY, pz = idx / (SX * SY);
        const int gx = tl.y + px - H, gy = tl.z + py - H, gz = tl.w + pz - HZ;
        const bool interior = px >= H && px < H + TX && py >= H && py < H + TY && pz >= HZ && pz < HZ + TZ;
        if (interior && gx < nx && gy < ny && gz < nz) continue;
        Real v = Real(0);
        if (gx < nx + H && gy < ny + H && gz < nz + HZ) {
            const bool sm = S.small != 0;
            const Nbr nb(sm ? wrapm(gx, nx) : wrap2(gx, nx), sm ? wrapm(gy, ny) : wrap2(gy, ny),
                         L::D == 3 ? (sm ? wrapm(gz, nz) : wrap2(gz, nz)) : 0, nx, ny, nz, L::D == 3);
            Real g[Q];
            pull_site<L, Real>(fb, N, nb, g);
            sfor<0, Q>([&](auto I) { v += g[decltype(I)::value]; });
        }
        srho[idx] = v;
    }
    __syncthreads();

    int lidx = 0;
    if constexpr (CP == GUO) {
        // Laplacian of rho on tile + 1
        for (int idx = tid; idx < LX * LY * LZ; idx += NT) {
            const int px = idx % LX, py = (idx / LX) % LY, pz = idx / (LX * LY);
            const int sidx = (pz + (L::D == 3 ? H - 1 : 0)) * SX * SY + (py + H - 1) * SX + (px + H - 1);
            const Real r0 = srho[sidx];
            Real lap = Real(0);
            sfor<1, Q>([&](auto I) {
                constexpr int i = I;
                constexpr int off = L::c(i, 0) + SX * (L::c(i, 1) + SY * L::c(i, 2));
                lap += Real(6.0 * L::w(i)) * (srho[sidx + off] - r0);
            });
            slap[idx] = lap;
        }
        __syncthreads();
        lidx = (tz + (L::D == 3 ? 1 : 0)) * LX * LY + (ty + 1) * LX + (tx + 1);
    }
    if (!valid) return;

    const int site = site_index(x, y, z, nx, ny);
    const int64_t step = *A.step_ptr + A.k;
    const TileView<Real, SX, SY> rv{srho, cidx};
    const TileView<Real, LX, LY> lv{slap, lidx};
    if constexpr (CP == MODEQ && L::D == 2) {
        Real d0, jx, jy;
        moments_d2q9<Real>(f, d0, jx, jy);
        collide_d2q9_modeq<MODE, Real>(f, drho, jx, jy, rv, A.phys[tl.x], noise_key(S, step), uint32_t(site),
                                       A.status);
    } else if constexpr (CP == GUO && BGK_ONLY)
        collide_guo_bgk<L, Real, TAU1>(f, drho, lv, S, A.phys[tl.x], uint32_t(site), step, A.status);
    else
        collide_site<L, CP, Real, BGK_ONLY, TileView<Real, SX, SY>, TileView<Real, LX, LY>, TAU1>(
            f, drho, rv, lv, S, A.phys[tl.x], uint32_t(site), step, A.status);

    Real* __restrict__ fo = A.fout + S.pop_offset;
    sfor<0, Q>([&](auto I) {
        constexpr int i = I;
        fo[i * N + site] = f[i];
    });
}

// Density deviation on the 3 x 3 neighbourhood of a site, held in registers:
// at<cx, cy, 0>() is the value at r + c.
template <class Real>
struct Nbr9 {
    Real v[3][3];   // [1 + c_y][1 + c_x]
    template <int CX, int CY, int CZ>
    __device__ __forceinline__ Real at() const { return v[1 + CY][1 + CX]; }
};

// Row-marching strips for the D2Q9 modified-equilibrium step (Eq. 65 needs
// the density on the 3 x 3 neighbourhood only).  Each warp owns 32
// consecutive sites of a row and walks YC rows; a tile (system, x0, y0) is SW
// sites wide (32, or 64 for the tiles of the two-site kernel, whose one-site
// form gives each tile two warps).  Per footprint row yy a lane pulls its
// site's 9 populations, forms rho, and the neighbours' rho comes by warp
// shuffles; lanes 0 and 31 also pull the halo sites x0 - 1 and x0 + 32.
// Three density rows live in registers as (x - 1, x, x + 1) triples, and the
// site of row yy - 1 collides from its populations pulled one iteration
// earlier (with every mode at tau = 1, from its density and momentum only;
// the collision is collide_d2q9_modeq for every relaxation setting).
// No shared memory and no CTA barrier: every footprint value is formed once
// per chunk (halo 2/32 in x, 2/YC in y).  Lanes past the system's last column
// form the periodic image of their column for their neighbours and do not
// collide.  (Colliding two rows behind, to overlap the next row's loads,
// measured slower: 8 more registers per thread, fewer warps in flight.)
template <class L, int CP, class Real, int YC, int WPC, int MINB, int MODE, int SW = 32>
__global__ void __launch_bounds__(32 * WPC, MINB) step_kernel_strip(const StepArgs<Real> A, int n_tiles) {
    static_assert(L::D == 2 && CP == MODEQ, "row strips: D2Q9 with the modified equilibrium");
    constexpr bool BGK_ONLY = MODE >= 1;
    constexpr bool TAU1 = MODE == 2;
    constexpr int Q = L::Q;
    constexpr int WPT = SW / 32;                     // warps per tile
    const int lane = threadIdx.x & 31;
    const int wg = blockIdx.x * WPC + int(threadIdx.x >> 5);
    if (wg >= n_tiles * WPT) return;                 // the whole warp leaves together
    const int4 tl = A.tiles[wg / WPT];
    // register copies of the per-system records: read once, not again after every row's stores
    const SysDev S = A.sys[tl.x];
    const SysPhys<Real> P = A.phys[tl.x];
    const int nx = S.nx, ny = S.ny, N = S.ns;
    const bool sm = S.small != 0;
    const Real* __restrict__ fb = A.fin + S.pop_offset;
    Real* __restrict__ fo = A.fout + S.pop_offset;
    const int x0 = tl.y + 32 * (wg % WPT);
    const int x = x0 + lane;
    const bool own = x < nx;
    const bool extra = lane == 0 || lane == 31;
    // pulled columns x - c_x for c_x = -1, 0, 1 (index 1 + c_x), of the lane's site and of its halo site
    const int xs = wrapm(x, nx);
    const int xh = wrapm(lane == 0 ? x0 - 1 : x0 + 32, nx);
    const int xo[3] = {wrap1(xs + 1, nx), xs, wrap1(xs - 1, nx)};
    const int ho[3] = {wrap1(xh + 1, nx), xh, wrap1(xh - 1, nx)};
    const int64_t step = *A.step_ptr + A.k;
    const int y0 = tl.z, y1 = min(y0 + YC, ny);

    Real fp[TAU1 ? 1 : Q];                           // pulled populations of row yy - 1
    Real pr = Real(0), pjx = Real(0), pjy = Real(0); // tau = 1: (drho, j) of row yy - 1
    Real Rm[3] = {Real(0), Real(0), Real(0)}, R0[3] = {Real(0), Real(0), Real(0)},
         Rp[3] = {Real(0), Real(0), Real(0)};        // rho rows yy - 2, yy - 1, yy
    if constexpr (!TAU1) sfor<0, Q>([&](auto I) { fp[decltype(I)::value] = Real(0); });
    for (int yy = y0 - 1; yy <= y1; ++yy) {
        // pulled rows yy - c_y for c_y = -1, 0, 1 (index 1 + c_y)
        const int ro[3] = {(sm ? wrapm(yy + 1, ny) : wrap2(yy + 1, ny)) * nx,
                           (sm ? wrapm(yy, ny) : wrap2(yy, ny)) * nx,
                           (sm ? wrapm(yy - 1, ny) : wrap2(yy - 1, ny)) * nx};
        Real fc[Q];
        sfor<0, Q>([&](auto I) {
            constexpr int i = I;
            fc[i] = fb[i * N + ro[1 + L::c(i, 1)] + xo[1 + L::c(i, 0)]];
        });
        Real re = Real(0);
        if (extra) {
            Real g[Q];
            sfor<0, Q>([&](auto I) {
                constexpr int i = I;
                g[i] = fb[i * N + ro[1 + L::c(i, 1)] + ho[1 + L::c(i, 0)]];
            });
            sfor<0, Q>([&](auto I) { re = vadd(re, g[decltype(I)::value]); });
        }
        Real rc, jx, jy;
        moments_d2q9<Real>(fc, rc, jx, jy);
        Real rl = __shfl_up_sync(0xffffffffu, rc, 1);
        Real rr = __shfl_down_sync(0xffffffffu, rc, 1);
        if (lane == 0) rl = re;
        if (lane == 31) rr = re;
        sfor<0, 3>([&](auto K) {
            constexpr int k = K;
            Rm[k] = R0[k];
            R0[k] = Rp[k];
        });
        Rp[0] = rl;
        Rp[1] = rc;
        Rp[2] = rr;
        if (yy > y0 && own) {
            const int y = yy - 1;
            const Nbr9<Real> nb{{{Rm[0], Rm[1], Rm[2]}, {R0[0], R0[1], R0[2]}, {Rp[0], Rp[1], Rp[2]}}};
            const int site = y * nx + x;
            Real fr[Q];
            if constexpr (TAU1) {
                collide_d2q9_modeq<2, Real>(fr, pr, pjx, pjy, nb, P, noise_key(S, step), uint32_t(site), A.status);
            } else {
                sfor<0, Q>([&](auto I) { fr[decltype(I)::value] = fp[decltype(I)::value]; });
                collide_d2q9_modeq<MODE, Real>(fr, R0[1], pjx, pjy, nb, P, noise_key(S, step), uint32_t(site),
                                               A.status);
            }
            sfor<0, Q>([&](auto I) {
                constexpr int i = I;
                fo[i * N + site] = fr[i];
            });
        }
        pr = rc;
        pjx = jx;
        pjy = jy;
        if constexpr (!TAU1) sfor<0, Q>([&](auto I) { fp[decltype(I)::value] = fc[decltype(I)::value]; });
    }
}

}  // namespace lbf

namespace lbf {

// z-marching variant for 3-D lattices.  A CTA owns a TX x TY column of sites
// and walks a chunk of ZC planes.  (Keeping each thread's own populations in
// shared memory instead of re-reading them was measured slower: the carve-out
// takes the L1 space that serves the overlapping footprint pulls.)  The density deviation of each plane is
// computed once on the column's footprint (halo H in x and y) into a ring of
// 2H+1 planes in shared memory, the Laplacian (Guo force) into a ring of 3
// planes, so every footprint value is formed once per chunk instead of once
// per tile, and the collision of plane z follows two planes behind.
template <class L, int CP, class Real, int TX, int TY, int ZC>
struct ZLayout {
    static constexpr size_t bytes = 0;     // static shared memory only
};

template <class L, int CP, class Real, int TX, int TY, int ZC, int MINB, int MODE>
__global__ void __launch_bounds__(TX* TY, MINB)
    step_kernel_z(const StepArgs<Real> A) {
    static_assert(L::D == 3, "z-marching is for 3-D lattices");
    static_assert(CP == GUO, "the z-marching kernel implements the Guo-forced coupling");
    constexpr bool BGK_ONLY = MODE >= 1;
    constexpr bool TAU1 = MODE == 2;
    constexpr int Q = L::Q;
    constexpr int H = HaloOf<L, CP>::H;
    constexpr int SX = TX + 2 * H, SY = TY + 2 * H, SP = SX * SY;     // rho footprint plane
    // One barrier per plane: the collision trails the density by H + 1 planes,
    // so the Laplacian planes it reads were written before the iteration's
    // barrier.  Ring sizes: rho planes zz-2..zz are read by the Laplacian while a
    // thread past the barrier may already write plane zz+1 (4 slots); Laplacian
    // planes zz-4..zz-2 are read by the collision while plane zz-1 is written (4).
    // PULLFREE (every mode fully relaxed): the collision needs only the conserved
    // moments of the site, which the footprint pass already sums; they are kept
    // in a ring (sj, with the density in srho) instead of pulling the site again.
    // The collided plane zz - 3 then stays live while plane zz + 1 is written: 5 slots.
    constexpr bool PULLFREE = MODE == 2;
    constexpr int NR = PULLFREE ? 5 : 4;                              // rho ring planes
    constexpr int LX = TX + 2, LY = TY + 2, LP = LX * LY;             // Laplacian plane
    constexpr int NL = 4;
    constexpr int NT = TX * TY;
    __shared__ Real srho[NR * SP];
    __shared__ Real slap[NL * LP];
    __shared__ Real sj[PULLFREE ? NR * 3 * NT : 1];

    const int4 tl = A.tiles[blockIdx.x];
    const SysDev& S = A.sys[tl.x];
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const int N = S.ns;
    const Real* __restrict__ fb = A.fin + S.pop_offset;
    Real* __restrict__ fo = A.fout + S.pop_offset;
    const int z0 = tl.w, z1 = min(z0 + ZC, nz);
    const int64_t step = *A.step_ptr + A.k;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x = tl.y + tx, y = tl.z + ty;
    const bool valid_xy = x < nx && y < ny;

    // footprint of plane zz: the density at the tile + halo H sites, from the
    // populations pulled to them; thread tid handles footprint sites tid + s NT
    const bool sm = S.small != 0;
    auto foot_site = [&](int idx, int zz, int& gxw, int& gyw, int& wz) {
        const int px = idx % SX, py = idx / SX;
        const int gx = tl.y + px - H, gy = tl.z + py - H;
        if (!(gx < nx + H && gy < ny + H)) return false;
        gxw = sm ? wrapm(gx, nx) : wrap2(gx, nx);
        gyw = sm ? wrapm(gy, ny) : wrap2(gy, ny);
        wz = sm ? wrapm(zz, nz) : wrap2(zz, nz);
        return true;
    };

    // rho planes z0 - H .. z1 + H - 1, Laplacian planes z0 - 1 .. z1, collisions z0 .. z1 - 1
    for (int zz = z0 - H; zz <= z1 + H; ++zz) {
        const int zc = zz - H - 1;
        const bool collide = zc >= z0 && valid_xy;
        if (zz < z1 + H) {
            const int slot = (zz - z0 + 2 * NR) % NR;
            for (int idx = tid; idx < SP; idx += NT) {
                int gxw, gyw, wz;
                Real v = Real(0);
                if (foot_site(idx, zz, gxw, gyw, wz)) {
                    const Nbr nb(gxw, gyw, wz, nx, ny, nz, true);
                    Real g[Q];
                    pull_site<L, Real>(fb, N, nb, g);
                    sfor<0, Q>([&](auto I) { v += g[decltype(I)::value]; });
                    if constexpr (PULLFREE) {
                        const int px = idx % SX - H, py = idx / SX - H;
                        if (px >= 0 && px < TX && py >= 0 && py < TY) {
                            Real jm[3];
                            momentum_of<L, Real>(g, jm);
                            sfor<0, 3>([&](auto A) {
                                sj[(slot * 3 + int(A)) * NT + py * TX + px] = jm[decltype(A)::value];
                            });
                        }
                    }
                }
                srho[slot * SP + idx] = v;
            }
        }
        __syncthreads();
        // Laplacian of plane zl = zz - 1 on the column + 1 (needs rho planes zl-1 .. zl+1)
        const int zl = zz - 1;
        if (zl >= z0 - 1 && zl <= z1) {
            const int lslot = (zl - z0 + 2 * NL) % NL;
            const int r0 = (zl - z0 + 2 * NR) % NR;
            const int rm = (zl - 1 - z0 + 2 * NR) % NR;
            const int rp = (zl + 1 - z0 + 2 * NR) % NR;
            for (int idx = tid; idx < LP; idx += NT) {
                const int px = idx % LX, py = idx / LX;
                const int c = (py + H - 1) * SX + (px + H - 1);
                const RingView<Real, SX> rv{srho, rm * SP, r0 * SP, rp * SP, c};
                slap[lslot * LP + idx] = lap_d3q19<Real>(rv);
            }
        }
        // collision of plane zc = zz - H - 1
        if (collide) {
            Real f[Q];
            Real drho = Real(0);
            Real jc[3];
            const int cslot = (zc - z0 + 2 * NR) % NR;
            if constexpr (PULLFREE) {
                drho = srho[cslot * SP + (ty + H) * SX + (tx + H)];
                sfor<0, 3>([&](auto A) { jc[decltype(A)::value] = sj[(cslot * 3 + int(A)) * NT + tid]; });
            } else {
                pull_site<L, Real>(fb, N, Nbr(x, y, zc, nx, ny, nz, true), f);
                sfor<0, Q>([&](auto I) { drho += f[decltype(I)::value]; });
            }
            const int site = site_index(x, y, zc, nx, ny);
            // the Guo collision reads only the Laplacian planes zc-1..zc+1 around the
            // site (a 3-plane view); the density view is unused by this coupling
            const RingView<Real, SX> rv{srho, 0, 0, 0, (ty + H) * SX + (tx + H)};
            const RingView<Real, LX> lv{slap, ((zc - 1 - z0 + 2 * NL) % NL) * LP, ((zc - z0 + 2 * NL) % NL) * LP,
                                        ((zc + 1 - z0 + 2 * NL) % NL) * LP, (ty + 1) * LX + (tx + 1)};
            if constexpr (PULLFREE)
                collide_d3q19_tau1<Real>(f, drho, jc[0], jc[1], jc[2], lv, A.phys[tl.x], noise_key(S, step),
                                         uint32_t(site), A.status);
            else if constexpr (BGK_ONLY)
                collide_guo_bgk<L, Real, TAU1>(f, drho, lv, S, A.phys[tl.x], uint32_t(site), step, A.status);
            else
                collide_site<L, CP, Real, BGK_ONLY>(f, drho, rv, lv, S, A.phys[tl.x], uint32_t(site), step, A.status);
            sfor<0, Q>([&](auto I) {
                constexpr int i = I;
                fo[i * N + site] = f[i];
            });
        }
        // no second barrier: the next iteration writes rho plane zz + 1 (a slot
        // none of this iteration's reads use) before its barrier, and Laplacian
        // plane zz only after it
    }
}

// Warp-specialised z-marching step for the fully relaxed Guo path (every mode
// at tau = 1, FP32): PW producer warps stage each plane -- the footprint pulls,
// the density on the tile + halo, the momentum of the tile sites and the
// Laplacian on the tile + 1 -- into shared-memory rings; TX x TY consumer
// threads collide one site each from those rings and store.  The consumers
// read no global memory, so their arithmetic overlaps the producers' loads.
//
// Rings (R planes, data slot of plane z: (z - z0 + H) % R): density and
// momentum of footprint planes z0 - H .. z1 + H - 1, Laplacian planes
// z0 - 1 .. z1.  mbarriers: full[(zl - z0 + 1) % R] completes when all
// producers have written Laplacian plane zl (and so every plane the collision
// of zl - 1 reads); empty[(zc - z0) % R] completes when all consumers have
// collided plane zc.  Before writing footprint plane zz (slot of zz - R) the
// producers wait for the collision of plane zz - R; that also frees the
// Laplacian slot written next.  A phase of one slot cannot complete twice
// before its waiter looks (each side runs at most R - 2 planes ahead), so the
// parity of the use count identifies the phase.  Every wait is bounded
// (mbar_wait): a timeout flags the CTA and the status, and all threads keep
// the same control flow, so the producers' named barrier is always reached.
//
// Staging (STG):
//  0  each producer thread pulls the populations of its footprint sites with
//     plain loads (any system shape);
//  1  bulk copies (cp.async.bulk): for footprint plane zz and direction i the
//     producers copy the BH rows of population i on plane zz - c_iz that the
//     footprint pulls from, each row the BW = TX + 8 floats from x0 - 4
//     (16-byte aligned; split where it crosses the periodic seam) into a
//     shared stage; two stages alternate, so the copies of plane zz + 2 run
//     while plane zz + 1 is summed.  A footprint site then reads its 19 pulled
//     values from the stage at fixed offsets.  Needs nx % 4 == 0, nx >= 8 and
//     every side >= 3 (the host checks; the stage is dynamic shared memory).
// Footprint slot -> footprint index (row-major over the (TX + 2H) x (TY + 2H)
// plane): slots 0 .. TX TY - 1 are the tile's own sites row by row, then the
// H rows above and below, then the H columns on each side, so a warp's slots
// are all tile sites or all halo sites.
template <int TX, int TY, int H>
__device__ __forceinline__ int foot_slot(int s) {
    constexpr int SX = TX + 2 * H;
    if (s < TX * TY) return (s / TX + H) * SX + (s % TX + H);
    int h = s - TX * TY;
    if (h < 2 * H * SX) {
        const int r = h / SX, c = h % SX;
        return (r < H ? r : TY + r) * SX + c;
    }
    h -= 2 * H * SX;
    const int r = h / (2 * H), c = h % (2 * H);
    return (H + r) * SX + (c < H ? c : TX + c);
}

template <class L, int TX, int TY, int ZC, int PW>
struct BulkStage {
    static constexpr int H = HaloOf<L, GUO>::H;
    static constexpr int BW = TX + 8;              // staged row: x0 - 4 .. x0 + TX + 3
    static constexpr int BH = TY + 2 * H;          // rows per direction (the footprint rows)
    static constexpr int BD = BH * BW;             // floats per direction
    static constexpr int BSTAGE = L::Q * BD;       // floats per stage
    static constexpr int NTASK = L::Q * BH;        // row copies per plane (before seam splits)
    static constexpr size_t bytes = 2 * size_t(BSTAGE) * sizeof(float);
};

template <class L, int TX, int TY, int ZC, int PW, int MINB, int STG>
__global__ void __launch_bounds__(TX* TY + 32 * PW, MINB) step_kernel_ws(const StepArgs<float> A) {
    using Real = float;
    static_assert(L::D == 3, "z-marching is for 3-D lattices");
    constexpr int Q = L::Q;
    constexpr int H = HaloOf<L, GUO>::H;
    constexpr int SX = TX + 2 * H, SY = TY + 2 * H, SP = SX * SY;     // rho footprint plane
    constexpr int LX = TX + 2, LY = TY + 2, LP = LX * LY;             // Laplacian plane
    constexpr int NC = TX * TY;                                       // consumer threads
    constexpr int NP = 32 * PW;                                       // producer threads
    constexpr int R = 6;                                              // ring planes
    static_assert(R >= 4, "ring too short for the plane lags");
    __shared__ Real srho[R * SP];
    __shared__ Real slap[R * LP];
    __shared__ Real sj[R * 3 * NC];
    __shared__ uint64_t full[R], empty[R];
    __shared__ int abort_flag;
    using BS = BulkStage<L, TX, TY, ZC, PW>;
    static_assert(STG == 0 || TX % 4 == 0, "staged rows start 16-byte aligned");
    extern __shared__ __align__(128) float stage_smem[];
    __shared__ uint64_t tfull[2];                  // bulk-copy stages
    __shared__ int2 rowtab[STG ? BS::NTASK : 1];   // per row copy: (i N + y nx, c_iz + 1)
    __shared__ int4 pieces[4];                     // (source x, stage column, length) of the row

    const int4 tl = A.tiles[blockIdx.x];
    const SysDev S = A.sys[tl.x];          // register copy: not re-read after the stores
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const int N = S.ns;
    const int z0 = tl.w, z1 = min(z0 + ZC, nz);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int r = 0; r < R; ++r) {
            mbar_init(&full[r], NP);
            mbar_init(&empty[r], NC);
        }
        if constexpr (STG == 1) {
            mbar_init(&tfull[0], 1);
            mbar_init(&tfull[1], 1);
            fence_proxy_async_smem();              // the inits are seen by the copy engine
        }
        abort_flag = 0;
    }
    __syncthreads();
    auto dslot = [&](int z) { return (z - z0 + H) % R; };

    if (tid >= NC) {
        // ---------------- producers ----------------
        const Real* __restrict__ fb = A.fin + S.pop_offset;
        const int ptid = tid - NC;
        const bool sm = S.small != 0;
        // row copies of footprint plane zp into stage st: direction i reads plane
        // zp - c_iz (rowtab: c_iz + 1 selects the plane offset)
        auto issue_rows = [&](int zp, int st) {
            if constexpr (STG == 1) {
                const int pl = nx * ny;
                const int zo[3] = {wrap2(zp + 1, nz) * pl, wrap2(zp, nz) * pl, wrap2(zp - 1, nz) * pl};
                Real* dst0 = stage_smem + st * BS::BSTAGE;
                for (int t = ptid; t < BS::NTASK; t += NP) {
                    const int2 rt = rowtab[t];
                    const Real* src = fb + rt.x + (rt.y == 0 ? zo[0] : (rt.y == 1 ? zo[1] : zo[2]));
                    Real* dst = dst0 + t * BS::BW;
                    sfor<0, 4>([&](auto P) {
                        const int4 pc = pieces[int(P)];
                        if (pc.z > 0)
                            bulk_copy_g2s(dst + pc.y, src + pc.x, unsigned(pc.z * sizeof(Real)), &tfull[st]);
                    });
                }
            }
        };
        // bulk staging: row-copy table and seam pieces, then the first two planes
        if constexpr (STG == 1) {
            if (ptid < BS::BH) {
                const int r = ptid;
                sfor<0, Q>([&](auto I) {
                    constexpr int i = I;
                    const int gy = wrapm(tl.z - H - L::c(i, 1) + r, ny);
                    rowtab[i * BS::BH + r] = make_int2(i * N + gy * nx, L::c(i, 2) + 1);
                });
            }
            if (ptid == 0) {
                const int xs = tl.y - 4;
                int pos = xs;
                for (int p = 0; p < 4; ++p) {
                    const int rem = xs + BS::BW - pos;
                    if (rem > 0) {
                        const int w = wrapm(pos, nx);
                        const int len = min(rem, nx - w);
                        pieces[p] = make_int4(w, pos - xs, len, 0);
                        pos += len;
                    } else {
                        pieces[p] = make_int4(0, 0, 0, 0);
                    }
                }
                mbar_arrive_expect_tx(&tfull[0], unsigned(BS::BSTAGE * sizeof(Real)));
                mbar_arrive_expect_tx(&tfull[1], unsigned(BS::BSTAGE * sizeof(Real)));
            }
            named_barrier(1, NP);
            issue_rows(z0 - H, 0);
            issue_rows(z0 - H + 1, 1);
        }
        int it = 0;
        for (int zz = z0 - H; zz < z1 + H; ++zz, ++it) {
            const int zw = zz - R;                       // plane whose slots this iteration reuses
            if (zw >= z0) mbar_wait(&empty[(zw - z0) % R], unsigned(((zw - z0) / R) & 1), &abort_flag, A.status);
            const int slot = dslot(zz);
            if constexpr (STG == 0) {
            const int wz = sm ? wrapm(zz, nz) : wrap2(zz, nz);
            // the footprint sites of this producer thread go in batches of FB: all
            // FB x Q loads of a batch are requested before any is summed
            constexpr int FS = (SP + NP - 1) / NP;
            constexpr int FB = FS < 2 ? FS : 2;
#pragma unroll 1
            for (int b0 = 0; b0 < FS; b0 += FB) {
            Real g[FB][Q];
            bool inb[FB];
            sfor<0, FB>([&](auto SI) {
                constexpr int si = SI;
                const int sl = ptid + (b0 + si) * NP;
                const int idx = sl < SP ? foot_slot<TX, TY, H>(sl) : SP;
                const int px = idx % SX, py = idx / SX;
                const int gx = tl.y + px - H, gy = tl.z + py - H;
                inb[si] = b0 + si < FS && sl < SP && gx < nx + H && gy < ny + H;
                if (inb[si]) {
                    const Nbr nb(sm ? wrapm(gx, nx) : wrap2(gx, nx), sm ? wrapm(gy, ny) : wrap2(gy, ny), wz, nx, ny,
                                 nz, true);
                    pull_site<L, Real>(fb, N, nb, g[si]);
                }
            });
            sfor<0, FB>([&](auto SI) {
                constexpr int si = SI;
                const int sl = ptid + (b0 + si) * NP;
                if (b0 + si < FS && sl < SP) {
                    const int idx = foot_slot<TX, TY, H>(sl);
                    Real v = Real(0);
                    if (inb[si]) {
                        sfor<0, Q>([&](auto I) { v += g[si][decltype(I)::value]; });
                        if (sl < NC) {                   // slots 0 .. NC - 1 are the tile sites, row by row
                            Real jm[3];
                            momentum_of<L, Real>(g[si], jm);
                            sfor<0, 3>([&](auto C) {
                                sj[(slot * 3 + int(C)) * NC + sl] = jm[decltype(C)::value];
                            });
                        }
                    }
                    srho[slot * SP + idx] = v;
                }
            });
            }
            } else {
            // the copies of this plane were issued two planes ago (or in the prologue)
            const int st = it & 1;
            mbar_wait_copies(&tfull[st], unsigned((it >> 1) & 1), &abort_flag, A.status);
            const Real* stg = stage_smem + st * BS::BSTAGE;
            constexpr int FS = (SP + NP - 1) / NP;
            sfor<0, FS>([&](auto SI) {
                constexpr int si = SI;
                const int idx = ptid + si * NP;
                if (idx < SP) {
                    const int px = idx % SX, py = idx / SX;
                    Real v = Real(0);
                    if (tl.y + px - H < nx + H && tl.z + py - H < ny + H) {
                        // pulled value of direction i: row py, column px + 2 - c_ix of its block
                        const Real* sb = stg + py * BS::BW + px + 2;
                        Real g[Q];
                        sfor<0, Q>([&](auto I) {
                            constexpr int i = I;
                            g[i] = sb[i * BS::BD - L::c(i, 0)];
                        });
                        sfor<0, Q>([&](auto I) { v += g[decltype(I)::value]; });
                        const int ix = px - H, iy = py - H;
                        if (ix >= 0 && ix < TX && iy >= 0 && iy < TY) {
                            Real jm[3];
                            momentum_of<L, Real>(g, jm);
                            sfor<0, 3>([&](auto C) {
                                sj[(slot * 3 + int(C)) * NC + iy * TX + ix] = jm[decltype(C)::value];
                            });
                        }
                    }
                    srho[slot * SP + idx] = v;
                }
            });
            if (zz + 2 < z1 + H && ptid == 0) mbar_arrive_expect_tx(&tfull[st], unsigned(BS::BSTAGE * sizeof(Real)));
            }
            named_barrier(1, NP);                        // density plane zz complete (producers)
            if constexpr (STG == 1) {
                // every producer has read stage it & 1: refill it with plane zz + 2
                if (zz + 2 < z1 + H) {
                    fence_proxy_async_smem();
                    issue_rows(zz + 2, it & 1);
                }
            }
            const int zl = zz - 1;                       // Laplacian plane (needs density zl-1 .. zl+1)
            if (zl >= z0 - 1) {
                const int r0 = dslot(zl) * SP, rm = dslot(zl - 1) * SP, rp = dslot(zl + 1) * SP;
                const int lslot = dslot(zl);
                for (int idx = ptid; idx < LP; idx += NP) {
                    const int px = idx % LX, py = idx / LX;
                    const int c = (py + H - 1) * SX + (px + H - 1);
                    const RingView<Real, SX> rv{srho, rm, r0, rp, c};
                    slap[lslot * LP + idx] = lap_d3q19<Real>(rv);
                }
                mbar_arrive(&full[(zl - z0 + 1) % R]);
            }
        }
    } else {
        // ---------------- consumers ----------------
        Real* __restrict__ fo = A.fout + S.pop_offset;
        const int64_t step = *A.step_ptr + A.k;
        const SysPhys<Real> P = A.phys[tl.x];
        const int tx = tid % TX, ty = tid / TX;
        const int x = tl.y + tx, y = tl.z + ty;
        const bool valid_xy = x < nx && y < ny;
        for (int zc = z0; zc < z1; ++zc) {
            const int zl = zc + 1;                       // the last Laplacian plane the collision reads
            const bool ok = mbar_wait(&full[(zl - z0 + 1) % R], unsigned(((zl - z0 + 1) / R) & 1), &abort_flag,
                                      A.status);
            if (valid_xy && ok) {
                const int cs = dslot(zc);
                const Real drho = srho[cs * SP + (ty + H) * SX + (tx + H)];
                Real jc[3];
                sfor<0, 3>([&](auto C) { jc[decltype(C)::value] = sj[(cs * 3 + int(C)) * NC + tid]; });
                const RingView<Real, LX> lv{slap, dslot(zc - 1) * LP, cs * LP, dslot(zc + 1) * LP,
                                            (ty + 1) * LX + (tx + 1)};
                const int site = site_index(x, y, zc, nx, ny);
                Real f[Q];
                collide_d3q19_tau1<Real>(f, drho, jc[0], jc[1], jc[2], lv, P, noise_key(S, step), uint32_t(site),
                                         A.status);
                sfor<0, Q>([&](auto I) {
                    constexpr int i = I;
                    fo[i * N + site] = f[i];
                });
            }
            mbar_arrive(&empty[(zc - z0) % R]);
        }
    }
}

}  // namespace lbf

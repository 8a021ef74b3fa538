// Fused fluctuating LB time step (Eq. 61): pull-stream, moments (Eq. 62),
// density gradients from a shared-memory halo, equilibrium (Eq. 65 or the
// Landau-pressure form with a Guo body force), moment-space relaxation with
// per-mode rates (Eq. 66), local Cholesky-factored noise (Eq. 68), aligned store.
//
// Storage: per system, SoA populations [q][z][y][x] holding deviations
// delta f_i = f_i - f^eq_i(rho_c, u = 0), i.e. f_0 - rho_c on the rest velocity
// and f_i elsewhere.  The buffer read by step t holds the post-collision
// populations of step t-1 at their origin sites, so the pre-collision value
// f_i(r, t) is pulled from r - c_i and every store is aligned.
#pragma once

#include "lb_device.cuh"

namespace lbf {

template <class Real>
struct StepArgs {
    const SysDev* sys;
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

// Collision of one site given its pulled deviations f[], the density halo and
// (Guo) the Laplacian halo.  Returns post-collision deviations in f[].
template <class L, int CP, class Real, int SX, int SY, int LX, int LY>
__device__ __forceinline__ void collide_site(Real (&f)[L::Q], const Real drho, const Real* __restrict__ srho,
                                             const int cidx, const Real* __restrict__ slap, const int lidx,
                                             const SysDev& S, const uint32_t site, const int64_t step,
                                             int* status) {
    constexpr int Q = L::Q;
    const Real rho = Real(S.rho_c) + drho;
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
    const Real irc = Real(S.inv_rho_c);
    const Real phi = drho * irc;
    const Real A_ = Real(S.a), B_ = Real(S.b), kap = Real(S.kappa);
    const Real df0 = phi * (A_ + B_ * phi * phi);
    const Real f0 = phi * phi * (Real(0.5) * A_ + Real(0.25) * B_ * phi * phi);
    const Real p0 = rho * irc * df0 - f0;
    const Real cs2 = rho * irc * irc * (A_ + Real(3) * B_ * phi * phi);

    Real feq[Q];
    Real fsrc[Q];   // Guo population force
    Real F[3] = {Real(0), Real(0), Real(0)};
    if constexpr (CP == MODEQ) {
        // d_a rho = 3 sum_i t_i c_ia rho(r+c_i);  lap rho = 6 sum_i t_i (rho(r+c_i) - rho(r))
        Real g[2] = {Real(0), Real(0)};
        Real lap = Real(0);
        sfor<1, Q>([&](auto I) {
            constexpr int i = I;
            constexpr int off = L::c(i, 0) + SX * (L::c(i, 1) + SY * L::c(i, 2));
            const Real rn = srho[cidx + off];
            if constexpr (L::c(i, 0) != 0) g[0] += Real(3.0 * L::w(i) * L::c(i, 0)) * rn;
            if constexpr (L::c(i, 1) != 0) g[1] += Real(3.0 * L::w(i) * L::c(i, 1)) * rn;
            lap += Real(6.0 * L::w(i)) * (rn - drho);
        });
        const Real ir = Real(1) / rho;
        const Real ux = j[0] * ir, uy = j[1] * ir;
        const Real nu = Real(S.nu);
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
            feq[i] = v;
            s += v;
        });
        feq[0] = drho - s;   // deviation form of f_0 = rho - sum_{i>=1} f_i
    } else {
        // Guo body force F = kappa rho grad(lap rho)
        Real gl[3] = {Real(0), Real(0), Real(0)};
        sfor<1, Q>([&](auto I) {
            constexpr int i = I;
            constexpr int off = L::c(i, 0) + LX * (L::c(i, 1) + LY * L::c(i, 2));
            const Real ln = slap[lidx + off];
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
            feq[i] = v;
            fsrc[i] = Real(wi) * (Real(3) * (cF - uF) + Real(9) * cu * cF);
            s += v;
        });
        feq[0] = drho - s;
        fsrc[0] = Real(-3.0 * L::w(0)) * uF;
    }

    // moments of f (deviation), relaxation of the non-conserved ones
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
        const Real lam = Real(S.lam[a]);
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
    });
    if constexpr (CP == GUO) {
        sfor<0, L::D>([&](auto A) {
            constexpr int a = A;
            m[1 + a] += F[a];   // (T F)_a = F_a on the momentum rows
        });
    }

    // noise (Eq. 68): xi = sqrt(3 rho kT) L n on the non-conserved modes
    const Real kT = Real(S.kT);
    if (kT > Real(0)) {
        constexpr int K = Q - L::NC;
        constexpr int NDRAW = (K + 3) / 4;
        Real nrm[4 * NDRAW];
        sfor<0, NDRAW>([&](auto D) {
            constexpr int d = D;
            const uint4 w = site_draw(S, site, step, uint32_t(d));
            box_muller(w.x, w.y, nrm[4 * d + 0], nrm[4 * d + 1]);
            box_muller(w.z, w.w, nrm[4 * d + 2], nrm[4 * d + 3]);
        });
        const Real sc = sqrt(Real(3) * (rho > Real(0) ? rho : Real(0)) * kT);
        // the coupled pair (P, R): M = [N + (1 - 3 c_s^2) v v^T] g, v_a = T_a(c = 0)
        constexpr int P = L::PP, R = L::PR;
        constexpr double vP = double(L::T(P, 0)), vR = double(L::T(R, 0));
        constexpr double NP = norm2<L>(P), NR = norm2<L>(R);
        const Real om = Real(1) - Real(3) * cs2;
        const Real Mpp = (Real(NP) + om * Real(vP * vP)) * Real(S.g_diag[P]);
        const Real Mrr = (Real(NR) + om * Real(vR * vR)) * Real(S.g_diag[R]);
        const Real Mpr = om * Real(vP * vR) * Real(S.g_pair);
        const Real det = Mpp * Mrr - Mpr * Mpr;
        if (Mpp > Real(0) && det > Real(0)) {
            const Real l11 = sqrt(Mpp);
            const Real l21 = Mpr / l11;
            const Real l22 = sqrt(det / Mpp);
            const Real nP = nrm[P - L::NC], nR = nrm[R - L::NC];
            m[P] += sc * l11 * nP;
            m[R] += sc * (l21 * nP + l22 * nR);
        } else {
            atomicOr(status, ST_NOISE);
        }
        sfor<L::NC, Q>([&](auto A) {
            constexpr int a = A;
            if constexpr (a != P && a != R) {
                constexpr double Na = norm2<L>(a);
                m[a] += sc * sqrt(Real(Na) * Real(S.g_diag[a])) * nrm[a - L::NC];
            }
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

template <class L, int CP, class Real, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX* TY* TZ)
    step_kernel(const StepArgs<Real> A) {
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
    const int64_t N = S.n_sites;
    const Real* __restrict__ fb = A.fin + S.pop_offset;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
    const int x = tl.y + tx, y = tl.z + ty, z = tl.w + tz;
    const bool valid = x < nx && y < ny && z < nz;

    // ---- own site: pull f_i(r, t) = f*_i(r - c_i, t - 1) ----------------
    Real f[Q];
    Real drho = Real(0);
    if (valid) {
        sfor<0, Q>([&](auto I) {
            constexpr int i = I;
            const int sx = L::c(i, 0) == 0 ? x : wrap1(x - L::c(i, 0), nx);
            const int sy = L::c(i, 1) == 0 ? y : wrap1(y - L::c(i, 1), ny);
            const int sz = L::D == 3 ? (L::c(i, 2) == 0 ? z : wrap1(z - L::c(i, 2), nz)) : 0;
            f[i] = fb[int64_t(i) * N + site_index(sx, sy, sz, nx, ny)];
            drho += f[i];
        });
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
            // the wrapped base lies in [0, n), so its pulls need a single-branch wrap
            const int wx = wrapm(gx, nx), wy = wrapm(gy, ny), wz = L::D == 3 ? wrapm(gz, nz) : 0;
            sfor<0, Q>([&](auto I) {
                constexpr int i = I;
                const int sx = L::c(i, 0) == 0 ? wx : wrap1(wx - L::c(i, 0), nx);
                const int sy = L::c(i, 1) == 0 ? wy : wrap1(wy - L::c(i, 1), ny);
                const int sz = L::D == 3 ? (L::c(i, 2) == 0 ? wz : wrap1(wz - L::c(i, 2), nz)) : 0;
                v += fb[int64_t(i) * N + site_index(sx, sy, sz, nx, ny)];
            });
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
    collide_site<L, CP, Real, SX, SY, LX, LY>(f, drho, srho, cidx, slap, lidx, S, uint32_t(site), step, A.status);

    Real* __restrict__ fo = A.fout + S.pop_offset;
    sfor<0, Q>([&](auto I) {
        constexpr int i = I;
        fo[int64_t(i) * N + site] = f[i];
    });
}

}  // namespace lbf

// Fused step of the modified-equilibrium coupling on D3Q19.
//
// The paper prints its modified equilibrium (Eq. 65) for D2Q9 only.  On D3Q19
// the library uses the same structure with the isotropic weights 3 t_i,
//   f_i^eq = 3 t_i [p0 - kappa rho lap rho + rho c_i.u + (3/2)(c_ia c_ib - delta_ab/3) X_ab]
//          + kappa t_i [(9/2)(c_i.g)^2 - (9/2) c_i^2 |g|^2 + (9/2) |g|^2]      (i >= 1),
//   f_0^eq = rho - sum_{i>=1} f_i^eq,
// g = grad rho, X_ab = rho u_a u_b + nu (u_a g_b + u_b g_a + u.g delta_ab):
// the square-gradient terms are the rotation-invariant form of the printed
// D2Q9 weights with the one coefficient that the second-moment condition
// (Eq. 63) leaves free kept at its D2Q9 value, -9/2 for c_i^2 |g|^2.  Every
// moment condition of Eqs. 62-64 then holds in three dimensions.  The noise is
// the lattice-general form of Eq. 68 (exact at kappa = 0 for this
// equilibrium, whose linearisation is the Landau-pressure one).
//
// The coupling needs the density on the 3 x 3 x 3 neighbourhood only, so the
// z-marching kernel keeps one footprint ring of radius 1.  With every mode at
// tau = 1 the collision is the closed form collide_d3q19_modeq_tau1 (its
// moments on the D3Q19 basis); the other settings take collide_modeq3 below.
#pragma once

#include "step_kernels.cuh"

namespace lbf {

// Post-collision deviations of one site: drho and j = sum_i c_i f_i are its
// conserved moments, rv views the density deviation around it, f holds the
// pre-collision deviations on entry (not read when MODE == 2, every mode at
// tau = 1) and the post-collision ones on exit.  MODE 1: one rate; 0: per mode.
template <class L, class Real, int MODE, class RhoV>
__device__ __forceinline__ void collide_modeq3(Real (&f)[L::Q], const Real drho, const Real (&j)[3], const RhoV& rv,
                                               const SysDev& S, const SysPhys<Real>& P, const uint32_t site,
                                               const int64_t step, int* status) {
    static_assert(L::D == 3, "three-dimensional modified equilibrium");
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

    // d_a rho = 3 sum_i t_i c_ia rho(r + c_i); lap rho = 6 sum_i t_i (rho(r + c_i) - rho(r))
    Real g[3] = {Real(0), Real(0), Real(0)};
    Real lap = Real(0);
    sfor<1, Q>([&](auto I) {
        constexpr int i = I;
        const Real rn = rv.template at<L::c(i, 0), L::c(i, 1), L::c(i, 2)>();
        sfor<0, 3>([&](auto A) {
            constexpr int a = A;
            if constexpr (L::c(i, a) != 0) g[a] += Real(3.0 * L::w(i) * L::c(i, a)) * rn;
        });
        lap += Real(6.0 * L::w(i)) * (rn - drho);
    });
    const Real ir = fast_rcp(rho);
    const Real u[3] = {j[0] * ir, j[1] * ir, j[2] * ir};
    const Real nu = P.nu;
    const Real iso = p0 - kap * rho * lap;
    const Real udg = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
    const Real g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    Real X[3][3];
    sfor<0, 3>([&](auto Aa) {
        constexpr int a = Aa;
        sfor<a, 3>([&](auto Bb) {
            constexpr int b = Bb;
            Real v = rho * u[a] * u[b] + nu * (u[a] * g[b] + u[b] * g[a]);
            if constexpr (a == b) v += nu * udg;
            X[a][b] = v;
            X[b][a] = v;
        });
    });
    Real feq[Q];
    Real s = Real(0);
    sfor<1, Q>([&](auto I) {
        constexpr int i = I;
        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        constexpr double c2 = double(cx * cx + cy * cy + cz * cz);
        Real xcc = Real(0), cu = Real(0), cg = Real(0);
        sfor<0, 3>([&](auto Aa) {
            constexpr int a = Aa;
            constexpr int ca = L::c(i, a);
            xcc += Real(ca * ca - 1.0 / 3.0) * X[a][a];
            if constexpr (ca != 0) {
                cu += Real(ca) * u[a];
                cg += Real(ca) * g[a];
            }
            sfor<a + 1, 3>([&](auto Bb) {
                constexpr int b = Bb;
                if constexpr (ca * L::c(i, b) != 0) xcc += Real(2.0 * ca * L::c(i, b)) * X[a][b];
            });
        });
        constexpr double w3 = 3.0 * L::w(i);
        const Real v = Real(w3) * (iso + rho * cu + Real(1.5) * xcc) +
                       kap * Real(L::w(i)) * (Real(4.5) * cg * cg + Real(4.5 * (1.0 - c2)) * g2);
        feq[i] = v;
        s += v;
    });
    feq[0] = drho - s;                              // deviation form of f_0 = rho - sum_{i>=1} f_i

    Real xi[K];
    sfor<0, K>([&](auto Aa) { xi[decltype(Aa)::value] = Real(0); });
    if (P.kT > Real(0)) noise_modes<L, Real, MODE == 2>(S, P, site, step, rho, cs2, xi, status);

    if constexpr (MODE >= 1) {
        const Real lam = MODE == 2 ? Real(1) : P.lam_bgk;
        sfor<0, Q>([&](auto I) {
            constexpr int i = I;
            Real v = MODE == 2 ? feq[i] : f[i] - lam * (f[i] - feq[i]);
            sfor<L::NC, Q>([&](auto Aa) {
                constexpr int a = Aa;
                constexpr double coef = tinv<L>(i, a);
                if constexpr (coef != 0.0) v += Real(coef) * xi[a - L::NC];
            });
            f[i] = v;
        });
    } else {
        // per-mode rates: moments of f and f^eq, relaxation of the non-conserved ones
        Real m[Q];
        sfor<0, Q>([&](auto Aa) {
            constexpr int a = Aa;
            Real sm = Real(0), se = Real(0);
            sfor<0, Q>([&](auto I) {
                constexpr int i = I;
                constexpr int t = L::T(a, i);
                if constexpr (t != 0) {
                    sm += Real(t) * f[i];
                    se += Real(t) * feq[i];
                }
            });
            m[a] = a < L::NC ? sm : sm - P.lam[a] * (sm - se) + xi[a < L::NC ? 0 : a - L::NC];
        });
        sfor<0, Q>([&](auto I) {
            constexpr int i = I;
            Real v = Real(0);
            sfor<0, Q>([&](auto Aa) {
                constexpr int a = Aa;
                constexpr double coef = tinv<L>(i, a);
                if constexpr (coef != 0.0) v += Real(coef) * m[a];
            });
            f[i] = v;
        });
    }
}

// z-marching step for the modified equilibrium on D3Q19: a CTA owns a TX x TY
// column and walks a chunk of ZC planes; iteration zz forms the density of
// footprint plane zz (tile + 1 site, from the pulled populations; with every
// mode at tau = 1 also the momentum of the tile sites, so the collision needs
// no second pull) into a ring of 4 planes, and after one barrier collides plane
// zz - 1, whose density neighbourhood (planes zz - 2 .. zz) is complete.  The
// next iteration writes the slot of plane zz - 3, which no collision of
// iteration zz reads, and no thread starts it before every thread has passed
// the barrier of iteration zz.
template <class L, class Real, int TX, int TY, int ZC, int MINB, int MODE>
__global__ void __launch_bounds__(TX* TY, MINB) step_kernel_zm(const StepArgs<Real> A) {
    static_assert(L::D == 3, "z-marching is for 3-D lattices");
    constexpr int Q = L::Q;
    constexpr int SX = TX + 2, SY = TY + 2, SP = SX * SY, NT = TX * TY, NR = 4;
    constexpr bool PULLFREE = MODE == 2;
    __shared__ Real srho[NR * SP];
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
    const bool sm = S.small != 0;

    for (int zz = z0 - 1; zz <= z1; ++zz) {
        const int slot = (zz - z0 + 1) & (NR - 1);
        for (int idx = tid; idx < SP; idx += NT) {
            const int px = idx % SX, py = idx / SX;
            const int gx = tl.y + px - 1, gy = tl.z + py - 1;
            Real v = Real(0);
            if (gx < nx + 1 && gy < ny + 1) {
                const Nbr nb(sm ? wrapm(gx, nx) : wrap2(gx, nx), sm ? wrapm(gy, ny) : wrap2(gy, ny),
                             sm ? wrapm(zz, nz) : wrap2(zz, nz), nx, ny, nz, true);
                Real g[Q];
                pull_site<L, Real>(fb, N, nb, g);
                sfor<0, Q>([&](auto I) { v += g[decltype(I)::value]; });
                if constexpr (PULLFREE) {
                    if (px >= 1 && px <= TX && py >= 1 && py <= TY) {
                        Real jm[3];
                        momentum_of<L, Real>(g, jm);
                        sfor<0, 3>([&](auto C) {
                            sj[(slot * 3 + int(C)) * NT + (py - 1) * TX + (px - 1)] = jm[decltype(C)::value];
                        });
                    }
                }
            }
            srho[slot * SP + idx] = v;
        }
        __syncthreads();
        const int zc = zz - 1;
        if (zc >= z0 && valid_xy) {
            const int cs = (zc - z0 + 1) & (NR - 1), rm = (zc - z0) & (NR - 1), rp = (zc - z0 + 2) & (NR - 1);
            const int c = (ty + 1) * SX + (tx + 1);
            const RingView<Real, SX> rv{srho, rm * SP, cs * SP, rp * SP, c};
            const Real drho = srho[cs * SP + c];
            Real f[Q];
            Real jc[3];
            if constexpr (PULLFREE) {
                sfor<0, 3>([&](auto C) { jc[decltype(C)::value] = sj[(cs * 3 + int(C)) * NT + tid]; });
            } else {
                pull_site<L, Real>(fb, N, Nbr(x, y, zc, nx, ny, nz, true), f);
                momentum_of<L, Real>(f, jc);
            }
            const int site = site_index(x, y, zc, nx, ny);
            if constexpr (MODE == 2)
                collide_d3q19_modeq_tau1<Real>(f, drho, jc[0], jc[1], jc[2], rv, A.phys[tl.x], noise_key(S, step),
                                               uint32_t(site), A.status);
            else
                collide_modeq3<L, Real, MODE>(f, drho, jc, rv, S, A.phys[tl.x], uint32_t(site), step, A.status);
            sfor<0, Q>([&](auto I) {
                constexpr int i = I;
                fo[i * N + site] = f[i];
            });
        }
    }
}

}  // namespace lbf

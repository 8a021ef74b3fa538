// Collision of the D2Q9 model with the modified equilibrium of Eq. 65 (the
// paper's coupling; Eq. 61 with the moment expansion of Eq. 66 and the noise
// of Eq. 68), written out for the basis 1, c_x, c_y, 3c^2 - 2, c_x^2 - c_y^2,
// c_x c_y, (3c^2 - 4) c_x, (3c^2 - 4) c_y, 9c^4 - 15c^2 + 2 (squared lengths
// N_a = 1, 1/3, 1/3, 4, 4/9, 1/9, 2/3, 2/3, 16):
//
//  * the moments of the equilibrium (deviation form; taking Eq. 65's
//    populations through the basis) are
//      m_0 = drho,  m_1 = j_x,  m_2 = j_y,
//      m_3 = 3 (X_xx + X_yy) - 2 drho + 6 iso,
//      m_4 = X_xx - X_yy + K_xx - K_yy,   m_5 = X_xy + K_xy,   m_6 = m_7 = 0,
//      m_8 = 2 drho - 3 (K_xx + K_yy) - 6 iso,
//    with iso = p0 - kappa rho lap rho, X_ab = rho u_a u_b + nu (u_a d_b rho +
//    u_b d_a rho + u.grad rho delta_ab) and K_ab = kappa d_a rho d_b rho;
//  * post-collision moments w_a = m_a - lambda_a (m_a - m^eq_a) + xi_a on the
//    non-conserved modes; with k_a = w_a / (36 N_a) the populations are
//    f_i = 36 t_i sum_a T_ai k_a, formed through the sums that opposite
//    velocities share.  MODE 2: every lambda_a = 1 (w = m^eq + xi, the
//    pre-collision populations are not read); MODE 1: one rate lambda,
//    f' = (1 - lambda) f + 36 t_i sum_a T_ai (lambda k^eq_a + k^xi_a);
//    MODE 0: a rate per mode, from the moments of f.
//
// V is float or double (one site) or float2 (two sites in lockstep, paired
// FP32 instructions; each lane gives the bits of the float form).  Every D2Q9
// kernel of the modified equilibrium goes through this function, so they
// agree bit for bit whatever registers the compiler gives each of them.
#pragma once

#include "collide_d3q19.cuh"

namespace lbf {

// Density deviation and momentum of one site (or a pair) from its pulled
// deviations: drho = sum_i f_i, j = sum_i c_i f_i, each summed in population
// order from zero.
template <class V>
__device__ __forceinline__ void moments_d2q9(const V (&f)[9], V& drho, V& jx, V& jy) {
    V r = vadd(vk<V>(0.0), f[0]);
#pragma unroll
    for (int i = 1; i < 9; ++i) r = vadd(r, f[i]);
    drho = r;
    // c_x: +1 for 1, 5, 7; -1 for 2, 6, 8.  c_y: +1 for 3, 5, 8; -1 for 4, 6, 7.
    jx = vsub(vadd(vsub(vadd(vsub(vadd(vk<V>(0.0), f[1]), f[2]), f[5]), f[6]), f[7]), f[8]);
    jy = vadd(vsub(vsub(vadd(vsub(vadd(vk<V>(0.0), f[3]), f[4]), f[5]), f[6]), f[7]), f[8]);
}

// f[i] <- post-collision deviations of the site(s) with density deviation
// drho and momentum j (f[i] holds the pre-collision deviations on entry,
// read unless MODE == 2); rv.at<cx, cy, 0>() is the density deviation at r + c.
template <int MODE, class V, class RhoV>
__device__ __forceinline__ void collide_d2q9_modeq(V (&f)[9], const V drho, const V jx, const V jy,
                                                   const RhoV& rv, const SysPhys<typename VT<V>::S>& P,
                                                   const NoiseKey& key, const typename SiteIdx<V>::type site,
                                                   int* status) {
    using S = typename VT<V>::S;
    constexpr int W = VT<V>::W;
    const V rho = vadd(vbc<V>(P.rho_c), drho);
    bool bad_rho = false;
#pragma unroll
    for (int l = 0; l < W; ++l) bad_rho |= !(lane(rho, l) > S(0));
    if (bad_rho) atomicOr(status, ST_RHO);

    // thermodynamics (Eq. 3 and below Eq. 64), phi = drho / rho_c
    const V phi = vmul(drho, vbc<V>(P.inv_rho_c));
    const V phi2 = vmul(phi, phi);
    const V df0 = vmul(phi, vfma(vbc<V>(P.b), phi2, vbc<V>(P.a)));
    const V f0 = vmul(phi2, vfma(vbc<V>(S(0.25) * P.b), phi2, vbc<V>(S(0.5) * P.a)));
    const V rr = vmul(rho, vbc<V>(P.inv_rho_c));
    const V p0 = vsub(vmul(rr, df0), f0);
    const V cs2 = vmul(vmul(rr, vbc<V>(P.inv_rho_c)), vfma(vbc<V>(S(3) * P.b), phi2, vbc<V>(P.a)));

    // d_a rho = 3 sum_i t_i c_ia rho(r + c_i) = (4 (E - W) + (NE - SW) +- (SE - NW)) / 12,
    // lap rho = 6 sum_i t_i (rho(r + c_i) - rho(r)) = (2/3) axes + (1/6) diagonals - (10/3) rho(r)
    const V dx = vsub(rv.template at<1, 0, 0>(), rv.template at<-1, 0, 0>());
    const V dy = vsub(rv.template at<0, 1, 0>(), rv.template at<0, -1, 0>());
    const V dp = vsub(rv.template at<1, 1, 0>(), rv.template at<-1, -1, 0>());
    const V dq = vsub(rv.template at<1, -1, 0>(), rv.template at<-1, 1, 0>());
    const V gx = vfma(dx, vk<V>(1.0 / 3.0), vmul(vadd(dp, dq), vk<V>(1.0 / 12.0)));
    const V gy = vfma(dy, vk<V>(1.0 / 3.0), vmul(vsub(dp, dq), vk<V>(1.0 / 12.0)));
    const V sa = vadd(vadd(rv.template at<1, 0, 0>(), rv.template at<-1, 0, 0>()),
                      vadd(rv.template at<0, 1, 0>(), rv.template at<0, -1, 0>()));
    const V sd = vadd(vadd(rv.template at<1, 1, 0>(), rv.template at<-1, -1, 0>()),
                      vadd(rv.template at<1, -1, 0>(), rv.template at<-1, 1, 0>()));
    const V lap = vfma(sa, vk<V>(2.0 / 3.0), vfma(sd, vk<V>(1.0 / 6.0), vmul(drho, vk<V>(-10.0 / 3.0))));

    const V ir = vmap(rho, [](S x) { return fast_rcp(x); });
    const V ux = vmul(jx, ir), uy = vmul(jy, ir);
    const V iso = vfma(vmul(rho, vbc<V>(-P.kappa)), lap, p0);          // p0 - kappa rho lap rho
    const V nu = vbc<V>(P.nu);
    const V udg = vfma(ux, gx, vmul(uy, gy));
    const V Xxx = vfma(jx, ux, vmul(nu, vfma(vadd(ux, ux), gx, udg)));
    const V Xyy = vfma(jy, uy, vmul(nu, vfma(vadd(uy, uy), gy, udg)));
    const V Xxy = vfma(jx, uy, vmul(nu, vfma(ux, gy, vmul(uy, gx))));
    const V kgx = vmul(vbc<V>(P.kappa), gx), kgy = vmul(vbc<V>(P.kappa), gy);
    const V Kxx = vmul(kgx, gx), Kyy = vmul(kgy, gy), Kxy = vmul(kgx, gy);
    const V Ksum = vadd(Kxx, Kyy);

    // k_a = m^eq_a / (36 N_a)
    V k[9];
    k[0] = vmul(drho, vk<V>(1.0 / 36.0));
    k[1] = vmul(jx, vk<V>(1.0 / 12.0));
    k[2] = vmul(jy, vk<V>(1.0 / 12.0));
    k[3] = vmul(vfma(vadd(Xxx, Xyy), vk<V>(3.0), vfma(iso, vk<V>(6.0), vmul(drho, vk<V>(-2.0)))),
                vk<V>(1.0 / 144.0));
    k[4] = vmul(vadd(vsub(Xxx, Xyy), vsub(Kxx, Kyy)), vk<V>(1.0 / 16.0));
    k[5] = vmul(vadd(Xxy, Kxy), vk<V>(1.0 / 4.0));
    k[6] = vk<V>(0.0);
    k[7] = vk<V>(0.0);
    k[8] = vmul(vfma(Ksum, vk<V>(-3.0), vfma(iso, vk<V>(-6.0), vadd(drho, drho))), vk<V>(1.0 / 576.0));
    if constexpr (MODE == 1) {
        // one rate: lambda k^eq (the (1 - lambda) f part is added at the end)
        const V lam = vbc<V>(P.lam_bgk);
#pragma unroll
        for (int a = 0; a < 9; ++a) k[a] = vmul(lam, k[a]);
    } else if constexpr (MODE == 0) {
        // per-mode rates on the moments of f, over 36 N_a:
        // k_a <- m_a / (36 N_a) + lambda_a (k^eq_a - m_a / (36 N_a)) on a >= 3
        const V ax = vadd(vadd(f[1], f[2]), vadd(f[3], f[4]));
        const V dg = vadd(vadd(f[5], f[6]), vadd(f[7], f[8]));
        V m[9];
        m[3] = vmul(vfma(dg, vk<V>(4.0), vfma(f[0], vk<V>(-2.0), ax)), vk<V>(1.0 / 144.0));
        m[4] = vmul(vsub(vadd(f[1], f[2]), vadd(f[3], f[4])), vk<V>(1.0 / 16.0));
        m[5] = vmul(vsub(vadd(f[5], f[6]), vadd(f[7], f[8])), vk<V>(1.0 / 4.0));
        const V d56 = vsub(f[5], f[6]), d78 = vsub(f[7], f[8]);
        m[6] = vmul(vfma(vadd(d56, d78), vk<V>(2.0), vsub(f[2], f[1])), vk<V>(1.0 / 24.0));
        m[7] = vmul(vfma(vsub(d56, d78), vk<V>(2.0), vsub(f[4], f[3])), vk<V>(1.0 / 24.0));
        m[8] = vmul(vfma(dg, vk<V>(8.0), vfma(ax, vk<V>(-4.0), vadd(f[0], f[0]))), vk<V>(1.0 / 576.0));
#pragma unroll
        for (int a = 3; a < 9; ++a) k[a] = vfma(vbc<V>(P.lam[a]), vsub(k[a], m[a]), m[a]);
    }

    if (P.kT > S(0)) {
        // scale sqrt(3 rho kT) (Eq. 68 with Delta V = Delta t = 1; the variance
        // carries the factor the draws of the lane precision expect) and the
        // Cholesky factor of the coupled pair (modes 3c^2 - 2 and 9c^4 - 15c^2 + 2,
        // rest components -2 and 2): M = [[(4 + 4 om) g_33, -4 om g_38],
        // [-4 om g_38, (16 + 4 om) g_88]], om = 1 - 3 c_s^2, g = 1 at tau = 1,
        // where the determinant is 64 + 80 om (positive only where 4 + 4 om is
        // too); paired arithmetic, the special functions lane by lane
        const V sc = vsqrt_pos(vmul(vbc<V>(vmul(S(3.0 * DrawScale<S>::v), P.kT)), rho));
        const V om = vfma(cs2, vk<V>(-3.0), vk<V>(1.0));
        V mpp, det, mpr;
        if constexpr (MODE == 2) {
            mpp = vfma(om, vk<V>(4.0), vk<V>(4.0));
            mpr = vmul(om, vk<V>(-4.0));
            det = vfma(om, vk<V>(80.0), vk<V>(64.0));
        } else {
            mpp = vmul(vfma(om, vk<V>(4.0), vk<V>(4.0)), vbc<V>(P.g_diag[3]));
            mpr = vmul(vmul(om, vk<V>(-4.0)), vbc<V>(P.g_pair));
            det = vfma(mpp, vmul(vfma(om, vk<V>(4.0), vk<V>(16.0)), vbc<V>(P.g_diag[8])),
                       vmul(vmul(mpr, mpr), vk<V>(-1.0)));
        }
        const V q = vrsqrt(mpp);
        V k11 = vmul(vmul(mpp, q), vk<V>(1.0 / 144.0));
        V k21 = vmul(vmul(mpr, q), vk<V>(1.0 / 576.0));
        V k22 = vmul(vmul(det, vrsqrt(vmul(det, mpp))), vk<V>(1.0 / 576.0));
        auto bad = [&](int l) { return !(lane(det, l) > S(0)) || (MODE != 2 && !(lane(mpp, l) > S(0))); };
        bool bad_noise = false;
#pragma unroll
        for (int l = 0; l < W; ++l) bad_noise = bad_noise || bad(l);
        if (bad_noise) {
#pragma unroll
            for (int l = 0; l < W; ++l) {
                if (bad(l)) {
                    set_lane(k11, l, S(0));
                    set_lane(k21, l, S(0));
                    set_lane(k22, l, S(0));
                }
            }
            atomicOr(status, ST_NOISE);
        }
        // the normal of mode a is number a - 3 in draw order; its amplitude over
        // 36 N_a: sqrt(N_a g_aa) / (36 N_a)
        V c4, c5, c67a, c67b;
        if constexpr (MODE == 2) {
            c4 = vk<V>(1.0 / 24.0);
            c5 = vk<V>(1.0 / 12.0);
            c67a = c67b = vk<V>(1.0 / (36.0 * 0.81649658092772603));
        } else {
            c4 = vbc<V>(vmul(P.namp[4], S(1.0 / 16.0)));
            c5 = vbc<V>(vmul(P.namp[5], S(1.0 / 4.0)));
            c67a = vbc<V>(vmul(P.namp[6], S(1.0 / 24.0)));
            c67b = vbc<V>(vmul(P.namp[7], S(1.0 / 24.0)));
        }
        V n[4];
        draw4(key, site, 0u, sc, sc, n, true);
        const V n3 = n[0];
        k[3] = vfma(k11, n3, k[3]);
        k[4] = vfma(n[1], c4, k[4]);
        k[5] = vfma(n[2], c5, k[5]);
        k[6] = vfma(n[3], c67a, k[6]);
        draw4(key, site, 1u, sc, sc, n, false);
        k[7] = vfma(n[0], c67b, k[7]);
        k[8] = vfma(k22, n[1], vfma(k21, n3, k[8]));
    }

    // g_i = 36 t_i sum_a T_ai k_a (36 t = 16 rest, 4 axes, 1 diagonals)
    V g[9];
    g[0] = vmul(vfma(vsub(k[8], k[3]), vk<V>(2.0), k[0]), vk<V>(16.0));
    {
        const V B = vfma(k[8], vk<V>(-4.0), vadd(k[0], k[3]));
        const V Ex = vadd(B, k[4]), Ey = vsub(B, k[4]);
        const V Ox = vsub(k[1], k[6]), Oy = vsub(k[2], k[7]);
        g[1] = vmul(vadd(Ex, Ox), vk<V>(4.0));
        g[2] = vmul(vsub(Ex, Ox), vk<V>(4.0));
        g[3] = vmul(vadd(Ey, Oy), vk<V>(4.0));
        g[4] = vmul(vsub(Ey, Oy), vk<V>(4.0));
    }
    {
        const V C = vfma(k[8], vk<V>(8.0), vfma(k[3], vk<V>(4.0), k[0]));
        const V Xd = vfma(k[6], vk<V>(2.0), k[1]), Yd = vfma(k[7], vk<V>(2.0), k[2]);
        const V Ep = vadd(C, k[5]), Em = vsub(C, k[5]);
        const V Op = vadd(Xd, Yd), Om = vsub(Xd, Yd);
        g[5] = vadd(Ep, Op);
        g[6] = vsub(Ep, Op);
        g[7] = vadd(Em, Om);
        g[8] = vsub(Em, Om);
    }
    if constexpr (MODE == 1) {
        const V oml = vbc<V>(S(1) - P.lam_bgk);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = vfma(oml, f[i], g[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = g[i];
    }
}

}  // namespace lbf

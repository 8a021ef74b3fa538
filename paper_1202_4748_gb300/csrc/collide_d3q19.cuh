// Fully relaxed (every non-conserved mode at tau = 1) Guo-forced collision of
// the D3Q19 model (Eq. 61 with the moment expansion of Eq. 66, the noise of
// Eq. 68 in its lattice-general form, and the Landau pressure p0 of Eq. 3 in
// the equilibrium), written out for this basis so that the arithmetic is a
// short straight line:
//
//  * post-collision moments (deviation form, lambda = 1):
//      w_0 = drho,  w_a = j_a + F_a (a = x, y, z),
//      with A_bc = rho u_b u_c + (u_b F_c + u_c F_b) / 2 (the equilibrium's
//      second moments plus half the Guo source, whose projections on the
//      second-order modes come out with unit coefficients),
//      w_4 = tr A - iso + xi_4,  w_5 = 3 A_xx - tr A + xi_5,  w_6 = A_yy - A_zz + xi_6,
//      w_7 = A_xy + xi_7,  w_8 = A_yz + xi_8,  w_9 = A_zx + xi_9,
//      w_16 = iso + xi_16,  w_a = xi_a on the other ghost modes,
//      iso = drho - 3 p0, u = (j + F / 2) / rho, F = kappa rho grad(lap rho);
//  * h_a = w_a / (36 N_a), and f_i = 36 t_i sum_a T_ai h_a evaluated through
//    the sums that the velocities share (the rest, face and edge classes of
//    the basis table), about half the operations of a dense T^-1 product.
//
// V is float or double (one site) or float2 (two sites in lockstep, the
// paired FP32 instructions); each lane of the float2 form gives the bits of
// the float form.  The noise draws (Philox4x32-10, Box-Muller) are per site.
#pragma once

#include "lb_device.cuh"
#include "vec2.cuh"

namespace lbf {

// Philox counter words shared by the sites of one step of one system, and the
// parts of rounds 1 and 2 of Philox4x32-10 on the counter (site, step low
// word, step high word, tag | d) that depend on neither the site nor the draw
// d: the step words enter those rounds' products only through counter words 1
// and 2, so noise_key forms them once per kernel and a draw starts from one
// product of the site (shared by the site's draws) and one of its own.
struct NoiseKey {
    uint32_t k0, k1;      // key: the seed
    uint32_t slo, shi;    // step
    uint32_t tag;         // system_id << 8 (the draw index fills the low byte)
    uint32_t t1;          // tag ^ k1: round 1 gives word 2 = hi(M0 site) ^ t1 ^ d
    uint32_t y1k;         // lo(M1 shi) ^ (k0 + W0): round 2 gives word 0 = hi(M1 z1) ^ y1k
    uint32_t z2k, w2;     // hi(M0 x1) ^ (k1 + W1) and lo(M0 x1), x1 = hi(M1 shi) ^ slo ^ k0:
                          // round 2 gives word 2 = z2k ^ lo(M0 site) and word 3 = w2
};
__device__ __forceinline__ NoiseKey noise_key(const SysDev& S, int64_t step) {
    NoiseKey k;
    k.k0 = S.seed_lo;
    k.k1 = S.seed_hi;
    k.slo = uint32_t(uint64_t(step) & 0xffffffffu);
    k.shi = uint32_t(uint64_t(step) >> 32);
    k.tag = S.system_id << 8;
    k.t1 = k.tag ^ k.k1;
    const uint64_t q1 = uint64_t(kPhiloxM1) * k.shi;
    const uint32_t x1 = uint32_t(q1 >> 32) ^ k.slo ^ k.k0;
    k.y1k = uint32_t(q1) ^ (k.k0 + kPhiloxW0);
    const uint64_t q2 = uint64_t(kPhiloxM0) * x1;
    k.z2k = uint32_t(q2 >> 32) ^ (k.k1 + kPhiloxW1);
    k.w2 = uint32_t(q2);
    return k;
}

// philox4x32_10((site, slo, shi, tag | d), k0, k1) for a draw d < 256, with
// rounds 1 and 2 completed from the words noise_key formed.
__device__ __forceinline__ uint4 philox_draw(const NoiseKey& k, uint32_t site, uint32_t d) {
    const uint64_t p0 = uint64_t(kPhiloxM0) * site;                // round 1
    const uint32_t z1 = uint32_t(p0 >> 32) ^ k.t1 ^ d;
    const uint64_t p1 = uint64_t(kPhiloxM1) * z1;                  // round 2
    uint4 c = make_uint4(uint32_t(p1 >> 32) ^ k.y1k, uint32_t(p1), k.z2k ^ uint32_t(p0), k.w2);
    uint32_t k0 = k.k0 + kPhiloxW0, k1 = k.k1 + kPhiloxW1;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
        const uint64_t pa = uint64_t(kPhiloxM0) * c.x;
        const uint64_t pb = uint64_t(kPhiloxM1) * c.z;
        c = make_uint4(uint32_t(pb >> 32) ^ c.y ^ k0, uint32_t(pb), uint32_t(pa >> 32) ^ c.w ^ k1, uint32_t(pa));
    }
    return c;
}

// Site indices of the lanes: one per lane.
template <class V>
struct SiteIdx {
    using type = uint32_t;
};
template <>
struct SiteIdx<float2> {
    using type = uint2;
};

// Special-function-unit approximations (the PTX .approx instructions) with
// subnormal operands flushed: every operand they get here is a normal number
// or zero (uniforms U >= 2^-33, -log2 U >= 0, angles in [-pi, pi] with a
// spacing of 2^-24 pi, noise variances of order kT), where flushing changes
// no result and saves the subnormal handling around each instruction.
__device__ __forceinline__ float sfu_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_sin(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_cos(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Factor that the draws of a lane precision expect in the variance from which
// their scale is formed (draw4): 2 ln 2 in float, 1 in double.
template <class S>
struct DrawScale;
template <>
struct DrawScale<float> {
    static constexpr double v = 1.3862943611198906;
};
template <>
struct DrawScale<double> {
    static constexpr double v = 1.0;
};

// Four normals of draw d for every lane: n0, n1 from the words (w0, w1)
// scaled by sc0, n2, n3 from (w2, w3) scaled by sc1 (two scales, so that a
// mode's constant can ride on its pair's scale).  Float: the scales carry
// the factor sqrt(2 ln 2) of the Box-Muller radius sqrt(-2 ln U) =
// sqrt(2 ln 2) sqrt(-log2 U), so the radius is formed from -log2 U directly,
// and the angle 2 pi U_b - pi (in [-pi, pi], where the hardware sine and
// cosine are accurate; the half turn flips the signs of both, which the
// negated scales undo) is formed from the word in one rounding.
// need3 = false skips the sine of the second pair (its normal is not used).
__device__ __forceinline__ void draw4(const NoiseKey& k, uint32_t site, uint32_t d, float sc0, float sc1,
                                      float (&n)[4], bool need3) {
    const uint4 w = philox_draw(k, site, d);
    constexpr float kU = 2.3283064365386963e-10f, kU0 = 1.1641532182693481e-10f;   // U = (w + 1/2) 2^-32
    constexpr float kT = 1.4629180792671596e-09f, kT0 = -3.1415926528583340f;      // 2 pi U - pi
    const float ua0 = vfma(float(w.x), kU, kU0);
    const float ua1 = vfma(float(w.z), kU, kU0);
    const float rr0 = vmul(sfu_sqrt(fmaxf(-sfu_lg2(ua0), 0.0f)), -sc0);
    const float rr1 = vmul(sfu_sqrt(fmaxf(-sfu_lg2(ua1), 0.0f)), -sc1);
    const float t0 = vfma(float(w.y), kT, kT0);
    const float t1 = vfma(float(w.w), kT, kT0);
    n[0] = vmul(rr0, sfu_cos(t0));
    n[1] = vmul(rr0, sfu_sin(t0));
    n[2] = vmul(rr1, sfu_cos(t1));
    n[3] = need3 ? vmul(rr1, sfu_sin(t1)) : 0.0f;
}

// Two sites: the same sequence lane by lane, the lane-independent arithmetic paired.
__device__ __forceinline__ void draw4(const NoiseKey& k, uint2 site, uint32_t d, float2 sc0, float2 sc1,
                                      float2 (&n)[4], bool need3) {
    const uint4 wa = philox_draw(k, site.x, d);
    const uint4 wb = philox_draw(k, site.y, d);
    const float2 kU = vk<float2>(2.3283064365386963e-10), kU0 = vk<float2>(1.1641532182693481e-10);
    const float2 kT = vk<float2>(1.4629180792671596e-09), kT0 = vk<float2>(-3.1415926528583340);
    const float2 ua0 = vfma(make_float2(float(wa.x), float(wb.x)), kU, kU0);
    const float2 ua1 = vfma(make_float2(float(wa.z), float(wb.z)), kU, kU0);
    const float2 r0 = make_float2(sfu_sqrt(fmaxf(-sfu_lg2(ua0.x), 0.0f)), sfu_sqrt(fmaxf(-sfu_lg2(ua0.y), 0.0f)));
    const float2 r1 = make_float2(sfu_sqrt(fmaxf(-sfu_lg2(ua1.x), 0.0f)), sfu_sqrt(fmaxf(-sfu_lg2(ua1.y), 0.0f)));
    const float2 rr0 = vmul(r0, make_float2(-sc0.x, -sc0.y));
    const float2 rr1 = vmul(r1, make_float2(-sc1.x, -sc1.y));
    const float2 t0 = vfma(make_float2(float(wa.y), float(wb.y)), kT, kT0);
    const float2 t1 = vfma(make_float2(float(wa.w), float(wb.w)), kT, kT0);
    n[0] = vmul(rr0, make_float2(sfu_cos(t0.x), sfu_cos(t0.y)));
    n[1] = vmul(rr0, make_float2(sfu_sin(t0.x), sfu_sin(t0.y)));
    n[2] = vmul(rr1, make_float2(sfu_cos(t1.x), sfu_cos(t1.y)));
    n[3] = need3 ? vmul(rr1, make_float2(sfu_sin(t1.x), sfu_sin(t1.y))) : make_float2(0.0f, 0.0f);
}

// FP64: U = (x + 1/2) 2^-32 exactly, R = sqrt(-2 ln U), angle 2 pi U_b, with
// the library's correctly rounded functions.
__device__ __forceinline__ void draw4(const NoiseKey& k, uint32_t site, uint32_t d, double sc0, double sc1,
                                      double (&n)[4], bool need3) {
    const uint4 w = philox_draw(k, site, d);
    double a, b;
    box_muller(w.x, w.y, a, b);
    n[0] = vmul(sc0, a);
    n[1] = vmul(sc0, b);
    box_muller(w.z, w.w, a, b);
    n[2] = vmul(sc1, a);
    n[3] = need3 ? vmul(sc1, b) : 0.0;
}

// 1 / sqrt(x) lane by lane.
__device__ __forceinline__ float vrsqrt(float x) { return sfu_rsqrt(x); }
__device__ __forceinline__ float2 vrsqrt(float2 x) { return make_float2(sfu_rsqrt(x.x), sfu_rsqrt(x.y)); }
__device__ __forceinline__ double vrsqrt(double x) { return rsqrt(x); }

// Noise scale sqrt(max(x, 0)) lane by lane: the special-function square root
// in float, the library's in double.
__device__ __forceinline__ float vsqrt_pos(float x) { return sfu_sqrt(fmaxf(x, 0.0f)); }
__device__ __forceinline__ float2 vsqrt_pos(float2 x) {
    return make_float2(sfu_sqrt(fmaxf(x.x, 0.0f)), sfu_sqrt(fmaxf(x.y, 0.0f)));
}
__device__ __forceinline__ double vsqrt_pos(double x) { return sqrt(x > 0.0 ? x : 0.0); }

// Laplacian of the density, lap rho = 6 sum_i t_i (rho(r + c_i) - rho(r))
// = (1/3) (sum of the 6 face neighbours) + (1/6) (sum of the 12 edge
// neighbours) - 4 rho(r), summed in a fixed order (rv.at<cx, cy, cz>() is the
// density at r + c).
template <class V, class RV>
__device__ __forceinline__ V lap_d3q19(const RV& rv) {
    const V faces = vadd(vadd(vadd(rv.template at<1, 0, 0>(), rv.template at<-1, 0, 0>()),
                              vadd(rv.template at<0, 1, 0>(), rv.template at<0, -1, 0>())),
                         vadd(rv.template at<0, 0, 1>(), rv.template at<0, 0, -1>()));
    const V exy = vadd(vadd(rv.template at<1, 1, 0>(), rv.template at<-1, -1, 0>()),
                       vadd(rv.template at<1, -1, 0>(), rv.template at<-1, 1, 0>()));
    const V exz = vadd(vadd(rv.template at<1, 0, 1>(), rv.template at<-1, 0, -1>()),
                       vadd(rv.template at<1, 0, -1>(), rv.template at<-1, 0, 1>()));
    const V eyz = vadd(vadd(rv.template at<0, 1, 1>(), rv.template at<0, -1, -1>()),
                       vadd(rv.template at<0, 1, -1>(), rv.template at<0, -1, 1>()));
    const V edges = vadd(vadd(exy, exz), eyz);
    return vfma(faces, vk<V>(1.0 / 3.0), vfma(edges, vk<V>(1.0 / 6.0), vmul(rv.template at<0, 0, 0>(), vk<V>(-4.0))));
}

// Gradient of the Laplacian, times 12: 12 sum_i 3 t_i c_ia lap(r + c_i), i.e.
// 2 (L(+a) - L(-a)) plus the four edges with c_a = +1 minus the four with -1.
template <class V, class LapV>
__device__ __forceinline__ void grad_lap12_d3q19(const LapV& lv, V& gx, V& gy, V& gz) {
    {
        const V p = vadd(vadd(lv.template at<1, 1, 0>(), lv.template at<1, -1, 0>()),
                         vadd(lv.template at<1, 0, 1>(), lv.template at<1, 0, -1>()));
        const V m = vadd(vadd(lv.template at<-1, -1, 0>(), lv.template at<-1, 1, 0>()),
                         vadd(lv.template at<-1, 0, -1>(), lv.template at<-1, 0, 1>()));
        gx = vfma(vsub(lv.template at<1, 0, 0>(), lv.template at<-1, 0, 0>()), vk<V>(2.0), vsub(p, m));
    }
    {
        const V p = vadd(vadd(lv.template at<1, 1, 0>(), lv.template at<-1, 1, 0>()),
                         vadd(lv.template at<0, 1, 1>(), lv.template at<0, 1, -1>()));
        const V m = vadd(vadd(lv.template at<-1, -1, 0>(), lv.template at<1, -1, 0>()),
                         vadd(lv.template at<0, -1, -1>(), lv.template at<0, -1, 1>()));
        gy = vfma(vsub(lv.template at<0, 1, 0>(), lv.template at<0, -1, 0>()), vk<V>(2.0), vsub(p, m));
    }
    {
        const V p = vadd(vadd(lv.template at<1, 0, 1>(), lv.template at<-1, 0, 1>()),
                         vadd(lv.template at<0, 1, 1>(), lv.template at<0, -1, 1>()));
        const V m = vadd(vadd(lv.template at<-1, 0, -1>(), lv.template at<1, 0, -1>()),
                         vadd(lv.template at<0, -1, -1>(), lv.template at<0, 1, -1>()));
        gz = vfma(vsub(lv.template at<0, 0, 1>(), lv.template at<0, 0, -1>()), vk<V>(2.0), vsub(p, m));
    }
}

// The part every fully relaxed D3Q19 collision shares: given h_a = w_a /
// (36 N_a) of the equilibrium moments (h[0..9] and h[16]; h[10..15], h[17],
// h[18] are set here), adds the noise of Eq. 68 in its lattice-general form
// (rate 1 on every mode) and forms f_i = 36 t_i sum_a T_ai h_a.
template <class V>
__device__ __forceinline__ void d3q19_tau1_noise_and_populations(V (&h)[19], V (&f)[19], const V rho, const V cs2,
                                                                 const SysPhys<typename VT<V>::S>& P,
                                                                 const NoiseKey& key,
                                                                 const typename SiteIdx<V>::type site, int* status) {
    using S = typename VT<V>::S;
    constexpr int W = VT<V>::W;
    if (P.kT > S(0)) {
        // scale sqrt(3 rho kT) (Eq. 68 with Delta V = Delta t = 1; the variance
        // carries the factor the draws of the lane precision expect) and the
        // Cholesky factor of the coupled pair (modes c^2 - 1, 3c^4 - 6c^2 + 1):
        // M = [[2/3 + om, -om], [-om, 2 + om]], om = 1 - 3 c_s^2, whose
        // determinant is 4/3 + 8/3 om (positive only where 2/3 + om is too);
        // paired arithmetic, the special functions lane by lane
        const V sc = vsqrt_pos(vmul(vbc<V>(vmul(S(3.0 * DrawScale<S>::v), P.kT)), rho));
        const V om = vfma(cs2, vk<V>(-3.0), vk<V>(1.0));
        const V mpp = vadd(vk<V>(2.0 / 3.0), om);
        const V det = vfma(om, vk<V>(8.0 / 3.0), vk<V>(4.0 / 3.0));
        const V q = vrsqrt(mpp);
        V k11 = vmul(vmul(mpp, q), vk<V>(1.0 / 24.0));
        V k21 = vmul(vmul(om, q), vk<V>(-1.0 / 72.0));
        V k22 = vmul(vmul(det, vrsqrt(vmul(det, mpp))), vk<V>(1.0 / 72.0));
        bool bad_noise = false;
#pragma unroll
        for (int l = 0; l < W; ++l) bad_noise = bad_noise || !(lane(det, l) > S(0));
        if (bad_noise) {
#pragma unroll
            for (int l = 0; l < W; ++l) {
                if (!(lane(det, l) > S(0))) {
                    set_lane(k11, l, S(0));
                    set_lane(k21, l, S(0));
                    set_lane(k22, l, S(0));
                }
            }
            atomicOr(status, ST_NOISE);
        }
        // the normal of mode a is number a - 4 in draw order; c_a = 1 / (36 sqrt(N_a)),
        // carried by the pair's scale where both normals of a pair share it
        const double c5 = 1.0 / (36.0 * 1.1547005383792515), c6 = 1.0 / 24.0, c7 = 1.0 / 12.0;
        const double c10 = 1.0 / (36.0 * 0.81649658092772603), c13 = 1.0 / (12.0 * 1.4142135623730951);
        V n[4];
        draw4(key, site, 0u, sc, sc, n, true);
        const V n4 = n[0];
        h[4] = vfma(k11, n4, h[4]);
        h[5] = vfma(n[1], vk<V>(c5), h[5]);
        h[6] = vfma(n[2], vk<V>(c6), h[6]);
        h[7] = vfma(n[3], vk<V>(c7), h[7]);
        draw4(key, site, 1u, sc, vmul(sc, vk<V>(c10)), n, true);
        h[8] = vfma(n[0], vk<V>(c7), h[8]);
        h[9] = vfma(n[1], vk<V>(c7), h[9]);
        h[10] = n[2];
        h[11] = n[3];
        draw4(key, site, 2u, sc, vmul(sc, vk<V>(c13)), n, true);
        h[12] = vmul(n[0], vk<V>(c10));
        h[13] = vmul(n[1], vk<V>(c13));
        h[14] = n[2];
        h[15] = n[3];
        draw4(key, site, 3u, sc, sc, n, false);
        h[16] = vfma(k22, n[0], vfma(k21, n4, h[16]));
        h[17] = vmul(n[1], vk<V>(c5));
        h[18] = vmul(n[2], vk<V>(c6));
    } else {
#pragma unroll
        for (int a = 10; a < 16; ++a) h[a] = vk<V>(0.0);
        h[17] = vk<V>(0.0);
        h[18] = vk<V>(0.0);
    }

    // f_i = 36 t_i sum_a T_ai h_a.  Rest: 12 (h0 - h4 + h16).
    f[0] = vmul(vadd(vsub(h[0], h[4]), h[16]), vk<V>(12.0));
    // faces (36 t = 2): even parts G + 2 D5, G - D5 +- D6; odd parts h_a - 2 h_{a+9}
    {
        const V G = vfma(h[16], vk<V>(-2.0), h[0]);
        const V D5 = vsub(h[5], h[17]), D6 = vsub(h[6], h[18]);
        const V Ex = vfma(D5, vk<V>(2.0), G);
        const V GD = vsub(G, D5);
        const V Ey = vadd(GD, D6), Ez = vsub(GD, D6);
        const V Ox = vfma(h[10], vk<V>(-2.0), h[1]);
        const V Oy = vfma(h[11], vk<V>(-2.0), h[2]);
        const V Oz = vfma(h[12], vk<V>(-2.0), h[3]);
        V s;
        s = vadd(Ex, Ox); f[1] = vadd(s, s);
        s = vsub(Ex, Ox); f[2] = vadd(s, s);
        s = vadd(Ey, Oy); f[3] = vadd(s, s);
        s = vsub(Ey, Oy); f[4] = vadd(s, s);
        s = vadd(Ez, Oz); f[5] = vadd(s, s);
        s = vsub(Ez, Oz); f[6] = vadd(s, s);
    }
    // edges (36 t = 1): even parts C + P5 +- P6 (xy, xz), C - 2 P5 (yz), plus the
    // off-diagonal stress mode of the plane; odd parts from X+-, Y+-, Z+-
    {
        const V C = vadd(vadd(h[0], h[4]), h[16]);
        const V P5 = vadd(h[5], h[17]), P6 = vadd(h[6], h[18]);
        const V CP5 = vadd(C, P5);
        const V Bxy = vadd(CP5, P6), Bxz = vsub(CP5, P6), Byz = vfma(P5, vk<V>(-2.0), C);
        const V X = vadd(h[1], h[10]), Y = vadd(h[2], h[11]), Z = vadd(h[3], h[12]);
        const V Xp = vadd(X, h[13]), Xm = vsub(X, h[13]);
        const V Yp = vadd(Y, h[14]), Ym = vsub(Y, h[14]);
        const V Zp = vadd(Z, h[15]), Zm = vsub(Z, h[15]);
        V E, O;
        E = vadd(Bxy, h[7]); O = vadd(Xp, Ym); f[7] = vadd(E, O); f[8] = vsub(E, O);
        E = vsub(Bxy, h[7]); O = vsub(Xp, Ym); f[9] = vadd(E, O); f[10] = vsub(E, O);
        E = vadd(Bxz, h[9]); O = vadd(Xm, Zp); f[11] = vadd(E, O); f[12] = vsub(E, O);
        E = vsub(Bxz, h[9]); O = vsub(Xm, Zp); f[13] = vadd(E, O); f[14] = vsub(E, O);
        E = vadd(Byz, h[8]); O = vadd(Yp, Zm); f[15] = vadd(E, O); f[16] = vsub(E, O);
        E = vsub(Byz, h[8]); O = vsub(Yp, Zm); f[17] = vadd(E, O); f[18] = vsub(E, O);
    }
}

// f[i] <- post-collision deviations of the site(s) with density deviation
// drho and momentum j = sum_i c_i f_i; lv views the Laplacian of the density
// around the site(s).
template <class V, class LapV>
__device__ __forceinline__ void collide_d3q19_tau1(V (&f)[19], const V drho, const V jx, const V jy, const V jz,
                                                   const LapV& lv, const SysPhys<typename VT<V>::S>& P,
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
    const V iso = vfma(p0, vk<V>(-3.0), drho);

    // Guo force F = kappa rho grad(lap rho); u = (j + F / 2) / rho
    V gx, gy, gz;
    grad_lap12_d3q19<V>(lv, gx, gy, gz);
    const V kr = vmul(rho, vbc<V>(P.kappa * S(1.0 / 12.0)));
    const V Fx = vmul(kr, gx), Fy = vmul(kr, gy), Fz = vmul(kr, gz);
    const V ir = vmap(rho, [](S x) { return fast_rcp(x); });
    const V ux = vmul(vfma(Fx, vk<V>(0.5), jx), ir);
    const V uy = vmul(vfma(Fy, vk<V>(0.5), jy), ir);
    const V uz = vmul(vfma(Fz, vk<V>(0.5), jz), ir);
    // A_bc with V_b = rho u_b + F_b:  A_bb = u_b V_b,  2 A_bc = u_b V_c + u_c V_b
    const V Vx = vfma(rho, ux, Fx), Vy = vfma(rho, uy, Fy), Vz = vfma(rho, uz, Fz);
    const V Axx = vmul(ux, Vx), Ayy = vmul(uy, Vy), Azz = vmul(uz, Vz);
    const V Axy2 = vfma(ux, Vy, vmul(uy, Vx));
    const V Ayz2 = vfma(uy, Vz, vmul(uz, Vy));
    const V Azx2 = vfma(uz, Vx, vmul(ux, Vz));
    const V tr = vadd(vadd(Axx, Ayy), Azz);

    // h_a = w_a / (36 N_a); N = (1, 1/3 x3, 2/3, 4/3, 4/9, 1/9 x3, 2/3 x3, 2/9 x3, 2, 4/3, 4/9)
    V h[19];
    h[0] = vmul(drho, vk<V>(1.0 / 36.0));
    h[1] = vmul(vadd(jx, Fx), vk<V>(1.0 / 12.0));
    h[2] = vmul(vadd(jy, Fy), vk<V>(1.0 / 12.0));
    h[3] = vmul(vadd(jz, Fz), vk<V>(1.0 / 12.0));
    h[4] = vmul(vsub(tr, iso), vk<V>(1.0 / 24.0));
    h[5] = vmul(vfma(Axx, vk<V>(3.0), vsub(vk<V>(0.0), tr)), vk<V>(1.0 / 48.0));
    h[6] = vmul(vsub(Ayy, Azz), vk<V>(1.0 / 16.0));
    h[7] = vmul(Axy2, vk<V>(1.0 / 8.0));
    h[8] = vmul(Ayz2, vk<V>(1.0 / 8.0));
    h[9] = vmul(Azx2, vk<V>(1.0 / 8.0));
    h[16] = vmul(iso, vk<V>(1.0 / 72.0));

    d3q19_tau1_noise_and_populations<V>(h, f, rho, cs2, P, key, site, status);
}

// The modified equilibrium carried to D3Q19 (Eq. 65's structure with the
// isotropic weights 3 t_i and the rotation-invariant square-gradient terms),
// fully relaxed.  Its moments on this basis (deviation form) are
//   m_0 = drho, m_a = j_a,
//   m_4 = tr X + 3 iso - drho - (kappa/2)|g|^2,
//   m_5 = 2 X_xx - X_yy - X_zz + kappa (2 g_x^2 - g_y^2 - g_z^2),
//   m_6 = X_yy - X_zz + kappa (g_y^2 - g_z^2),
//   m_7 = X_xy + kappa g_x g_y,  m_8 = X_yz + kappa g_y g_z,  m_9 = X_zx + kappa g_z g_x,
//   m_16 = drho - (3 kappa/2)|g|^2 - 3 iso,  the third- and fourth-order ghosts 0,
// with g = grad rho, iso = p0 - kappa rho lap rho and X_ab = rho u_a u_b +
// nu (u_a g_b + u_b g_a + u.g delta_ab); rv.at<cx, cy, cz>() is the density
// deviation at r + c.
template <class V, class RhoV>
__device__ __forceinline__ void collide_d3q19_modeq_tau1(V (&f)[19], const V drho, const V jx, const V jy,
                                                         const V jz, const RhoV& rv,
                                                         const SysPhys<typename VT<V>::S>& P, const NoiseKey& key,
                                                         const typename SiteIdx<V>::type site, int* status) {
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

    // g_a = 3 sum_i t_i c_ia rho(r + c_i) = (face difference) / 6 + (edge differences) / 12
    V g[3];
    {
        const V dfx = vsub(rv.template at<1, 0, 0>(), rv.template at<-1, 0, 0>());
        const V dfy = vsub(rv.template at<0, 1, 0>(), rv.template at<0, -1, 0>());
        const V dfz = vsub(rv.template at<0, 0, 1>(), rv.template at<0, 0, -1>());
        const V exy = vsub(rv.template at<1, 1, 0>(), rv.template at<-1, -1, 0>());
        const V exm = vsub(rv.template at<1, -1, 0>(), rv.template at<-1, 1, 0>());
        const V exz = vsub(rv.template at<1, 0, 1>(), rv.template at<-1, 0, -1>());
        const V ezm = vsub(rv.template at<1, 0, -1>(), rv.template at<-1, 0, 1>());
        const V eyz = vsub(rv.template at<0, 1, 1>(), rv.template at<0, -1, -1>());
        const V eym = vsub(rv.template at<0, 1, -1>(), rv.template at<0, -1, 1>());
        // x: (1,1,0), (1,-1,0), (1,0,1), (1,0,-1) minus their opposites
        g[0] = vfma(dfx, vk<V>(1.0 / 6.0), vmul(vadd(vadd(exy, exm), vadd(exz, ezm)), vk<V>(1.0 / 12.0)));
        // y: (1,1,0), (-1,1,0) = -exm, (0,1,1), (0,1,-1)
        g[1] = vfma(dfy, vk<V>(1.0 / 6.0), vmul(vadd(vsub(exy, exm), vadd(eyz, eym)), vk<V>(1.0 / 12.0)));
        // z: (1,0,1), (-1,0,1) = -ezm, (0,1,1), (0,-1,1) = -eym
        g[2] = vfma(dfz, vk<V>(1.0 / 6.0), vmul(vadd(vsub(exz, ezm), vsub(eyz, eym)), vk<V>(1.0 / 12.0)));
    }
    const V lap = lap_d3q19<V>(rv);

    const V ir = vmap(rho, [](S x) { return fast_rcp(x); });
    const V ux = vmul(jx, ir), uy = vmul(jy, ir), uz = vmul(jz, ir);
    const V iso = vfma(vmul(rho, vbc<V>(-P.kappa)), lap, p0);          // p0 - kappa rho lap rho
    const V nu = vbc<V>(P.nu);
    const V udg = vfma(ux, g[0], vfma(uy, g[1], vmul(uz, g[2])));
    const V Xxx = vfma(jx, ux, vmul(nu, vfma(vadd(ux, ux), g[0], udg)));
    const V Xyy = vfma(jy, uy, vmul(nu, vfma(vadd(uy, uy), g[1], udg)));
    const V Xzz = vfma(jz, uz, vmul(nu, vfma(vadd(uz, uz), g[2], udg)));
    const V Xxy = vfma(jx, uy, vmul(nu, vfma(ux, g[1], vmul(uy, g[0]))));
    const V Xyz = vfma(jy, uz, vmul(nu, vfma(uy, g[2], vmul(uz, g[1]))));
    const V Xzx = vfma(jz, ux, vmul(nu, vfma(uz, g[0], vmul(ux, g[2]))));
    const V kgx = vmul(vbc<V>(P.kappa), g[0]), kgy = vmul(vbc<V>(P.kappa), g[1]), kgz = vmul(vbc<V>(P.kappa), g[2]);
    const V Kxx = vmul(kgx, g[0]), Kyy = vmul(kgy, g[1]), Kzz = vmul(kgz, g[2]);
    const V Ksum = vadd(vadd(Kxx, Kyy), Kzz);
    const V trX = vadd(vadd(Xxx, Xyy), Xzz);

    // h_a = m_a / (36 N_a); N = (1, 1/3 x3, 2/3, 4/3, 4/9, 1/9 x3, ..., 2 for mode 16)
    V h[19];
    h[0] = vmul(drho, vk<V>(1.0 / 36.0));
    h[1] = vmul(jx, vk<V>(1.0 / 12.0));
    h[2] = vmul(jy, vk<V>(1.0 / 12.0));
    h[3] = vmul(jz, vk<V>(1.0 / 12.0));
    h[4] = vmul(vfma(Ksum, vk<V>(-0.5), vfma(iso, vk<V>(3.0), vsub(trX, drho))), vk<V>(1.0 / 24.0));
    h[5] = vmul(vadd(vfma(Xxx, vk<V>(2.0), vsub(vk<V>(0.0), vadd(Xyy, Xzz))),
                     vfma(Kxx, vk<V>(2.0), vsub(vk<V>(0.0), vadd(Kyy, Kzz)))),
                vk<V>(1.0 / 48.0));
    h[6] = vmul(vadd(vsub(Xyy, Xzz), vsub(Kyy, Kzz)), vk<V>(1.0 / 16.0));
    h[7] = vmul(vfma(kgx, g[1], Xxy), vk<V>(1.0 / 4.0));
    h[8] = vmul(vfma(kgy, g[2], Xyz), vk<V>(1.0 / 4.0));
    h[9] = vmul(vfma(kgz, g[0], Xzx), vk<V>(1.0 / 4.0));
    h[16] = vmul(vfma(Ksum, vk<V>(-1.5), vfma(iso, vk<V>(-3.0), drho)), vk<V>(1.0 / 72.0));

    d3q19_tau1_noise_and_populations<V>(h, f, rho, cs2, P, key, site, status);
}

}  // namespace lbf

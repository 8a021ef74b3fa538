// Row-marching strips of the D2Q9 modified-equilibrium step with two sites
// per lane (FP32, every mode at tau = 1).
//
// A warp owns 64 consecutive sites of a row (tile (system, x0, y0), x0 a
// multiple of 64) and walks YC rows; lane l holds the sites x0 + 2l and
// x0 + 2l + 1 as one float2.  Per footprint row yy each lane loads, for every
// population, the aligned pair of its own two columns at the pulled row
// (one 8-byte load, issued one row ahead); the pull's x shift of -c_x is done in registers: the
// column left of the pair comes from the previous lane by a warp shuffle, the
// column right of it from the next lane.  Lanes 0 and 31 also load the pair
// just outside the strip (columns x0 - 2, x0 - 1 and x0 + 64, x0 + 65) for the
// outermost shifted values and the density of the halo sites x0 - 1 and
// x0 + 64.  The density of the row is then formed for both sites, the
// neighbours' densities come by shuffles, and three density rows stay in
// registers.  With every mode at tau = 1 the post-collision state depends on
// the pre-collision populations only through the density and momentum, so the
// site of row yy - 1 collides from the (drho, j) carried over from the
// previous iteration, two sites at once in paired FP32 (the collision of
// collide_d2q9.cuh), and stores an aligned pair per population.
//
// Every x side is a multiple of 4 (checked on the host), so each pair is
// 8-byte aligned and lies inside one row; lanes past the system's last column
// hold the periodic image of their columns for their neighbours and do not
// collide.  The results are bit-identical to the one-site kernels.
#pragma once

#include "collide_d2q9.cuh"
#include "step_kernels.cuh"

namespace lbf {

// Density deviations of one row around a lane's two sites: l = site x - 1,
// c = (x, x + 1), r = site x + 2.
struct PairRow {
    float l;
    float2 c;
    float r;
};

// 3 x 3 density neighbourhood of the two sites: at<cx, cy, 0>() is the pair
// of densities at (x + cx, y + cy) and (x + 1 + cx, y + cy).
struct PairNbr {
    PairRow m, o, p;    // rows y - 1, y, y + 1
    template <int CX>
    __device__ __forceinline__ static float2 pick(const PairRow& w) {
        if constexpr (CX == -1) return make_float2(w.l, w.c.x);
        else if constexpr (CX == 0) return w.c;
        else return make_float2(w.c.y, w.r);
    }
    template <int CX, int CY, int CZ>
    __device__ __forceinline__ float2 at() const {
        if constexpr (CY == -1) return pick<CX>(m);
        else if constexpr (CY == 0) return pick<CX>(o);
        else return pick<CX>(p);
    }
};

template <int YC, int WPC, int MINB>
__global__ void __launch_bounds__(32 * WPC, MINB)
    step_kernel_strip_pair(const StepArgs<float> A, int n_tiles) {
    using L = D2Q9;
    const int lane = threadIdx.x & 31;
    const int wt = blockIdx.x * WPC + int(threadIdx.x >> 5);
    if (wt >= n_tiles) return;                       // the whole warp leaves together
    const int4 tl = A.tiles[wt];
    // register copies of the per-system records: read once, not again after every row's stores
    const SysDev S = A.sys[tl.x];
    const SysPhys<float> P = A.phys[tl.x];
    const int nx = S.nx, ny = S.ny, N = S.ns;
    const bool sm = S.small != 0;
    const float* __restrict__ fb = A.fin + S.pop_offset;
    float* __restrict__ fo = A.fout + S.pop_offset;
    const int x = tl.y + 2 * lane;
    const bool own = x < nx;
    const bool edge = lane == 0 || lane == 31;
    const bool left = lane == 0;
    const int xs = wrapm(x, nx);                                   // even: the pair is aligned
    const int xt = wrapm(left ? tl.y - 2 : tl.y + 64, nx);         // the pair just outside the strip
    const NoiseKey key = noise_key(S, *A.step_ptr + A.k);
    const int y0 = tl.z, y1 = min(y0 + YC, ny);

    // pulled rows yy - c_y for c_y = -1, 0, 1 (index 1 + c_y), as offsets
    auto rows_of = [&](int yy, int (&ro)[3]) {
        ro[0] = (sm ? wrapm(yy + 1, ny) : wrap2(yy + 1, ny)) * nx;
        ro[1] = (sm ? wrapm(yy, ny) : wrap2(yy, ny)) * nx;
        ro[2] = (sm ? wrapm(yy - 1, ny) : wrap2(yy - 1, ny)) * nx;
    };
    // the loads of row yy + 1 (the lane's pairs and, on lanes 0 and 31, the
    // values outside the strip) are issued before row yy is summed and row
    // yy - 1 collided, so they are in flight across that work.  Outside the
    // strip lane 0 needs columns x0 - 2, x0 - 1 of the populations with
    // c_x = +1 (1, 5, 7) and column x0 - 1 of those with c_x = 0 (0, 3, 4);
    // lane 31 columns x0 + 64, x0 + 65 of those with c_x = -1 (2, 6, 8) and
    // column x0 + 64 of those with c_x = 0.
    float2 sn[9], ewn[3];
    float ezn[3];
    auto load_row = [&](int yy) {
        int ro[3];
        rows_of(yy, ro);
        sfor<0, 9>([&](auto I) {
            constexpr int i = I;
            sn[i] = *reinterpret_cast<const float2*>(fb + i * N + ro[1 + L::c(i, 1)] + xs);
        });
        if (edge) {
            sfor<0, 3>([&](auto K) {
                constexpr int k = K;
                constexpr int ip = k == 0 ? 1 : (k == 1 ? 5 : 7), im = ip + 1;   // c_x = +1 and -1 of group k
                const int i = left ? ip : im;
                const int r = left ? ro[1 + L::c(ip, 1)] : ro[1 + L::c(im, 1)];
                ewn[k] = *reinterpret_cast<const float2*>(fb + i * N + r + xt);
                constexpr int i0 = k == 0 ? 0 : (k == 1 ? 3 : 4);                 // the c_x = 0 populations
                ezn[k] = fb[i0 * N + ro[1 + L::c(i0, 1)] + xt + (left ? 1 : 0)];
            });
        }
    };
    sfor<0, 3>([&](auto K) {
        ewn[decltype(K)::value] = make_float2(0.f, 0.f);
        ezn[decltype(K)::value] = 0.f;
    });
    load_row(y0 - 1);

    float2 pr = make_float2(0.f, 0.f), pjx = pr, pjy = pr;        // (drho, j) of row yy - 1
    PairRow Rm{0.f, pr, 0.f}, R0 = Rm, Rp = Rm;                  // density rows yy - 2, yy - 1, yy
    for (int yy = y0 - 1; yy <= y1; ++yy) {
        float2 s[9], ew[3];
        float ez[3];
        sfor<0, 9>([&](auto I) { s[decltype(I)::value] = sn[decltype(I)::value]; });
        sfor<0, 3>([&](auto K) {
            ew[decltype(K)::value] = ewn[decltype(K)::value];
            ez[decltype(K)::value] = ezn[decltype(K)::value];
        });
        if (yy < y1) load_row(yy + 1);
        // edge lanes: the outermost shifted values e (lane 0: column x0 - 1 of the
        // populations with c_x = +1; lane 31: column x0 + 64 of those with c_x = -1)
        // and the density of the halo site (x0 - 1 or x0 + 64), summed in
        // population order
        float rh = 0.f, e[3] = {0.f, 0.f, 0.f};
        if (edge) {
            float v = 0.f;
            sfor<0, 9>([&](auto I) {
                constexpr int i = I;
                constexpr int cx = L::c(i, 0);
                constexpr int k = (i == 1 || i == 2) ? 0 : ((i == 5 || i == 6) ? 1 : 2);   // x-pair group
                constexpr int m = i == 0 ? 0 : (i == 3 ? 1 : 2);                            // c_x = 0 slot
                float h;
                if constexpr (cx == 1) h = left ? ew[k].x : s[i].y;
                else if constexpr (cx == 0) h = ez[m];
                else h = left ? s[i].x : ew[k].y;
                v = vadd(v, h);
            });
            rh = v;
            sfor<0, 3>([&](auto K) {
                constexpr int k = K;
                e[k] = left ? ew[k].y : ew[k].x;
            });
        }
        // the pull's x shift: f_i(x) = s_i(x - c_x)
        float2 g[9];
        sfor<0, 9>([&](auto I) {
            constexpr int i = I;
            constexpr int cx = L::c(i, 0);
            constexpr int ke = (i == 1 || i == 2) ? 0 : ((i == 5 || i == 6) ? 1 : 2);   // x-pair group
            if constexpr (cx == 0) {
                g[i] = s[i];
            } else if constexpr (cx == 1) {
                float up = __shfl_up_sync(0xffffffffu, s[i].y, 1);
                if (lane == 0) up = e[ke];
                g[i] = make_float2(up, s[i].x);
            } else {
                float dn = __shfl_down_sync(0xffffffffu, s[i].x, 1);
                if (lane == 31) dn = e[ke];
                g[i] = make_float2(s[i].y, dn);
            }
        });
        float2 r, jx, jy;
        moments_d2q9<float2>(g, r, jx, jy);
        float rl = __shfl_up_sync(0xffffffffu, r.y, 1);
        float rr = __shfl_down_sync(0xffffffffu, r.x, 1);
        if (lane == 0) rl = rh;
        if (lane == 31) rr = rh;
        Rm = R0;
        R0 = Rp;
        Rp = PairRow{rl, r, rr};
        if (yy > y0 && own) {
            const int y = yy - 1;
            const PairNbr nb{Rm, R0, Rp};
            const uint32_t site = uint32_t(y * nx + x);
            float2 f[9];
            collide_d2q9_modeq<2, float2>(f, pr, pjx, pjy, nb, P, key, make_uint2(site, site + 1u), A.status);
            sfor<0, 9>([&](auto I) {
                constexpr int i = I;
                *reinterpret_cast<float2*>(fo + i * N + site) = f[i];
            });
        }
        pr = r;
        pjx = jx;
        pjy = jy;
    }
}

}  // namespace lbf

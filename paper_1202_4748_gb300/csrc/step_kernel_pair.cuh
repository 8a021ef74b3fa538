// Warp-specialised z-marching D3Q19 step with two x-adjacent sites per
// consumer thread (fully relaxed Guo path, FP32, every nx a multiple of 4).
//
// Per CTA a TX x TY column of sites walks a chunk of ZC planes.  PW producer
// warps stage each plane into shared-memory rings of R planes:
//   * density deviation on the footprint (columns x0 - 4 .. x0 + TX + 3, rows
//     y0 - 2 .. y0 + TY + 1; y0 - 1 .. y0 + TY for the modified equilibrium,
//     which reads radius 1), from the 19 populations pulled to each footprint
//     site (pull streaming, f_i(r) = f*_i(r - c_i)).  A producer lane owns four
//     consecutive footprint sites: each direction is one aligned 128-bit load
//     of the source row, and the c_x = +-1 directions take the value that
//     crosses the quad boundary from the neighbouring lane by a warp shuffle
//     (quads never straddle the periodic seam because nx is a multiple of 4).
//     Every load of a plane is issued before any is summed, and the loads of
//     plane z + 1 are issued as soon as plane z is summed;
//   * momentum j = sum_i c_i f_i of the tile sites;
//   * Laplacian of the density on the tile + 1, stored twice (at column px and
//     px + 1) so that every stencil pair a consumer needs is one aligned
//     64-bit shared load.
// TX TY / 2 consumer threads collide two sites each from the rings with the
// paired FP32 instructions (collide_d3q19_tau1<float2>) and store both sites
// of every population with one 64-bit store.  The consumers read no global
// memory.  Every per-site sum and product is done in the same order as in the
// one-site kernels, so both give the same bits.
//
// Ring slot of plane z: (z - z0 + 2) mod R.  mbarriers: full[(zl - z0 + 1) mod R]
// completes when every producer has written Laplacian plane zl (and so every
// plane the collision of zl - 1 reads); empty[(zc - z0) mod R] completes when
// every consumer has collided plane zc.  The producers reuse the slots of
// plane zz - R for plane zz only after the collision of zz - R, which also
// frees the Laplacian slot written in the same iteration; each side runs at
// most R - 2 planes ahead, so a phase of one barrier cannot complete twice
// before its waiter looks and the parity of the use count names the phase.
// Every wait is bounded (mbar_wait): a timeout flags the CTA and the status
// word, and every thread keeps the same control flow.
//
// CP = MODEQ runs the modified equilibrium carried to D3Q19
// (collide_d3q19_modeq_tau1), which reads the density within radius 1: the
// footprint has one halo row and a chunk one halo plane on each side
// (density planes z0 - 1 .. z1, ring slot (z - z0 + 1) mod R), no Laplacian
// planes are formed, full[(zc - z0) mod R] completes once density plane
// zc + 1 is written, the consumers read the density of the planes
// zc - 1 .. zc + 1 around their pair, and so the producers reuse the slots of
// plane zz - R + 1 (whose collision no longer reads them) instead of zz - R.
// A producer then writes plane zz only after the collision of zz - R + 1, and
// a consumer collides zc only after density plane zc + 1 is written, so again
// no phase of a barrier completes twice before its waiter looks.
#pragma once

#include "collide_d3q19.cuh"
#include "step_kernels.cuh"

namespace lbf {


// Shared-memory layout of one ring plane (floats): density footprint, the two
// Laplacian copies, momentum pairs.  Row pitches: when a half warp of
// consumers spans two rows (8 pairs per row) they read rows r and r + 2, so a
// pitch of 8 (mod 16) floats keeps the two rows' 64-bit loads on disjoint banks.
// HR: halo rows of the density footprint (2 for the Guo form's gradient of
// the Laplacian, 1 for the modified equilibrium).
template <int TX, int TY, int R, int HR = 2>
struct PairLayout {
    static constexpr int NPR = TX / 2;                 // site pairs per tile row
    static constexpr int SXQ = TX + 8, SY = TY + 2 * HR;  // footprint columns x0 - 4 .. x0 + TX + 3
    static constexpr int NQ = SXQ / 4;                 // producer quads per footprint row
    static constexpr int RPW = 32 / NQ;                // footprint rows per producer warp
    static constexpr int PWN = (SY + RPW - 1) / RPW;   // producer warps needed
    static constexpr int LX = TX + 2, LY = TY + 2;
    static constexpr int pitch(int w) {
        return NPR >= 16 ? (w + 3) / 4 * 4 : (w % 16 <= 8 ? w - w % 16 + 8 : w - w % 16 + 24);
    }
    static constexpr int SXP = pitch(SXQ);            // density row
    static constexpr int LXP = pitch(LX + 1);         // Laplacian row (copy E is shifted by one)
    static constexpr int JRP = NPR >= 16 ? NPR * 6 : pitch(NPR * 6);   // momentum row: 6 floats per pair
    static constexpr int RHO = SY * SXP;
    static constexpr int LAP = LY * LXP;
    static constexpr int JPL = TY * JRP;
    static constexpr int PLANE = RHO + 2 * LAP + JPL; // floats per ring plane
    static constexpr int O_LO = RHO, O_LE = RHO + LAP, O_J = RHO + 2 * LAP;
    static constexpr size_t bytes = size_t(R) * PLANE * sizeof(float);
    static constexpr int NLP = (LX / 2) * LY;         // Laplacian pairs
    static_assert(TX % 16 == 0 && TY % 4 == 0, "tile shape");
    static_assert(SXP % 4 == 0 && PLANE % 4 == 0, "16-byte aligned density quads");
    static_assert(RHO % 2 == 0 && LAP % 2 == 0 && JPL % 2 == 0, "64-bit aligned regions");
};

// Density pairs around a Laplacian pair (lanes at footprint columns fx, fx + 1
// with fx odd; c = footprint row * SXP + fx - 1): the c_x = -1 and +1
// neighbours are the aligned pairs at fx - 1 and fx + 1, and the c_x = 0
// neighbour pair straddles them.
template <int SXP>
struct PairRhoView {
    const float* p[3];      // density planes z - 1, z, z + 1
    int c;
    template <int CX, int CY, int CZ>
    __device__ __forceinline__ float2 at() const {
        if constexpr (CX != 0) {
            return *reinterpret_cast<const float2*>(p[1 + CZ] + c + SXP * CY + 1 + CX);
        } else {
            const float2 m = at<-1, CY, CZ>(), q = at<1, CY, CZ>();
            return make_float2(m.y, q.x);
        }
    }
};

// Density pairs around a consumer pair (sites at footprint columns fx, fx + 1
// with fx even; c = footprint row * SXP + fx): the c_x = 0 neighbour pair is
// the aligned pair at fx, the c_x = -1 and +1 pairs straddle it and its
// aligned neighbours at fx - 2 and fx + 2.
template <int SXP>
struct PairRhoViewEven {
    const float* p[3];      // density planes z - 1, z, z + 1
    int c;
    template <int CX, int CY, int CZ>
    __device__ __forceinline__ float2 at() const {
        const float* q = p[1 + CZ] + c + SXP * CY;
        if constexpr (CX == 0) {
            return *reinterpret_cast<const float2*>(q);
        } else if constexpr (CX == -1) {
            const float2 m = *reinterpret_cast<const float2*>(q - 2), o = *reinterpret_cast<const float2*>(q);
            return make_float2(m.y, o.x);
        } else {
            const float2 o = *reinterpret_cast<const float2*>(q), n = *reinterpret_cast<const float2*>(q + 2);
            return make_float2(o.y, n.x);
        }
    }
};

// Laplacian pairs around a consumer pair (sites at Laplacian columns 2k + 1,
// 2k + 2; c = (row + 1) * LXP + 2k): c_x = 0 from copy E (the value of column
// px sits at px + 1, lap_e floats after copy O), c_x = +-1 from copy O.
template <int LXP>
struct PairLapView {
    const float* o[3];      // copy O of the Laplacian planes z - 1, z, z + 1
    int c;
    int lap_e;
    template <int CX, int CY, int CZ>
    __device__ __forceinline__ float2 at() const {
        if constexpr (CX == 0)
            return *reinterpret_cast<const float2*>(o[1 + CZ] + lap_e + c + LXP * CY + 2);
        else
            return *reinterpret_cast<const float2*>(o[1 + CZ] + c + LXP * CY + 1 + CX);
    }
};

// Register split between the warpgroups, when consumers and producers are
// whole warpgroups of equal size: with register staging the producers'
// batched loads want about twice the registers of the collision, so the
// consumers give up registers (setmaxnreg.dec) and the producers take them
// (setmaxnreg.inc); with cp.async staging it is the other way round.  The
// launch count is the budget of MINB resident CTAs; the host checks that the
// compiled kernel has exactly that many registers before it launches the
// kernel (an increase that the decreases do not cover would wait forever).
template <int TX, int TY, int PW, int MINB, int STG>
struct PairRegs {
    static constexpr int NC = TX * TY / 2, NP = 32 * PW, NT = NC + NP;
    static constexpr int raw = 65536 / (MINB * NT);
    static constexpr int launch = (raw > 255 ? 255 : raw) & ~7;
    // register staging: the consumers keep 80 and the producers take the rest;
    // cp.async staging: the producers hold no loads in registers and need
    // about 48, so the collision takes the rest (112 of 2 x 80 at 3 CTAs per
    // SM: 0.516 -> 0.475 ms on the 160-system ensemble, no spills)
    static constexpr int cons = STG == 3 ? 2 * launch - 48 : 80;
    static constexpr bool split = NC % 128 == 0 && NC == NP && launch != cons && cons <= 256 && 2 * launch - cons >= 24;
    static constexpr int prod = split ? 2 * launch - cons : launch;
    static_assert(!split || (prod <= 256 && prod % 8 == 0 && cons <= 256 && cons % 8 == 0), "register split");
};

// STG: 0 = each producer lane loads its quads into registers (in flight one
// plane ahead); 3 = cp.async copies them into a per-lane staging area in
// shared memory (no registers held by loads in flight), which leaves room
// for more resident CTAs.  (Two staging areas, so that the copies run two
// planes ahead, need 2 CTAs per SM and measured slower.)
template <int TX, int TY, int PW, int R, int STG, int CP = GUO>
struct PairSmem {
    static constexpr size_t stage = STG == 3 ? size_t(19) * 32 * PW * 16 : 0;   // [19][producers] float4
    static constexpr size_t bytes = PairLayout<TX, TY, R, CP == MODEQ ? 1 : 2>::bytes + stage;
};

template <int TX, int TY, int ZC, int PW, int MINB, int R, int STG, int CP = GUO>
__global__ void __launch_bounds__(TX* TY / 2 + 32 * PW, MINB) step_kernel_pair(const StepArgs<float> A) {
    using RG = PairRegs<TX, TY, PW, MINB, STG>;
    using L = D3Q19;
    constexpr int HZ = CP == MODEQ ? 1 : 2;           // halo planes of a chunk
    constexpr int HR = CP == MODEQ ? 1 : 2;           // halo rows of the density footprint
    using LY_ = PairLayout<TX, TY, R, HR>;
    constexpr int NPR = LY_::NPR;
    constexpr int LX2 = LY_::LX / 2;
    constexpr int NC = TX * TY / 2;                   // consumer threads
    constexpr int NP = 32 * PW;                       // producer threads
    constexpr int SXP = LY_::SXP, LXP = LY_::LXP, JRP = LY_::JRP, PLANE = LY_::PLANE;
    static_assert((R & (R - 1)) == 0 && R >= 4, "ring of 2^k >= 4 planes");
    static_assert(NC % 32 == 0, "whole consumer warps");
    extern __shared__ __align__(16) float ring[];
    __shared__ uint64_t full[R], empty[R];
    __shared__ int abort_flag;

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
        abort_flag = 0;
    }
    __syncthreads();
    auto slot = [&](int z) { return (z - z0 + HZ) & (R - 1); };

    if (tid >= NC) {
        // ---------------- producers ----------------
        if constexpr (RG::split && RG::prod > RG::launch) regs_inc<RG::prod>();
        if constexpr (RG::split && RG::prod < RG::launch) regs_dec<RG::prod>();
        const float* __restrict__ fb = A.fin + S.pop_offset;
        const int ptid = tid - NC;
        static_assert(PW >= LY_::PWN, "producer warps cover the footprint rows");
        constexpr int NQ = LY_::NQ, RPW = LY_::RPW;
        // lane -> quad q of footprint row py: sites x0 - 4 + 4q .. + 3
        const int rw = (ptid & 31) / NQ, q = (ptid & 31) % NQ;
        const int py = (ptid >> 5) * RPW + rw;
        const bool act = rw < RPW && py < LY_::SY;
        const bool tile = act && py >= HR && py < HR + TY && q >= 1 && q <= TX / 4;
        const int xq = wrapm(tl.y - 4 + 4 * q, nx);  // first column of the quad (nx % 4 == 0: contiguous)
        const int gy = tl.z - HR + py;
        // source rows y - c_y for c_y = -1, 0, +1
        const float* const rowp[3] = {fb + wrapm(gy + 1, ny) * nx + xq, fb + wrapm(gy, ny) * nx + xq,
                                      fb + wrapm(gy - 1, ny) * nx + xq};
        const int dst = py * SXP + 4 * q;
        const int jdst = LY_::O_J + (py - HR) * JRP + (q - 1) * 12;   // pairs 2(q - 1), 2(q - 1) + 1
        const int pl = nx * ny;
        const bool sm = S.small != 0;
        // the loads of plane zz + 1 are issued as soon as plane zz has been
        // summed (staged by cp.async: direction by direction, each right after
        // the staged value it overwrites has been read back and used), so they
        // are in flight across the sums, the barrier and the Laplacian
        constexpr bool CPA = STG == 3;                   // staged by cp.async
        float4 g[CPA ? 1 : 19];
        float4* const stage = reinterpret_cast<float4*>(ring + R * PLANE) + ptid;   // [19][NP], this lane's column
        if constexpr (!CPA)
            sfor<0, 19>([&](auto I) { g[decltype(I)::value] = make_float4(0.0f, 0.0f, 0.0f, 0.0f); });
        // source planes z - c_z for c_z = -1, 0, +1 of plane zz
        auto planes_of = [&](int zz, int (&zo)[3]) {
            zo[0] = (sm ? wrapm(zz + 1, nz) : wrap2(zz + 1, nz)) * pl;
            zo[1] = (sm ? wrapm(zz, nz) : wrap2(zz, nz)) * pl;
            zo[2] = (sm ? wrapm(zz - 1, nz) : wrap2(zz - 1, nz)) * pl;
        };
        auto pull = [&](int zz) {
            int zo[3];
            planes_of(zz, zo);
            if (act) {
                sfor<0, 19>([&](auto I) {
                    constexpr int i = I;
                    constexpr int cy = L::c(i, 1), cz = L::c(i, 2);
                    const float* src = rowp[1 + cy] + (i * N + zo[1 + cz]);
                    if constexpr (CPA) cp_async16(stage + i * NP, src);
                    else g[i] = *reinterpret_cast<const float4*>(src);
                });
            }
            if constexpr (CPA) cp_async_commit();
        };
        auto pulled = [&](auto I) -> float4 {
            if constexpr (CPA) return stage[decltype(I)::value * NP];
            else return g[decltype(I)::value];
        };
        pull(z0 - HZ);
        for (int zz = z0 - HZ; zz < z1 + HZ; ++zz) {
            // plane whose slots this iteration reuses: the modified equilibrium's
            // consumers read the density of the planes on both sides of the one
            // they collide, so its producers also wait for the plane after it
            const int zw = zz - R + (CP == MODEQ ? 1 : 0);
            if (zw >= z0) mbar_wait(&empty[(zw - z0) & (R - 1)], unsigned(((zw - z0) / R) & 1), &abort_flag, A.status);
            float* const rp = ring + slot(zz) * PLANE;
            // per direction, the pulled values of the quad's four sites: the
            // c_x = +1 (-1) direction pulls x - 1 (x + 1), one of which lives in
            // the neighbouring lane.  Density and momentum are summed in the
            // order of the one-site kernels (from 0, direction by direction).
            if constexpr (CPA) cp_async_wait_all();      // this lane's copies of plane zz have landed
            const bool more = zz + 1 < z1 + HZ;
            int zn[3];
            planes_of(zz + 1, zn);
            float2 r01 = make_float2(0.0f, 0.0f), r23 = r01;
            float2 j01[3] = {r01, r01, r01}, j23[3] = {r01, r01, r01};
            sfor<0, 19>([&](auto I) {
                constexpr int i = I;
                constexpr int cx = L::c(i, 0);
                const float4 v = pulled(I);
                float2 a01, a23;
                if constexpr (cx == 0) {
                    a01 = make_float2(v.x, v.y);
                    a23 = make_float2(v.z, v.w);
                } else if constexpr (cx == 1) {
                    const float pw = __shfl_up_sync(0xffffffffu, v.w, 1);
                    a01 = make_float2(pw, v.x);
                    a23 = make_float2(v.y, v.z);
                } else {
                    const float nw = __shfl_down_sync(0xffffffffu, v.x, 1);
                    a01 = make_float2(v.y, v.z);
                    a23 = make_float2(v.w, nw);
                }
                r01 = vadd(r01, a01);
                r23 = vadd(r23, a23);
                if constexpr (CPA) {
                    // v has been used, so the read of this staged slot is complete
                    constexpr int cy = L::c(i, 1), cz = L::c(i, 2);
                    if (more && act) cp_async16(stage + i * NP, rowp[1 + cy] + (i * N + zn[1 + cz]));
                }
                if constexpr (i > 0) {
                    if (tile) {
                        sfor<0, 3>([&](auto C) {
                            constexpr int c = C;
                            if constexpr (L::c(i, c) == 1) {
                                j01[c] = vadd(j01[c], a01);
                                j23[c] = vadd(j23[c], a23);
                            }
                            if constexpr (L::c(i, c) == -1) {
                                j01[c] = vsub(j01[c], a01);
                                j23[c] = vsub(j23[c], a23);
                            }
                        });
                    }
                }
            });
            if (act) *reinterpret_cast<float4*>(rp + dst) = make_float4(r01.x, r01.y, r23.x, r23.y);
            if (tile) {
                sfor<0, 3>([&](auto C) {
                    constexpr int c = C;
                    *reinterpret_cast<float2*>(rp + jdst + 2 * c) = j01[c];
                    *reinterpret_cast<float2*>(rp + jdst + 6 + 2 * c) = j23[c];
                });
            }
            if constexpr (CPA) {
                if (more) cp_async_commit();
            } else {
                if (more) pull(zz + 1);
            }
            named_barrier(1, NP);                        // density plane zz complete (producers)
            if constexpr (CP == MODEQ) {
                // no Laplacian planes: density planes up to zz are complete, all
                // that the collision of zz - 1 reads
                if (zz >= z0 + 1) mbar_arrive(&full[(zz - z0 - 1) & (R - 1)]);
            } else if (zz >= z0) {
                const int zl = zz - 1;                   // Laplacian plane (needs density zl-1 .. zl+1)
                PairRhoView<SXP> rv{{ring + slot(zl - 1) * PLANE, ring + slot(zl) * PLANE, ring + slot(zl + 1) * PLANE},
                                    0};
                float* lo = ring + slot(zl) * PLANE + LY_::O_LO;
                float* le = ring + slot(zl) * PLANE + LY_::O_LE;
                for (int lq = ptid; lq < LY_::NLP; lq += NP) {
                    // with 16 pairs per tile row a half warp takes one Laplacian row
                    // (conflict-free 64-bit shared loads) and the last pair of every
                    // row comes after all rows
                    int lpx, lpy;
                    if constexpr (NPR == 16) {
                        constexpr int MAIN = 16 * LY_::LY;
                        lpy = lq < MAIN ? lq >> 4 : lq - MAIN;
                        lpx = lq < MAIN ? 2 * (lq & 15) : 32;
                    } else {
                        lpx = 2 * (lq % LX2);
                        lpy = lq / LX2;
                    }
                    // Laplacian column lpx <-> footprint column lpx + 3, row lpy <-> lpy + HR - 1
                    rv.c = (lpy + HR - 1) * SXP + lpx + 2;
                    const float2 lap = lap_d3q19<float2>(rv);
                    *reinterpret_cast<float2*>(lo + lpy * LXP + lpx) = lap;
                    le[lpy * LXP + lpx + 1] = lap.x;
                    le[lpy * LXP + lpx + 2] = lap.y;
                }
                mbar_arrive(&full[(zl - z0 + 1) & (R - 1)]);
            }
        }
    } else {
        // ---------------- consumers ----------------
        if constexpr (RG::split && RG::cons < RG::launch) regs_dec<RG::cons>();
        if constexpr (RG::split && RG::cons > RG::launch) regs_inc<RG::cons>();
        float* __restrict__ fo = A.fout + S.pop_offset;
        const int64_t step = *A.step_ptr + A.k;
        const SysPhys<float> P = A.phys[tl.x];
        const NoiseKey key = noise_key(S, step);
        const int w = tid >> 5, l = tid & 31;
        int pk, ty;
        if constexpr (NPR >= 16) {
            pk = tid % NPR;
            ty = tid / NPR;
        } else {
            static_assert(NPR == 8, "8 or >= 16 pairs per row");
            pk = l & 7;
            const int q = l >> 3;                        // half warp 0: rows 0 and 2; half warp 1: rows 1 and 3
            ty = 4 * w + (q == 1 ? 2 : (q == 2 ? 1 : q));
        }
        const int x = tl.y + 2 * pk, y = tl.z + ty;
        const bool valid = x < nx && y < ny;
        const int rho_off = (ty + HR) * SXP + 2 * pk + 4;
        const int j_off = LY_::O_J + ty * JRP + pk * 6;
        const int lap_c = (ty + 1) * LXP + 2 * pk;
        for (int zc = z0; zc < z1; ++zc) {
            // the hand-off of the last plane the collision reads: Laplacian plane
            // zc + 1 (full[zc - z0 + 2]), or density plane zc + 1 (full[zc - z0])
            const int kf = zc - z0 + (CP == MODEQ ? 0 : 2);
            const bool ok = mbar_wait(&full[kf & (R - 1)], unsigned((kf / R) & 1),
                                      &abort_flag, A.status);
            if (valid && ok) {
                const float* cp = ring + slot(zc) * PLANE;
                const float2 drho = *reinterpret_cast<const float2*>(cp + rho_off);
                const float2 jx = *reinterpret_cast<const float2*>(cp + j_off);
                const float2 jy = *reinterpret_cast<const float2*>(cp + j_off + 2);
                const float2 jz = *reinterpret_cast<const float2*>(cp + j_off + 4);
                const int site = site_index(x, y, zc, nx, ny);
                float2 f[19];
                if constexpr (CP == MODEQ) {
                    const PairRhoViewEven<SXP> rv{{ring + slot(zc - 1) * PLANE, cp, ring + slot(zc + 1) * PLANE},
                                                  rho_off};
                    collide_d3q19_modeq_tau1<float2>(f, drho, jx, jy, jz, rv, P, key, make_uint2(site, site + 1),
                                                     A.status);
                } else {
                    PairLapView<LXP> lv;
                    lv.o[0] = ring + slot(zc - 1) * PLANE + LY_::O_LO;
                    lv.o[1] = cp + LY_::O_LO;
                    lv.o[2] = ring + slot(zc + 1) * PLANE + LY_::O_LO;
                    lv.c = lap_c;
                    lv.lap_e = LY_::LAP;
                    collide_d3q19_tau1<float2>(f, drho, jx, jy, jz, lv, P, key, make_uint2(site, site + 1), A.status);
                }
                sfor<0, 19>([&](auto I) {
                    constexpr int i = I;
                    *reinterpret_cast<float2*>(fo + (i * N + site)) = f[i];
                });
            }
            mbar_arrive(&empty[(zc - z0) & (R - 1)]);
        }
    }
}

}  // namespace lbf

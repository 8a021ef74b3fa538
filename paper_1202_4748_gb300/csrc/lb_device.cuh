// Device-side building blocks of the fluctuating lattice Boltzmann library:
// velocity sets, moment bases, the Philox4x32-10 counter-based generator and
// per-system parameters.  Written for sm_103a; everything is header-only and
// templated so that each (lattice, coupling, precision) instantiation folds
// its constant tables at compile time.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace lbf {

constexpr int LB_MAX_Q_DEV = 19;

// Compile-time loop: f(std::integral_constant<int, k>) for k = B .. E-1, so
// that table entries indexed by k are constant expressions (folded by the
// C++ front end, not by the optimiser).
template <int B, int E, class F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(static_cast<F&&>(f));
    }
}

// ---------------------------------------------------------------------------
// Velocity sets and moment bases
// ---------------------------------------------------------------------------
// D2Q9 (the paper's lattice, Sec. III A).  Rest velocity first, then the axis
// pairs and the diagonal pairs (1,1)/(-1,-1) and (1,-1)/(-1,1) -- the order in
// which the printed weights of Eq. 65 (w^xy = +1/4 on the 5th/6th, -1/4 on the
// 7th/8th velocity) place them.
//
// Moment basis (Eq. 66 expands f_i = T_ai t_i m_a / N_a): rows
//   1, cx, cy, 3c^2-2, cx^2-cy^2, cx cy, (3c^2-4)cx, (3c^2-4)cy, 9c^4-15c^2+2
// whose squared lengths N = (1, 1/3, 1/3, 4, 4/9, 1/9, 2/3, 2/3, 16) are the
// diagonal of Eq. 68 at c_s^2 = 1/3.
struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    static constexpr int NC = 3;        // conserved moments: rho, jx, jy
    static constexpr int PP = 3;        // the two non-conserved modes with a rest-
    static constexpr int PR = 8;        // velocity component (coupled in Eq. 68)
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int v[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                 {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
        return v[i][a];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int T(int a, int i) {
        const int x = c(i, 0), y = c(i, 1), c2 = x * x + y * y;
        switch (a) {
            case 0: return 1;
            case 1: return x;
            case 2: return y;
            case 3: return 3 * c2 - 2;
            case 4: return x * x - y * y;
            case 5: return x * y;
            case 6: return (3 * c2 - 4) * x;
            case 7: return (3 * c2 - 4) * y;
            default: return 9 * c2 * c2 - 15 * c2 + 2;
        }
    }
};

// D3Q19 (3-D variant): rest, 6 face and 12 edge velocities, weights 1/3,
// 1/18, 1/36, and an orthogonal polynomial basis: rho, j, six second-order
// stresses (c^2-1, 3cx^2-c^2, cy^2-cz^2, cx cy, cy cz, cz cx), nine ghosts
// ((3c^2-5)c_a, (cy^2-cz^2)cx, (cz^2-cx^2)cy, (cx^2-cy^2)cz, 3c^4-6c^2+1,
// (2c^2-3)(3cx^2-c^2), (2c^2-3)(cy^2-cz^2)).
struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    static constexpr int NC = 4;
    static constexpr int PP = 4;
    static constexpr int PR = 16;
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int v[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
        return v[i][a];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int T(int a, int i) {
        const int x = c(i, 0), y = c(i, 1), z = c(i, 2);
        const int c2 = x * x + y * y + z * z;
        switch (a) {
            case 0: return 1;
            case 1: return x;
            case 2: return y;
            case 3: return z;
            case 4: return c2 - 1;
            case 5: return 3 * x * x - c2;
            case 6: return y * y - z * z;
            case 7: return x * y;
            case 8: return y * z;
            case 9: return z * x;
            case 10: return (3 * c2 - 5) * x;
            case 11: return (3 * c2 - 5) * y;
            case 12: return (3 * c2 - 5) * z;
            case 13: return (y * y - z * z) * x;
            case 14: return (z * z - x * x) * y;
            case 15: return (x * x - y * y) * z;
            case 16: return 3 * c2 * c2 - 6 * c2 + 1;
            case 17: return (2 * c2 - 3) * (3 * x * x - c2);
            default: return (2 * c2 - 3) * (y * y - z * z);
        }
    }
};

// Squared length N_a = sum_i t_i T_ai^2 and inverse-transform coefficients.
template <class L>
__host__ __device__ constexpr double norm2(int a) {
    double s = 0.0;
    for (int i = 0; i < L::Q; ++i) s += L::w(i) * double(L::T(a, i)) * double(L::T(a, i));
    return s;
}
template <class L>
__host__ __device__ constexpr double tinv(int i, int a) {
    return L::w(i) * double(L::T(a, i)) / norm2<L>(a);
}

// M_a,bc = sum_i t_i T_ai c_ib c_ic: second-moment projection of mode a.
template <class L>
__host__ __device__ constexpr double mproj(int a, int b, int c) {
    double s = 0.0;
    for (int i = 0; i < L::Q; ++i) s += L::w(i) * double(L::T(a, i)) * L::c(i, b) * L::c(i, c);
    return s;
}
// Parity of mode a under c -> -c (+1 even, -1 odd), read off the basis.
template <class L>
__host__ __device__ constexpr int mode_parity(int a) {
    for (int i = 1; i < L::Q; ++i)
        if (L::T(a, i) != 0) return L::T(a, i) == L::T(a, i + ((i & 1) ? 1 : -1)) ? 1 : -1;
    return 1;
}

enum Coupling { MODEQ = 0, GUO = 1 };

// Modified-equilibrium weights of Eq. 65 (D2Q9 order above; index 0 unused).
__host__ __device__ constexpr double pooley_w(int i) { return i == 0 ? 0.0 : (i < 5 ? 1.0 / 3.0 : 1.0 / 12.0); }
__host__ __device__ constexpr double pooley_wxx(int i) {
    return i == 0 ? 0.0 : (i < 3 ? 1.0 / 3.0 : (i < 5 ? -1.0 / 6.0 : -1.0 / 24.0));
}
__host__ __device__ constexpr double pooley_wyy(int i) {
    return i == 0 ? 0.0 : (i < 3 ? -1.0 / 6.0 : (i < 5 ? 1.0 / 3.0 : -1.0 / 24.0));
}
__host__ __device__ constexpr double pooley_wxy(int i) {
    return i < 5 ? 0.0 : (i < 7 ? 0.25 : -0.25);
}

// ---------------------------------------------------------------------------
// Per-system parameters, resident in the workspace
// ---------------------------------------------------------------------------
struct SysDev {
    int32_t nx, ny, nz;
    int32_t small;          // 1 if some side is shorter than 3 (the footprint wrap needs a modulo)
    int32_t ns;             // n_sites as 32 bit (q * n_sites < 2^31 is checked on the host)
    int32_t pad0;
    int64_t n_sites;
    int64_t site_offset;    // first site of this system in the concatenated site arrays
    int64_t pop_offset;     // first population element: pop_offset + i * n_sites + site
    double rho_c, a, b, kappa, kT;
    double inv_rho_c;
    double nu;              // kinematic viscosity of the Holdych term (tau[4])
    double lam[LB_MAX_Q_DEV];
    double g_diag[LB_MAX_Q_DEV];   // 1 - gamma_a^2
    double g_pair;                 // 1 - gamma_P gamma_R
    double namp[LB_MAX_Q_DEV];     // sqrt(N_a (1 - gamma_a^2)): amplitude of an uncoupled mode
    uint32_t seed_lo, seed_hi;
    uint32_t system_id;
    int32_t bgk;                   // 1: every non-conserved mode relaxes at the same rate lam_bgk
    double lam_bgk;
};

// Physical parameters of a system in the arithmetic precision of the step
// kernel (converted once on the host, so the FP32 kernel issues no FP64
// conversions per site).
template <class Real>
struct SysPhys {
    Real rho_c, inv_rho_c, a, b, kappa, kT, nu, lam_bgk, g_pair, pad;
    Real lam[LB_MAX_Q_DEV];
    Real g_diag[LB_MAX_Q_DEV];
    Real namp[LB_MAX_Q_DEV];
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): round multipliers M0, M1
// and key increments W0, W1
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        // one 32 x 32 -> 64-bit product per multiplier (high and low words together)
        const uint64_t pa = uint64_t(kPhiloxM0) * ctr.x;
        const uint64_t pb = uint64_t(kPhiloxM1) * ctr.z;
        ctr = make_uint4(uint32_t(pb >> 32) ^ ctr.y ^ k0, uint32_t(pb), uint32_t(pa >> 32) ^ ctr.w ^ k1,
                         uint32_t(pa));
    }
    return ctr;
}

// Counter layout: (site, step low word, step high word, system_id << 8 | draw).
__device__ __forceinline__ uint4 site_draw(const SysDev& s, uint32_t site, int64_t step, uint32_t draw) {
    const uint4 ctr = make_uint4(site, uint32_t(uint64_t(step) & 0xffffffffu), uint32_t(uint64_t(step) >> 32),
                                 (s.system_id << 8) | draw);
    return philox4x32_10(ctr, s.seed_lo, s.seed_hi);
}

// Uniform in (0,1): (x + 1/2) 2^-32, then Box-Muller (R = sqrt(-2 ln U_a),
// angle 2 pi U_b).  Float and double versions.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, double& n0, double& n1) {
    const double ua = (double(wa) + 0.5) * 2.3283064365386962890625e-10;
    const double ub = (double(wb) + 0.5) * 2.3283064365386962890625e-10;
    const double r = sqrt(-2.0 * log(ua));
    double s, c;
    sincospi(2.0 * ub, &s, &c);
    n0 = r * c;
    n1 = r * s;
}
// FP32 variant on the special-function unit: -2 ln U = -2 ln2 log2 U, clamped
// at a tiny positive value because log2 of U within an ulp of 1 may come out
// slightly positive, and its square root taken as x rsqrt(x) (a few ulp; the
// IEEE-rounded square root costs several more instructions); the angle is
// taken as 2 pi (U_b - 1/2) in [-pi, pi), where the hardware sine/cosine are
// accurate, and the half turn is undone by the sign flips.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& n0, float& n1) {
    const float ua = fmaf(float(wa), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float ub = fmaf(float(wb), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float r2 = fmaxf(-1.3862943611198906f * __log2f(ua), 1e-30f);
    const float r = r2 * rsqrtf(r2);
    float s, c;
    __sincosf(6.2831853071795865f * (ub - 0.5f), &s, &c);
    n0 = -r * c;
    n1 = -r * s;
}

// Reciprocal and reciprocal square root: exact-rounding library calls in
// double, the special-function unit in float (the FP32 path's error budget is
// ~1e-5 of the populations; these are good to a few ulp).
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float fast_rsqrt(float x) { return rsqrtf(x); }
// Square root of x >= 0: exact rounding in double; x rsqrt(x) in float (0 at 0).
__device__ __forceinline__ double fast_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// Periodic wrap of a coordinate in [-n, 2n).
__device__ __forceinline__ int wrap2(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }
// Periodic wrap of a coordinate that is at most one period outside [0, n).
__device__ __forceinline__ int wrap1(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }
// Any coordinate.
__device__ __forceinline__ int wrapm(int x, int n) {
    int r = x % n;
    return r < 0 ? r + n : r;
}

// Device status bits (OR-ed by kernels, mapped to lb_status on the host).
enum : int { ST_RHO = 1, ST_NOISE = 2, ST_NONFINITE = 4, ST_TIMEOUT = 8 };

// ---- mbarrier (shared-memory arrival barrier) helpers ----------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
// arrive (release semantics at CTA scope: the caller's earlier shared-memory
// accesses are ordered before the phase can complete)
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b))
                 : "memory");
}
// Wait (acquire semantics) for the completion of the phase with this parity;
// the thread may be suspended in hardware for up to about suspend_ns before the
// call returns false, so a waiting warp issues almost nothing.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity, unsigned suspend_ns) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(suspend_ns)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: gives up after about 0.3 s of wall time (global timer; also
// after 2^20 attempts), or at once when *abort is set, sets *abort and the
// status bit, and returns false; control flow then continues (results are
// flagged invalid), so no thread hangs.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, volatile int* abort, int* status) {
    if (mbar_try_wait(b, parity, 10000u)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 0; i < (1 << 20); ++i) {
        if (mbar_try_wait(b, parity, 10000u)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > 300000000ull) break;
    }
    *abort = 1;
    atomicOr(status, ST_TIMEOUT);
    return false;
}

// Bulk copies into shared memory (cp.async.bulk, no tensor map): the mbarrier
// phase completes when its arrivals are in and the expected bytes have landed.
// Both addresses and the size must be multiples of 16 bytes.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(b))
        : "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same locations.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Bounded wait for bulk copies: like mbar_wait, but it does not give up when
// the abort flag is set, so a CTA never exits with its own copies in flight
// (they read valid addresses and always complete; the limit only guards
// against a fault elsewhere).
__device__ __forceinline__ bool mbar_wait_copies(uint64_t* b, unsigned parity, volatile int* abort, int* status) {
    if (mbar_try_wait(b, parity, 10000u)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 0; i < (1 << 20); ++i) {
        if (mbar_try_wait(b, parity, 10000u)) return true;
        if (global_ns() - t0 > 300000000ull) break;
    }
    *abort = 1;
    atomicOr(status, ST_TIMEOUT);
    return false;
}

// Register reallocation between warpgroups (sm_90a and later): the calling
// warpgroup's per-thread register count becomes N (a multiple of 8 in
// [24, 256]).  An increase waits for registers that other warpgroups of the
// CTA released, so the decreases and increases of one CTA must balance
// against the registers it was launched with.
template <int N>
__device__ __forceinline__ void regs_dec() {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(N));
}
template <int N>
__device__ __forceinline__ void regs_inc() {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(N));
}

// 16-byte asynchronous copy global -> shared (cp.async, cached in L2 only),
// completed for the issuing thread by cp_async_wait_all.  Both addresses must
// be 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Named barrier over `count` threads (a multiple of 32) of the CTA.
__device__ __forceinline__ void named_barrier(int id, int count) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

}  // namespace lbf

// Shared body of the per-lattice translation units: tile-shape table and the
// launchers for the step, init, gather/scatter and observable-site kernels.
#pragma once

#include "lattice_kernels.cuh"
#include "lb_launch.h"
#include "step_kernel_modeq3.cuh"
#include "step_kernel_pair.cuh"
#include "step_kernel_strip_pair.cuh"
#include "step_kernels.cuh"

namespace lbf {

template <class L, int CP, class Real, int TX, int TY, int TZ, int MODE>
cudaError_t step_one_mode(const StepLaunch& a, cudaStream_t st) {
    StepArgs<Real> A;
    A.sys = a.sys;
    A.phys = static_cast<const SysPhys<Real>*>(a.phys);
    A.tiles = a.tiles;
    A.fin = static_cast<const Real*>(a.fin);
    A.fout = static_cast<Real*>(a.fout);
    A.step_ptr = a.step_ptr;
    A.k = a.k;
    A.status = a.status;
    step_kernel<L, CP, Real, TX, TY, TZ, MODE><<<a.n_tiles, TX * TY * TZ, 0, st>>>(A);
    return cudaGetLastError();
}

// Row-marching strips (D2Q9, modified equilibrium): WPC warps per CTA, tiles
// of SW sites x YC rows, one warp per 32 sites of a tile.
template <class L, int CP, class Real, int YC, int WPC, int MINB, int MODE, int SW>
cudaError_t step_strip_mode(const StepLaunch& a, cudaStream_t st) {
    StepArgs<Real> A;
    A.sys = a.sys;
    A.phys = static_cast<const SysPhys<Real>*>(a.phys);
    A.tiles = a.tiles;
    A.fin = static_cast<const Real*>(a.fin);
    A.fout = static_cast<Real*>(a.fout);
    A.step_ptr = a.step_ptr;
    A.k = a.k;
    A.status = a.status;
    const int warps = a.n_tiles * (SW / 32);
    const int grid = (warps + WPC - 1) / WPC;
    step_kernel_strip<L, CP, Real, YC, WPC, MINB, MODE, SW><<<grid, 32 * WPC, 0, st>>>(A, a.n_tiles);
    return cudaGetLastError();
}
template <class L, int CP, class Real, int YC, int WPC, int MINB, int SW = 32>
cudaError_t step_strip(const StepLaunch& a, cudaStream_t st) {
    constexpr int MB = sizeof(Real) == 4 && MINB > 0 ? MINB : 1;   // FP64 keeps its registers
    if (a.bgk_only == 2) return step_strip_mode<L, CP, Real, YC, WPC, MB, 2, SW>(a, st);
    if (a.bgk_only == 1) return step_strip_mode<L, CP, Real, YC, WPC, MB, 1, SW>(a, st);
    return step_strip_mode<L, CP, Real, YC, WPC, MB, 0, SW>(a, st);
}

// Two-site strips (D2Q9, modified equilibrium, FP32, every mode at tau = 1,
// every x side a multiple of 4) on tiles of 64 sites x YC rows; any other run
// of the same tiles takes the one-site strips, two warps per tile.
template <class L, int CP, class Real, int YC, int WPC, int MINB>
cudaError_t step_strip2(const StepLaunch& a, cudaStream_t st) {
    if constexpr (sizeof(Real) == 4 && CP == MODEQ) {
        if (a.bgk_only == 2 && a.pair_ok) {
            StepArgs<float> A;
            A.sys = a.sys;
            A.phys = static_cast<const SysPhys<float>*>(a.phys);
            A.tiles = a.tiles;
            A.fin = static_cast<const float*>(a.fin);
            A.fout = static_cast<float*>(a.fout);
            A.step_ptr = a.step_ptr;
            A.k = a.k;
            A.status = a.status;
            const int grid = (a.n_tiles + WPC - 1) / WPC;
            step_kernel_strip_pair<YC, WPC, MINB><<<grid, 32 * WPC, 0, st>>>(A, a.n_tiles);
            return cudaGetLastError();
        }
    }
    return step_strip<L, CP, Real, YC, WPC, MINB, 64>(a, st);
}

template <class L, int CP, class Real, int TX, int TY, int ZC, int MINB, int MODE>
cudaError_t step_z_mode(const StepLaunch& a, cudaStream_t st) {
    StepArgs<Real> A;
    A.sys = a.sys;
    A.phys = static_cast<const SysPhys<Real>*>(a.phys);
    A.tiles = a.tiles;
    A.fin = static_cast<const Real*>(a.fin);
    A.fout = static_cast<Real*>(a.fout);
    A.step_ptr = a.step_ptr;
    A.k = a.k;
    A.status = a.status;
    step_kernel_z<L, CP, Real, TX, TY, ZC, MINB, MODE><<<a.n_tiles, TX * TY, 0, st>>>(A);
    return cudaGetLastError();
}

// z-marching launch: tile = (TX, TY, z-chunk), register budget for MINB resident
// CTAs per SM (the FP64 instances use the natural register count).
template <class L, int CP, class Real, int TX, int TY, int ZC, int MINB>
cudaError_t step_z(const StepLaunch& a, cudaStream_t st) {
    constexpr int MB = sizeof(Real) == 4 ? MINB : 1;
    if (a.bgk_only == 2) return step_z_mode<L, CP, Real, TX, TY, ZC, MB, 2>(a, st);
    if (a.bgk_only == 1) return step_z_mode<L, CP, Real, TX, TY, ZC, MB, 1>(a, st);
    return step_z_mode<L, CP, Real, TX, TY, ZC, MB, 0>(a, st);
}

// z-marching launch of the D3Q19 modified equilibrium (density footprint of
// radius 1); the FP64 instances use the natural register count.
template <class L, class Real, int TX, int TY, int ZC, int MINB, int MODE>
cudaError_t step_zm_mode(const StepLaunch& a, cudaStream_t st) {
    StepArgs<Real> A;
    A.sys = a.sys;
    A.phys = static_cast<const SysPhys<Real>*>(a.phys);
    A.tiles = a.tiles;
    A.fin = static_cast<const Real*>(a.fin);
    A.fout = static_cast<Real*>(a.fout);
    A.step_ptr = a.step_ptr;
    A.k = a.k;
    A.status = a.status;
    step_kernel_zm<L, Real, TX, TY, ZC, MINB, MODE><<<a.n_tiles, TX * TY, 0, st>>>(A);
    return cudaGetLastError();
}
template <class L, class Real, int TX, int TY, int ZC, int MINB>
cudaError_t step_zm(const StepLaunch& a, cudaStream_t st) {
    constexpr int MB = sizeof(Real) == 4 ? (MINB < 2 ? 2 : MINB) : 1;
    if (a.bgk_only == 2) return step_zm_mode<L, Real, TX, TY, ZC, MB, 2>(a, st);
    if (a.bgk_only == 1) return step_zm_mode<L, Real, TX, TY, ZC, MB, 1>(a, st);
    return step_zm_mode<L, Real, TX, TY, ZC, MB, 0>(a, st);
}

// Warp-specialised launch (fully relaxed Guo path, FP32): TX x TY consumer
// threads and PW producer warps per CTA; STG = 1 stages the footprint with
// bulk copies (a dynamic shared-memory stage), 0 with plain loads.
template <class L, int TX, int TY, int ZC, int PW, int MINB, int STG>
cudaError_t step_ws(const StepLaunch& a, cudaStream_t st) {
    StepArgs<float> A;
    A.sys = a.sys;
    A.phys = static_cast<const SysPhys<float>*>(a.phys);
    A.tiles = a.tiles;
    A.fin = static_cast<const float*>(a.fin);
    A.fout = static_cast<float*>(a.fout);
    A.step_ptr = a.step_ptr;
    A.k = a.k;
    A.status = a.status;
    size_t dyn = 0;
    if constexpr (STG == 1) {
        dyn = BulkStage<L, TX, TY, ZC, PW>::bytes;
        static bool attr = false;              // once per instantiation
        if (!attr) {
            auto k = step_kernel_ws<L, TX, TY, ZC, PW, MINB, STG>;
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         int(cudaSharedmemCarveoutMaxShared));
            if (e != cudaSuccess) return e;
            attr = true;
        }
    }
    step_kernel_ws<L, TX, TY, ZC, PW, MINB, STG><<<a.n_tiles, TX * TY + 32 * PW, dyn, st>>>(A);
    return cudaGetLastError();
}

// Paired-site warp-specialised launch (fully relaxed path on D3Q19, FP32,
// every nx a multiple of 4; the Guo form, or CP = MODEQ the modified
// equilibrium): TX TY / 2 consumer threads and PW producer warps
// per CTA, rings of R planes (and, STG = 3, the producers' staging area) in
// dynamic shared memory.
template <int TX, int TY, int ZC, int PW, int MINB, int R, int STG, int CP = GUO>
cudaError_t step_pair(const StepLaunch& a, cudaStream_t st) {
    StepArgs<float> A;
    A.sys = a.sys;
    A.phys = static_cast<const SysPhys<float>*>(a.phys);
    A.tiles = a.tiles;
    A.fin = static_cast<const float*>(a.fin);
    A.fout = static_cast<float*>(a.fout);
    A.step_ptr = a.step_ptr;
    A.k = a.k;
    A.status = a.status;
    constexpr size_t dyn = PairSmem<TX, TY, PW, R, STG, CP>::bytes;
    static int state = 0;                      // once per instantiation: 1 usable, -1 not
    if (state == 0) {
        auto k = step_kernel_pair<TX, TY, ZC, PW, MINB, R, STG, CP>;
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
        // (no carve-out preference: the rings need a fraction of the SM's
        // shared memory, and the producers' load misses are staged in L1)
        if (e != cudaSuccess) return e;
        // the register split must balance against the launch count it assumes
        state = (!PairRegs<TX, TY, PW, MINB, STG>::split || fa.numRegs == PairRegs<TX, TY, PW, MINB, STG>::launch) ? 1 : -1;
    }
    if (state < 0) {
        if constexpr (CP == MODEQ) return step_zm<D3Q19, float, TX, TY, ZC, MINB>(a, st);
        else return step_ws<D3Q19, TX, TY, ZC, PW, 1, 0>(a, st);
    }
    step_kernel_pair<TX, TY, ZC, PW, MINB, R, STG, CP><<<a.n_tiles, TX * TY / 2 + 32 * PW, dyn, st>>>(A);
    return cudaGetLastError();
}

template <class L, int CP, class Real, int TX, int TY, int TZ>
cudaError_t step_one(const StepLaunch& a, cudaStream_t st) {
    if (a.bgk_only == 2) return step_one_mode<L, CP, Real, TX, TY, TZ, 2>(a, st);
    if (a.bgk_only == 1) return step_one_mode<L, CP, Real, TX, TY, TZ, 1>(a, st);
    return step_one_mode<L, CP, Real, TX, TY, TZ, 0>(a, st);
}

template <class L, class Real>
cudaError_t init_feq_any(int coupling, const SysDev* sys, const int4* items, int n_items, const double* d,
                         const double* dbar, void* fbuf, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    if (coupling == MODEQ) {
        init_feq_kernel<L, MODEQ, Real><<<n_items, AUX_THREADS, 0, st>>>(sys, items, d, dbar, static_cast<Real*>(fbuf));
    } else {
        init_feq_kernel<L, GUO, Real><<<n_items, AUX_THREADS, 0, st>>>(sys, items, d, dbar, static_cast<Real*>(fbuf));
    }
    return cudaGetLastError();
}

template <class L, class Real>
cudaError_t gather_any(const SysDev* sys, int s, int i, int64_t n, const void* fbuf, double* out, cudaStream_t st) {
    const unsigned grid = unsigned((n + AUX_THREADS - 1) / AUX_THREADS);
    gather_kernel<L, Real><<<grid, AUX_THREADS, 0, st>>>(sys, s, i, static_cast<const Real*>(fbuf), out);
    return cudaGetLastError();
}

template <class L, class Real>
cudaError_t scatter_any(const SysDev* sys, int s, int i, int64_t n, const double* in, void* fbuf, cudaStream_t st) {
    const unsigned grid = unsigned((n + AUX_THREADS - 1) / AUX_THREADS);
    scatter_kernel<L, Real><<<grid, AUX_THREADS, 0, st>>>(sys, s, i, in, static_cast<Real*>(fbuf));
    return cudaGetLastError();
}

template <class L, class Real>
cudaError_t obs_site_any(const SysDev* sys, const int4* items, int n_items, const void* fbuf, double* d,
                         double* partial, double* jout, int64_t jstride, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    obs_site_kernel<L, Real><<<n_items, AUX_THREADS, 0, st>>>(sys, items, static_cast<const Real*>(fbuf), d, partial,
                                                              jout, jstride);
    return cudaGetLastError();
}

}  // namespace lbf

// D3Q19 instantiations (3-D variant): the Guo-forced form with the Landau
// pressure in the equilibrium and the modified equilibrium carried to three
// dimensions, FP64 and FP32-deviation storage.
#include <type_traits>
#include <utility>

#include "lattice_tu.cuh"

namespace lbf {

namespace {
// (x, y, z-chunk, resident CTAs per SM, producer warps, staging, sites per
// consumer thread) of the z-marching kernel: producer warps 0 = every thread
// stages and collides its own column; > 0 = warp-specialised kernel (used on
// the fully relaxed FP32 path; the other paths run the plain kernel with the
// same tile), whose producers stage the footprint with plain loads (staging 0)
// or with bulk copies into shared memory (staging 1; systems that do not allow
// it run the staging-0 kernel of the same tile); the paired kernel stages
// aligned quads in registers (0) or with cp.async in shared memory (3).  Two sites per consumer
// thread: the paired kernel (x-adjacent site pairs, paired FP32 arithmetic;
// ensembles with an odd nx run the one-site warp-specialised kernel of the
// same tile).  The first entry is the default.
constexpr int kTiles[][kVariantCols] = {
    {32, 8, 32, 3, 4, 3, 2}, {32, 8, 64, 3, 4, 3, 2}, {16, 16, 32, 3, 4, 3, 2}, {16, 16, 64, 3, 4, 3, 2},
    {32, 8, 32, 2, 4, 0, 2}, {16, 16, 32, 2, 4, 0, 2},
    {32, 8, 64, 2, 4, 0, 2}, {16, 8, 32, 3, 4, 0, 1},  {16, 8, 64, 3, 4, 0, 1},  {16, 8, 16, 3, 4, 0, 1},
    {16, 8, 32, 3, 4, 1, 1}, {16, 8, 16, 6, 0, 0, 1},  {16, 8, 32, 6, 0, 0, 1},  {16, 16, 16, 4, 0, 0, 1},
    {16, 16, 32, 4, 0, 0, 1}};
constexpr int kNumTiles = int(sizeof(kTiles) / sizeof(kTiles[0]));
// ring planes of the paired kernel: 8 with register staging (2 CTAs per SM),
// 4 with cp.async staging (the staging areas share the shared memory)
constexpr int pair_ring(int stg) { return stg == 3 ? 4 : 8; }

template <int CP, class Real, int I>
cudaError_t step_variant(const StepLaunch& a, cudaStream_t st) {
    constexpr int PW = kTiles[I][4];
    if constexpr (CP == MODEQ) {
        // the modified equilibrium: the paired kernel on the paired rows (FP32,
        // every mode at tau = 1, every nx a multiple of 4), else the radius-1
        // z-marching kernel of the same tile
        if constexpr (PW > 0 && kTiles[I][5] == 3 && kTiles[I][6] == 2 && std::is_same<Real, float>::value) {
            if (a.bgk_only == 2 && a.pair_ok)
                return step_pair<kTiles[I][0], kTiles[I][1], kTiles[I][2], PW, kTiles[I][3], pair_ring(kTiles[I][5]),
                                 kTiles[I][5], MODEQ>(a, st);
        }
        return step_zm<D3Q19, Real, kTiles[I][0], kTiles[I][1], kTiles[I][2], kTiles[I][3]>(a, st);
    } else {
        if constexpr (PW > 0 && std::is_same<Real, float>::value) {
            if (a.bgk_only == 2) {
                if constexpr (kTiles[I][6] == 2) {
                    if (a.pair_ok)
                        return step_pair<kTiles[I][0], kTiles[I][1], kTiles[I][2], PW, kTiles[I][3],
                                         pair_ring(kTiles[I][5]), kTiles[I][5]>(a, st);
                    return step_ws<D3Q19, kTiles[I][0], kTiles[I][1], kTiles[I][2], PW, 1, 0>(a, st);
                } else {
                    if constexpr (kTiles[I][5] == 1) {
                        if (a.bulk_ok)
                            return step_ws<D3Q19, kTiles[I][0], kTiles[I][1], kTiles[I][2], PW, kTiles[I][3], 1>(a,
                                                                                                              st);
                    }
                    return step_ws<D3Q19, kTiles[I][0], kTiles[I][1], kTiles[I][2], PW, kTiles[I][3], 0>(a, st);
                }
            }
        }
        return step_z<D3Q19, CP, Real, kTiles[I][0], kTiles[I][1], kTiles[I][2], kTiles[I][3]>(a, st);
    }
}

template <int CP, class Real, int... I>
cudaError_t step_tile_of(const StepLaunch& a, cudaStream_t st, std::integer_sequence<int, I...>) {
    using Fn = cudaError_t (*)(const StepLaunch&, cudaStream_t);
    static constexpr Fn table[] = {&step_variant<CP, Real, I>...};
    if (a.tile_id < 0 || a.tile_id >= int(sizeof...(I))) return cudaErrorInvalidValue;
    return table[a.tile_id](a, st);
}

template <int CP, class Real>
cudaError_t step_tile(const StepLaunch& a, cudaStream_t st) {
    return step_tile_of<CP, Real>(a, st, std::make_integer_sequence<int, kNumTiles>{});
}
}  // namespace

int tile_shapes_d3q19(int (*out)[kVariantCols], int max) {
    for (int t = 0; t < kNumTiles && t < max; ++t)
        for (int k = 0; k < kVariantCols; ++k) out[t][k] = kTiles[t][k];
    return kNumTiles;
}

cudaError_t launch_step_d3q19(int coupling, int fp32, const StepLaunch& a, cudaStream_t st) {
    if (a.n_tiles == 0) return cudaSuccess;
    if (coupling == MODEQ) return fp32 ? step_tile<MODEQ, float>(a, st) : step_tile<MODEQ, double>(a, st);
    return fp32 ? step_tile<GUO, float>(a, st) : step_tile<GUO, double>(a, st);
}

cudaError_t launch_init_feq_d3q19(int coupling, int fp32, const SysDev* sys, const int4* items, int n_items,
                                 const double* d, const double* dbar, void* fbuf, cudaStream_t st) {
    return fp32 ? init_feq_any<D3Q19, float>(coupling, sys, items, n_items, d, dbar, fbuf, st)
                : init_feq_any<D3Q19, double>(coupling, sys, items, n_items, d, dbar, fbuf, st);
}
cudaError_t launch_gather_d3q19(int fp32, const SysDev* sys, int s, int i, int64_t n, const void* fbuf, double* out,
                               cudaStream_t st) {
    return fp32 ? gather_any<D3Q19, float>(sys, s, i, n, fbuf, out, st)
                : gather_any<D3Q19, double>(sys, s, i, n, fbuf, out, st);
}
cudaError_t launch_scatter_d3q19(int fp32, const SysDev* sys, int s, int i, int64_t n, const double* in, void* fbuf,
                                cudaStream_t st) {
    return fp32 ? scatter_any<D3Q19, float>(sys, s, i, n, in, fbuf, st)
                : scatter_any<D3Q19, double>(sys, s, i, n, in, fbuf, st);
}
cudaError_t launch_obs_site_d3q19(int fp32, const SysDev* sys, const int4* items, int n_items, const void* fbuf,
                                 double* d, double* partial, double* jout, int64_t jstride, cudaStream_t st) {
    return fp32 ? obs_site_any<D3Q19, float>(sys, items, n_items, fbuf, d, partial, jout, jstride, st)
                : obs_site_any<D3Q19, double>(sys, items, n_items, fbuf, d, partial, jout, jstride, st);
}

}  // namespace lbf

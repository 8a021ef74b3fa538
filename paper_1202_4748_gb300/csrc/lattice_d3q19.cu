// D3Q19 instantiations (3-D variant): Guo-forced form with the Landau
// pressure in the equilibrium, FP64 and FP32-deviation storage.
#include "lattice_tu.cuh"

namespace lbf {

namespace {
// (x, y, z-chunk, resident CTAs per SM) of the z-marching kernel
// (the first entry is the default: fastest on the 160-system ensemble by the autotuner)
constexpr int kTiles[][4] = {{16, 16, 16, 4}, {16, 16, 32, 4}, {16, 16, 8, 4}, {32, 16, 16, 2},
                             {16, 8, 16, 6}, {32, 8, 16, 4}};
constexpr int kNumTiles = int(sizeof(kTiles) / sizeof(kTiles[0]));

template <int CP, class Real>
cudaError_t step_tile(const StepLaunch& a, cudaStream_t st) {
    switch (a.tile_id) {
        case 0: return step_z<D3Q19, CP, Real, 16, 16, 16, 4>(a, st);
        case 1: return step_z<D3Q19, CP, Real, 16, 16, 32, 4>(a, st);
        case 2: return step_z<D3Q19, CP, Real, 16, 16, 8, 4>(a, st);
        case 3: return step_z<D3Q19, CP, Real, 32, 16, 16, 2>(a, st);
        case 4: return step_z<D3Q19, CP, Real, 16, 8, 16, 6>(a, st);
        case 5: return step_z<D3Q19, CP, Real, 32, 8, 16, 4>(a, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

int tile_shapes_d3q19(int (*out)[4], int max) {
    for (int t = 0; t < kNumTiles && t < max; ++t)
        for (int k = 0; k < 4; ++k) out[t][k] = kTiles[t][k];
    return kNumTiles;
}

cudaError_t launch_step_d3q19(int coupling, int fp32, const StepLaunch& a, cudaStream_t st) {
    if (a.n_tiles == 0) return cudaSuccess;
    if (coupling != GUO) return cudaErrorInvalidValue;   // Eq. 65 is a D2Q9 equilibrium
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
                                 double* d, double* partial, cudaStream_t st) {
    return fp32 ? obs_site_any<D3Q19, float>(sys, items, n_items, fbuf, d, partial, st)
                : obs_site_any<D3Q19, double>(sys, items, n_items, fbuf, d, partial, st);
}

}  // namespace lbf

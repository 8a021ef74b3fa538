// D2Q9 instantiations (the paper's lattice): modified equilibrium (Eq. 65)
// and the Guo-forced form, FP64 and FP32-deviation storage.
#include "lattice_tu.cuh"

namespace lbf {

namespace {
// (x, y, 1, resident CTAs per SM (0 = default), producer warps (0: none), scheme,
// sites per thread):
// scheme 2 = row-marching warp strips of x sites x y rows (modified equilibrium
// only; with 2 sites per thread each lane holds two x-adjacent sites, in
// paired FP32, when every mode is at tau = 1, the run is FP32 and every x side
// is a multiple of 4; otherwise the one-site strips run the same tiles),
// scheme 0 = CTA tiles of x by y sites with a density halo.
// Row 0 is the default of the modified equilibrium; the Guo form takes the
// first tile row.
constexpr int kTiles[][kVariantCols] = {{64, 32, 1, 3, 0, 2, 2}, {64, 16, 1, 3, 0, 2, 2}, {64, 64, 1, 3, 0, 2, 2},
                                        {64, 32, 1, 4, 0, 2, 2},
                                        {32, 32, 1, 6, 0, 2, 1}, {32, 64, 1, 6, 0, 2, 1}, {32, 16, 1, 6, 0, 2, 1},
                                        {32, 32, 1, 7, 0, 2, 1},
                                        {32, 8, 1, 0, 0, 0, 1},  {64, 4, 1, 0, 0, 0, 1},  {128, 2, 1, 0, 0, 0, 1},
                                        {32, 4, 1, 0, 0, 0, 1},  {32, 16, 1, 0, 0, 0, 1}, {64, 8, 1, 0, 0, 0, 1}};
constexpr int kNumTiles = int(sizeof(kTiles) / sizeof(kTiles[0]));

template <int CP, class Real, int YC, int MINB>
cudaError_t strip_of(const StepLaunch& a, cudaStream_t st) {
    if constexpr (CP == MODEQ) return step_strip<D2Q9, CP, Real, YC, 4, MINB>(a, st);
    return cudaErrorInvalidValue;            // the plan admits strips only with Eq. 65
}
template <int CP, class Real, int YC, int MINB>
cudaError_t strip2_of(const StepLaunch& a, cudaStream_t st) {
    if constexpr (CP == MODEQ) return step_strip2<D2Q9, CP, Real, YC, 4, MINB>(a, st);
    return cudaErrorInvalidValue;
}

template <int CP, class Real>
cudaError_t step_tile(const StepLaunch& a, cudaStream_t st) {
    switch (a.tile_id) {
        case 0: return strip2_of<CP, Real, 32, 3>(a, st);
        case 1: return strip2_of<CP, Real, 16, 3>(a, st);
        case 2: return strip2_of<CP, Real, 64, 3>(a, st);
        case 3: return strip2_of<CP, Real, 32, 4>(a, st);
        case 4: return strip_of<CP, Real, 32, 6>(a, st);
        case 5: return strip_of<CP, Real, 64, 6>(a, st);
        case 6: return strip_of<CP, Real, 16, 6>(a, st);
        case 7: return strip_of<CP, Real, 32, 7>(a, st);
        case 8: return step_one<D2Q9, CP, Real, 32, 8, 1>(a, st);
        case 9: return step_one<D2Q9, CP, Real, 64, 4, 1>(a, st);
        case 10: return step_one<D2Q9, CP, Real, 128, 2, 1>(a, st);
        case 11: return step_one<D2Q9, CP, Real, 32, 4, 1>(a, st);
        case 12: return step_one<D2Q9, CP, Real, 32, 16, 1>(a, st);
        case 13: return step_one<D2Q9, CP, Real, 64, 8, 1>(a, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

int tile_shapes_d2q9(int (*out)[kVariantCols], int max) {
    for (int t = 0; t < kNumTiles && t < max; ++t)
        for (int k = 0; k < kVariantCols; ++k) out[t][k] = kTiles[t][k];
    return kNumTiles;
}

cudaError_t launch_step_d2q9(int coupling, int fp32, const StepLaunch& a, cudaStream_t st) {
    if (a.n_tiles == 0) return cudaSuccess;
    if (coupling == MODEQ) return fp32 ? step_tile<MODEQ, float>(a, st) : step_tile<MODEQ, double>(a, st);
    return fp32 ? step_tile<GUO, float>(a, st) : step_tile<GUO, double>(a, st);
}

cudaError_t launch_init_feq_d2q9(int coupling, int fp32, const SysDev* sys, const int4* items, int n_items,
                                 const double* d, const double* dbar, void* fbuf, cudaStream_t st) {
    return fp32 ? init_feq_any<D2Q9, float>(coupling, sys, items, n_items, d, dbar, fbuf, st)
                : init_feq_any<D2Q9, double>(coupling, sys, items, n_items, d, dbar, fbuf, st);
}
cudaError_t launch_gather_d2q9(int fp32, const SysDev* sys, int s, int i, int64_t n, const void* fbuf, double* out,
                               cudaStream_t st) {
    return fp32 ? gather_any<D2Q9, float>(sys, s, i, n, fbuf, out, st)
                : gather_any<D2Q9, double>(sys, s, i, n, fbuf, out, st);
}
cudaError_t launch_scatter_d2q9(int fp32, const SysDev* sys, int s, int i, int64_t n, const double* in, void* fbuf,
                                cudaStream_t st) {
    return fp32 ? scatter_any<D2Q9, float>(sys, s, i, n, in, fbuf, st)
                : scatter_any<D2Q9, double>(sys, s, i, n, in, fbuf, st);
}
cudaError_t launch_obs_site_d2q9(int fp32, const SysDev* sys, const int4* items, int n_items, const void* fbuf,
                                 double* d, double* partial, double* jout, int64_t jstride, cudaStream_t st) {
    return fp32 ? obs_site_any<D2Q9, float>(sys, items, n_items, fbuf, d, partial, jout, jstride, st)
                : obs_site_any<D2Q9, double>(sys, items, n_items, fbuf, d, partial, jout, jstride, st);
}

}  // namespace lbf

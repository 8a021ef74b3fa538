// Block moments of one density snapshot without any device allocation.
//
// Most of this library works in a device workspace that the caller allocates.
// Some callers cannot allocate device memory at the point where they need the
// observables: an application whose framework has already reserved the whole
// device memory pool (so one more cudaMalloc fails), or a tight stepping loop
// that cannot afford the device-wide synchronisation cudaMalloc and cudaFree
// imply.  For them, lb_block_moments_noalloc takes only the caller's input and
// output buffers and keeps its scratch (work lists, partial sums, the block
// pyramid, accumulators) in one file-scope device array of fixed size.
//
// Consequences of the static array, for users:
//  * every GPU that loads this library holds kNoAllocScratchBytes of device
//    memory for it until the process exits;
//  * all calls share the array, so calls that overlap on the GPU (for example
//    on two streams of the same device) race on it; order them on one stream;
//  * the array keeps the previous call's contents; everything this entry point
//    needs zeroed is cleared at the start of each call;
//  * the first call on a device looks up the array's device address there
//    (cudaGetSymbolAddress); make that first call before any stream capture.
#include <cstring>

#include "../../include/lbfluct.h"
#include "lattice_kernels.cuh"
#include "lb_launch.h"

namespace lbf {

namespace {

constexpr int64_t kNoAllocMaxSites = LB_NOALLOC_MAX_SITES;
constexpr size_t kNoAllocScratchBytes = size_t(6) << 20;     // 6 MiB
constexpr int kMaxDevices = 64;
// host-side work-list bounds for kNoAllocMaxSites sites (item = 1024 sites or blocks)
constexpr int kMaxLevels = 33;
constexpr int kMaxItems = int(kNoAllocMaxSites / (AUX_THREADS * SITES_PER_THREAD)) + 1;
constexpr int kMaxUpItems = 2 * kMaxItems;

// The scratch itself.  Host code must not use this name as a pointer: on the
// host it is only a stand-in for the device object, whose address is obtained
// per device with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on each device (filled on first use).
static unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

// Sum of rho over each site item; partial[item * 4 + 0] = sum, the rest 0.
__global__ void __launch_bounds__(AUX_THREADS)
    rho_partial_kernel(const int4* __restrict__ items, const double* __restrict__ rho, double* __restrict__ partial) {
    __shared__ double sh[AUX_THREADS];
    const int4 it = items[blockIdx.x];
    double acc[1] = {0.0};
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int site = it.y + j * AUX_THREADS + threadIdx.x;
        if (site >= it.z) break;
        acc[0] += rho[site];
    }
    block_sum<1, AUX_THREADS>(acc, sh);
    if (threadIdx.x == 0) {
        partial[int64_t(blockIdx.x) * 4 + 0] = acc[0];
        partial[int64_t(blockIdx.x) * 4 + 1] = 0.0;
        partial[int64_t(blockIdx.x) * 4 + 2] = 0.0;
        partial[int64_t(blockIdx.x) * 4 + 3] = 0.0;
    }
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

}  // namespace lbf

using namespace lbf;

extern "C" lb_status lb_block_moments_noalloc(const double* d_rho, int nx, int ny, int nz, int lattice,
                                              double* d_out, int max_levels, int* n_levels, void* stream) {
    if (!d_rho || !d_out || !n_levels || nx < 1 || ny < 1 || nz < 1) return LB_ERR_ARG;
    if (lattice != LB_D2Q9 && lattice != LB_D3Q19) return LB_ERR_ARG;
    if (lattice == LB_D2Q9 && nz != 1) return LB_ERR_ARG;
    const int64_t n = int64_t(nx) * ny * nz;
    if (n > kNoAllocMaxSites) return LB_ERR_UNSUPPORTED;     // beyond the static scratch
    const bool dims3 = lattice == LB_D3Q19;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // levels L = S / 2^i while exact, then the single-site level
    // (no heap allocation: every host-side list lives in a bounded stack array)
    struct Lv {
        int bx, by, bz, gx, gy, gz;
        int64_t nb;
    };
    Lv lv[kMaxLevels];
    int nl = 0;
    for (int i = 0; i < 31; ++i) {
        const int p = 1 << i;
        if (nx % p || ny % p || (dims3 && nz % p)) break;
        lv[nl++] = {nx / p, ny / p, dims3 ? nz / p : 1, p, p, dims3 ? p : 1, int64_t(p) * p * (dims3 ? p : 1)};
        if (lv[nl - 1].bx == 1 && lv[nl - 1].by == 1 && lv[nl - 1].bz == 1) break;
    }
    const int imax = nl - 1;
    const bool unit_sep = !(lv[imax].bx == 1 && lv[imax].by == 1 && lv[imax].bz == 1);
    if (unit_sep) lv[nl++] = {1, 1, 1, nx, ny, nz, n};
    *n_levels = nl;
    if (max_levels < nl) return LB_ERR_ARG;

    // device-side work descriptors (built here, copied into the scratch)
    SysDev sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.nx = nx;
    sd.ny = ny;
    sd.nz = nz;
    sd.n_sites = n;
    sd.ns = int32_t(n);
    sd.rho_c = 0.0;              // the input is rho itself, so phi = (rho - mean) / mean
    sd.inv_rho_c = 1.0;

    LevelDev ld[kMaxLevels];
    int64_t blk = 0;
    for (int l = 0; l < nl; ++l) {
        LevelDev& D = ld[l];
        D.sys = 0;
        D.bx = lv[l].bx;
        D.by = lv[l].by;
        D.bz = lv[l].bz;
        D.gx = lv[l].gx;
        D.gy = lv[l].gy;
        D.gz = lv[l].gz;
        D.nblocks = lv[l].nb;
        const bool pyr = l <= imax;
        D.child = (pyr && l < imax) ? l + 1 : -1;
        D.off = pyr ? blk : -1;
        if (pyr) blk += lv[l].nb;
        D.rec_first = 0;
        D.rec_count = 0;
    }
    const int bchunk = OBS_THREADS * BLOCKS_PER_THREAD;
    ObsItem bottom[kMaxItems], up[kMaxUpItems];
    int n_bottom = 0, n_up = 0, rec = 0;
    for (int64_t b = 0; b < ld[imax].nblocks; b += bchunk) {
        if (n_bottom == kMaxItems) return LB_ERR_UNSUPPORTED;
        ObsItem& it = bottom[n_bottom++];
        it.level = imax;
        it.unit_level = unit_sep ? imax + 1 : -1;
        it.b0 = b;
        it.b1 = std::min<int64_t>(b + bchunk, ld[imax].nblocks);
        it.rec = -1;
        it.rec2 = -1;
    }
    ld[imax].rec_first = rec;
    ld[imax].rec_count = n_bottom;
    for (int j = 0; j < n_bottom; ++j) bottom[j].rec = rec + j;
    rec += n_bottom;
    if (unit_sep) {
        ld[imax + 1].rec_first = rec;
        ld[imax + 1].rec_count = n_bottom;
        for (int j = 0; j < n_bottom; ++j) bottom[j].rec2 = rec + j;
        rec += n_bottom;
    }
    int up_first[kMaxLevels + 1];
    up_first[0] = 0;
    for (int u = 1; u <= imax; ++u) {
        const int l = imax - u;
        ld[l].rec_first = rec;
        for (int64_t b = 0; b < ld[l].nblocks; b += bchunk) {
            if (n_up == kMaxUpItems) return LB_ERR_UNSUPPORTED;
            ObsItem& it = up[n_up++];
            it.level = l;
            it.unit_level = -1;
            it.b0 = b;
            it.b1 = std::min<int64_t>(b + bchunk, ld[l].nblocks);
            it.rec = rec++;
            it.rec2 = -1;
        }
        ld[l].rec_count = rec - ld[l].rec_first;
        up_first[u] = n_up;
    }
    int4 sites[kMaxItems];
    int n_items = 0;
    const int chunk = AUX_THREADS * SITES_PER_THREAD;
    for (int64_t b = 0; b < n; b += chunk) {
        if (n_items == kMaxItems) return LB_ERR_UNSUPPORTED;
        sites[n_items++] = make_int4(0, int(b), int(std::min<int64_t>(b + chunk, n)), 0);
    }
    const SysSpan span{0, n_items};

    // carve the static scratch
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + std::max<size_t>(bytes, 1));
        return at;
    };
    const size_t o_sys = take(sizeof(SysDev)), o_lv = take(sizeof(LevelDev) * nl),
                 o_bot = take(sizeof(ObsItem) * n_bottom), o_up = take(sizeof(ObsItem) * n_up),
                 o_items = take(sizeof(int4) * n_items), o_span = take(sizeof(SysSpan)),
                 o_part = take(sizeof(double) * 4 * n_items), o_red = take(sizeof(double) * 4),
                 o_dbar = take(sizeof(double)), o_glob = take(sizeof(double) * 8), o_stat = take(sizeof(int)),
                 o_S = take(sizeof(double) * blk), o_E = take(sizeof(double) * blk),
                 o_rec = take(sizeof(double) * REC * rec), o_acc = take(sizeof(double) * 7 * nl);
    if (off > kNoAllocScratchBytes) return LB_ERR_UNSUPPORTED;

    // device address of the static array on the current device (first call only)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LB_ERR_CUDA;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LB_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    unsigned char* base = g_scratch_addr[dev];

#define NA_CHECK(expr)                                  \
    do {                                                \
        if ((expr) != cudaSuccess) return LB_ERR_CUDA;  \
    } while (0)
    NA_CHECK(cudaMemcpyAsync(base + o_sys, &sd, sizeof(sd), cudaMemcpyHostToDevice, st));
    // (copies from pageable host memory return once the source has been staged)
    NA_CHECK(cudaMemcpyAsync(base + o_lv, ld, sizeof(LevelDev) * nl, cudaMemcpyHostToDevice, st));
    NA_CHECK(cudaMemcpyAsync(base + o_bot, bottom, sizeof(ObsItem) * n_bottom, cudaMemcpyHostToDevice, st));
    if (n_up) NA_CHECK(cudaMemcpyAsync(base + o_up, up, sizeof(ObsItem) * n_up, cudaMemcpyHostToDevice, st));
    NA_CHECK(cudaMemcpyAsync(base + o_items, sites, sizeof(int4) * n_items, cudaMemcpyHostToDevice, st));
    NA_CHECK(cudaMemcpyAsync(base + o_span, &span, sizeof(span), cudaMemcpyHostToDevice, st));
    // what this call accumulates into starts at zero (the array keeps the last call's contents)
    NA_CHECK(cudaMemsetAsync(base + o_acc, 0, sizeof(double) * 7 * nl, st));
    NA_CHECK(cudaMemsetAsync(base + o_glob, 0, sizeof(double) * 8, st));
    NA_CHECK(cudaMemsetAsync(base + o_stat, 0, sizeof(int), st));

    const SysDev* dsys = reinterpret_cast<const SysDev*>(base + o_sys);
    const LevelDev* dlv = reinterpret_cast<const LevelDev*>(base + o_lv);
    double* part = reinterpret_cast<double*>(base + o_part);
    double* red4 = reinterpret_cast<double*>(base + o_red);
    double* dbar = reinterpret_cast<double*>(base + o_dbar);
    double* S = reinterpret_cast<double*>(base + o_S);
    double* E = reinterpret_cast<double*>(base + o_E);
    double* recs = reinterpret_cast<double*>(base + o_rec);
    double* acc = reinterpret_cast<double*>(base + o_acc);

    rho_partial_kernel<<<n_items, AUX_THREADS, 0, st>>>(reinterpret_cast<const int4*>(base + o_items), d_rho,
                                                         part);
    NA_CHECK(cudaGetLastError());
    NA_CHECK(launch_reduce_sys(reinterpret_cast<const SysSpan*>(base + o_span), 1, part, 4, red4, st));
    NA_CHECK(launch_obs_globals(dsys, 1, red4, dbar, reinterpret_cast<double*>(base + o_glob), 1, 0, st));
    const HistDev no_hist{nullptr, 0, 0.0, 0.0};
    NA_CHECK(launch_pyr_bottom(dsys, dlv, reinterpret_cast<const ObsItem*>(base + o_bot), n_bottom, d_rho, dbar, S,
                               E, recs, no_hist, st));
    for (int u = 1; u <= imax; ++u) {
        const int first = up_first[u - 1], cnt = up_first[u] - first;
        NA_CHECK(launch_pyr_up(dsys, dlv, reinterpret_cast<const ObsItem*>(base + o_up) + first, cnt, dims3 ? 1 : 0,
                               S, E, recs, no_hist, st));
    }
    NA_CHECK(launch_obs_accum(dlv, nl, recs, acc, reinterpret_cast<int*>(base + o_stat), st));
    NA_CHECK(cudaMemcpyAsync(d_out, acc, sizeof(double) * 7 * nl, cudaMemcpyDeviceToDevice, st));
#undef NA_CHECK
    return LB_OK;
}

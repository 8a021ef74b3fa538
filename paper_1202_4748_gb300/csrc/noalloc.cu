// Block moments of one density snapshot without any device allocation.
//
// Most of this library works in a device workspace that the caller allocates.
// Some callers cannot allocate device memory at the point where they need the
// observables: an application whose framework has already reserved the whole
// device memory pool (so one more cudaMalloc fails), or a tight stepping loop
// that cannot afford the device-wide synchronisation cudaMalloc and cudaFree
// imply.  For them, lb_block_moments_noalloc takes only the caller's input and
// output buffers and keeps its scratch (work lists, partial sums, the block
// pyramid, accumulators) in one file-scope device array of fixed size.  The
// work lists are built on the device from the lattice shape by a setup
// kernel, so the call copies nothing from host memory and never waits for
// the stream.
//
// Consequences of the static array, for users:
//  * every GPU that loads this library holds kNoAllocScratchBytes of device
//    memory for it until the process exits;
//  * all calls share the array, so calls that overlap on the GPU (for example
//    on two streams of the same device) race on it; order them on one stream;
//  * the array keeps the previous call's contents; everything this entry point
//    needs zeroed is cleared at the start of each call;
//  * each call looks up the array's device address on the current device
//    (cudaGetSymbolAddress); the first call on a device also loads the
//    library's device code there, so make that first call before any stream
//    capture.
#include <algorithm>
#include <cstring>

#include "../../include/lbfluct.h"
#include "lattice_kernels.cuh"
#include "lb_launch.h"

namespace lbf {

namespace {

constexpr int64_t kNoAllocMaxSites = LB_NOALLOC_MAX_SITES;
constexpr size_t kNoAllocScratchBytes = size_t(6) << 20;     // 6 MiB
// host-side work-list bounds for kNoAllocMaxSites sites (item = 1024 sites or blocks)
constexpr int kMaxLevels = 33;
constexpr int kMaxItems = int(kNoAllocMaxSites / (AUX_THREADS * SITES_PER_THREAD)) + 1;
constexpr int kMaxUpItems = 2 * kMaxItems;

// The scratch itself.  Host code must not use this name as a pointer: on the
// host it is only a stand-in for the device object, whose address is obtained
// per device with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];


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

// The work plan of one call, a pure function of the lattice shape: computed on
// the host (sizes, launch counts, scratch carving) and, from the same code, by
// the setup kernel on the device (the descriptors themselves).
struct NaPlan {
    int nl, imax, unit_sep;
    int bx[kMaxLevels], by[kMaxLevels], bz[kMaxLevels], gx[kMaxLevels], gy[kMaxLevels], gz[kMaxLevels];
    int64_t nb[kMaxLevels];
    int64_t off[kMaxLevels];       // pyramid offset of the level's block sums (-1: unit level)
    int up_first[kMaxLevels + 1];  // up items of pyramid step u: [up_first[u - 1], up_first[u])
    int n_bottom, n_up, n_items, n_rec;
    int64_t blk;                   // pyramid blocks in all
};

__host__ __device__ inline int64_t na_min(int64_t a, int64_t b) { return a < b ? a : b; }

// Levels L = S / 2^i while every side divides exactly, then the single-site
// level; items of OBS_THREADS * BLOCKS_PER_THREAD blocks (bottom and up
// passes) and of AUX_THREADS * SITES_PER_THREAD sites.  False if a list would
// exceed its bound.
__host__ __device__ inline bool na_plan(int nx, int ny, int nz, bool dims3, NaPlan& P) {
    const int64_t n = int64_t(nx) * ny * nz;
    P.nl = 0;
    for (int i = 0; i < 31; ++i) {
        const int p = 1 << i;
        if (nx % p || ny % p || (dims3 && nz % p)) break;
        const int l = P.nl++;
        P.bx[l] = nx / p;
        P.by[l] = ny / p;
        P.bz[l] = dims3 ? nz / p : 1;
        P.gx[l] = p;
        P.gy[l] = p;
        P.gz[l] = dims3 ? p : 1;
        P.nb[l] = int64_t(p) * p * (dims3 ? p : 1);
        if (P.bx[l] == 1 && P.by[l] == 1 && P.bz[l] == 1) break;
    }
    P.imax = P.nl - 1;
    P.unit_sep = !(P.bx[P.imax] == 1 && P.by[P.imax] == 1 && P.bz[P.imax] == 1);
    if (P.unit_sep) {
        const int l = P.nl++;
        P.bx[l] = P.by[l] = P.bz[l] = 1;
        P.gx[l] = nx;
        P.gy[l] = ny;
        P.gz[l] = nz;
        P.nb[l] = n;
    }
    P.blk = 0;
    for (int l = 0; l < P.nl; ++l) {
        P.off[l] = l <= P.imax ? P.blk : -1;
        if (l <= P.imax) P.blk += P.nb[l];
    }
    const int64_t bchunk = OBS_THREADS * BLOCKS_PER_THREAD;
    P.n_bottom = int((P.nb[P.imax] + bchunk - 1) / bchunk);
    P.up_first[0] = 0;
    for (int u = 1; u <= P.imax; ++u) P.up_first[u] = P.up_first[u - 1] + int((P.nb[P.imax - u] + bchunk - 1) / bchunk);
    P.n_up = P.up_first[P.imax];
    const int64_t chunk = AUX_THREADS * SITES_PER_THREAD;
    P.n_items = int((n + chunk - 1) / chunk);
    P.n_rec = P.n_bottom * (1 + P.unit_sep) + P.n_up;
    return P.n_bottom <= kMaxItems && P.n_up <= kMaxUpItems && P.n_items <= kMaxItems;
}

struct NaLayout {                  // byte offsets of the scratch regions
    size_t sys, lv, bot, up, items, span, part, red, dbar, glob, stat, S, E, rec, acc, end;
};

NaLayout na_layout(const NaPlan& P) {
    NaLayout o;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + std::max<size_t>(bytes, 1));
        return at;
    };
    o.sys = take(sizeof(SysDev));
    o.lv = take(sizeof(LevelDev) * P.nl);
    o.bot = take(sizeof(ObsItem) * P.n_bottom);
    o.up = take(sizeof(ObsItem) * P.n_up);
    o.items = take(sizeof(int4) * P.n_items);
    o.span = take(sizeof(SysSpan));
    o.part = take(sizeof(double) * 4 * P.n_items);
    o.red = take(sizeof(double) * 4);
    o.dbar = take(sizeof(double));
    o.glob = take(sizeof(double) * 8);
    o.stat = take(sizeof(int));
    o.S = take(sizeof(double) * P.blk);
    o.E = take(sizeof(double) * P.blk);
    o.rec = take(sizeof(double) * REC * P.n_rec);
    o.acc = take(sizeof(double) * 7 * P.nl);
    o.end = off;
    return o;
}

// Writes the descriptors of the plan into the scratch and clears what the
// call accumulates into.  One CTA; thread 0 writes the per-system and
// per-level records, all threads the item lists.
__global__ void __launch_bounds__(AUX_THREADS)
    na_setup_kernel(const NaPlan P, const NaLayout o, int nx, int ny, int nz, unsigned char* base) {
    const int t = threadIdx.x;
    const int64_t n = int64_t(nx) * ny * nz;
    const int64_t bchunk = OBS_THREADS * BLOCKS_PER_THREAD;
    const int rec_unit = P.n_bottom, rec_up = P.n_bottom * (1 + P.unit_sep);
    if (t == 0) {
        SysDev* sd = reinterpret_cast<SysDev*>(base + o.sys);
        SysDev z{};
        z.nx = nx;
        z.ny = ny;
        z.nz = nz;
        z.n_sites = n;
        z.ns = int32_t(n);
        z.rho_c = 0.0;             // the input is rho itself, so phi = (rho - mean) / mean
        z.inv_rho_c = 1.0;
        *sd = z;
        LevelDev* ld = reinterpret_cast<LevelDev*>(base + o.lv);
        for (int l = 0; l < P.nl; ++l) {
            LevelDev D;
            D.sys = 0;
            D.bx = P.bx[l];
            D.by = P.by[l];
            D.bz = P.bz[l];
            D.gx = P.gx[l];
            D.gy = P.gy[l];
            D.gz = P.gz[l];
            D.nblocks = P.nb[l];
            D.child = l < P.imax ? l + 1 : -1;
            D.off = P.off[l];
            if (l == P.imax) {
                D.rec_first = 0;
                D.rec_count = P.n_bottom;
            } else if (l > P.imax) {
                D.rec_first = rec_unit;
                D.rec_count = P.n_bottom;
            } else {
                const int u = P.imax - l;
                D.rec_first = rec_up + P.up_first[u - 1];
                D.rec_count = P.up_first[u] - P.up_first[u - 1];
            }
            ld[l] = D;
        }
        *reinterpret_cast<SysSpan*>(base + o.span) = SysSpan{0, P.n_items};
        *reinterpret_cast<int*>(base + o.stat) = 0;
        double* glob = reinterpret_cast<double*>(base + o.glob);
        for (int k = 0; k < 8; ++k) glob[k] = 0.0;
    }
    ObsItem* bot = reinterpret_cast<ObsItem*>(base + o.bot);
    for (int j = t; j < P.n_bottom; j += AUX_THREADS) {
        ObsItem it;
        it.level = P.imax;
        it.unit_level = P.unit_sep ? P.imax + 1 : -1;
        it.b0 = j * bchunk;
        it.b1 = na_min(it.b0 + bchunk, P.nb[P.imax]);
        it.rec = j;
        it.rec2 = P.unit_sep ? rec_unit + j : -1;
        bot[j] = it;
    }
    ObsItem* up = reinterpret_cast<ObsItem*>(base + o.up);
    for (int j = t; j < P.n_up; j += AUX_THREADS) {
        int u = 1;
        while (j >= P.up_first[u]) ++u;
        const int l = P.imax - u, k = j - P.up_first[u - 1];
        ObsItem it;
        it.level = l;
        it.unit_level = -1;
        it.b0 = k * bchunk;
        it.b1 = na_min(it.b0 + bchunk, P.nb[l]);
        it.rec = rec_up + j;
        it.rec2 = -1;
        up[j] = it;
    }
    int4* items = reinterpret_cast<int4*>(base + o.items);
    const int64_t chunk = AUX_THREADS * SITES_PER_THREAD;
    for (int j = t; j < P.n_items; j += AUX_THREADS)
        items[j] = make_int4(0, int(j * chunk), int(na_min((j + 1) * chunk, n)), 0);
    double* acc = reinterpret_cast<double*>(base + o.acc);
    for (int k = t; k < 7 * P.nl; k += AUX_THREADS) acc[k] = 0.0;
}

// Copies the accumulated rows to the caller's output and the status word to
// the caller's status (when given).
__global__ void na_finish_kernel(const double* __restrict__ acc, int nvals, const int* __restrict__ stat,
                                 double* __restrict__ out, int* __restrict__ status) {
    for (int k = threadIdx.x; k < nvals; k += blockDim.x) out[k] = acc[k];
    if (threadIdx.x == 0 && status) *status = *stat;
}

}  // namespace

}  // namespace lbf

using namespace lbf;

extern "C" lb_status lb_block_moments_noalloc(const double* d_rho, int nx, int ny, int nz, int lattice,
                                              double* d_out, int max_levels, int* n_levels, int* d_status,
                                              void* stream) {
    if (!d_rho || !d_out || !n_levels || nx < 1 || ny < 1 || nz < 1) return LB_ERR_ARG;
    if (lattice != LB_D2Q9 && lattice != LB_D3Q19) return LB_ERR_ARG;
    if (lattice == LB_D2Q9 && nz != 1) return LB_ERR_ARG;
    const int64_t n = int64_t(nx) * ny * nz;
    if (n > kNoAllocMaxSites) return LB_ERR_UNSUPPORTED;     // beyond the static scratch
    const bool dims3 = lattice == LB_D3Q19;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    NaPlan P;
    if (!na_plan(nx, ny, nz, dims3, P)) return LB_ERR_UNSUPPORTED;
    *n_levels = P.nl;
    if (max_levels < P.nl) return LB_ERR_ARG;
    const NaLayout o = na_layout(P);
    if (o.end > kNoAllocScratchBytes) return LB_ERR_UNSUPPORTED;

    // device address of the static array on the current device
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return LB_ERR_CUDA;
    unsigned char* base = static_cast<unsigned char*>(addr);

#define NA_CHECK(expr)                                  \
    do {                                                \
        if ((expr) != cudaSuccess) return LB_ERR_CUDA;  \
    } while (0)
    na_setup_kernel<<<1, AUX_THREADS, 0, st>>>(P, o, nx, ny, nz, base);
    NA_CHECK(cudaGetLastError());

    const SysDev* dsys = reinterpret_cast<const SysDev*>(base + o.sys);
    const LevelDev* dlv = reinterpret_cast<const LevelDev*>(base + o.lv);
    double* part = reinterpret_cast<double*>(base + o.part);
    double* red4 = reinterpret_cast<double*>(base + o.red);
    double* dbar = reinterpret_cast<double*>(base + o.dbar);
    double* S = reinterpret_cast<double*>(base + o.S);
    double* E = reinterpret_cast<double*>(base + o.E);
    double* recs = reinterpret_cast<double*>(base + o.rec);
    double* acc = reinterpret_cast<double*>(base + o.acc);
    int* stat = reinterpret_cast<int*>(base + o.stat);

    rho_partial_kernel<<<P.n_items, AUX_THREADS, 0, st>>>(reinterpret_cast<const int4*>(base + o.items), d_rho,
                                                           part);
    NA_CHECK(cudaGetLastError());
    NA_CHECK(launch_reduce_sys(reinterpret_cast<const SysSpan*>(base + o.span), 1, part, 4, red4, st));
    NA_CHECK(launch_obs_globals(dsys, 1, red4, dbar, reinterpret_cast<double*>(base + o.glob), 1, 0, st));
    const HistDev no_hist{nullptr, 0, 0.0, 0.0};
    NA_CHECK(launch_pyr_bottom(dsys, dlv, reinterpret_cast<const ObsItem*>(base + o.bot), P.n_bottom, d_rho, dbar, S,
                               E, recs, no_hist, st));
    for (int u = 1; u <= P.imax; ++u) {
        const int first = P.up_first[u - 1], cnt = P.up_first[u] - first;
        NA_CHECK(launch_pyr_up(dsys, dlv, reinterpret_cast<const ObsItem*>(base + o.up) + first, cnt, dims3 ? 1 : 0,
                               S, E, recs, no_hist, st));
    }
    NA_CHECK(launch_obs_accum(dlv, P.nl, recs, acc, stat, st));
    na_finish_kernel<<<1, 256, 0, st>>>(acc, 7 * P.nl, stat, d_out, d_status);
    NA_CHECK(cudaGetLastError());
#undef NA_CHECK
    return LB_OK;
}

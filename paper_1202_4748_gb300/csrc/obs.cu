// Lattice-independent kernels: initial density perturbation, per-system FP64
// reductions, and the block-observable pyramid (Eqs. 46-50).
//
// The pyramid: block levels are L = S/2^i (i = 0..imax); the bottom level's
// block sums of phi and phi^2 are taken from the sites, every coarser level
// sums the 2^d children of the next finer one.  Per block the nonlinear terms
// m, m^2, |m|, m^4, E, E^2 (m = sum phi / V, E = sum phi^2 / 2V) are formed and
// reduced per item into a record; one thread per level then sums its records
// in order into the FP64 accumulators.  Every sum has a fixed order.
#include "lattice_kernels.cuh"
#include "lb_launch.h"

namespace lbf {

namespace {

__global__ void __launch_bounds__(AUX_THREADS)
    init_noise_kernel(const SysDev* __restrict__ sysv, const int4* __restrict__ items, double amp,
                      double* __restrict__ d, double* __restrict__ partial) {
    __shared__ double sh[AUX_THREADS];
    const int4 it = items[blockIdx.x];
    const SysDev& S = sysv[it.x];
    double acc[1] = {0.0};
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int site = it.y + j * AUX_THREADS + threadIdx.x;
        if (site >= it.z) break;
        const uint4 w = site_draw(S, uint32_t(site), 0, 0xFFu);
        const double u = (double(w.x) + 0.5) * 2.3283064365386962890625e-10;
        const double v = amp * (2.0 * u - 1.0);
        d[S.site_offset + site] = v;
        acc[0] += v;
    }
    block_sum<1, AUX_THREADS>(acc, sh);
    if (threadIdx.x == 0) partial[int64_t(blockIdx.x) * 4] = acc[0];
}

// out[s * K + k] = sum over the items of system s of partial[item * 4 + k], in order.
__global__ void __launch_bounds__(AUX_THREADS)
    reduce_sys_kernel(const SysSpan* __restrict__ spans, const double* __restrict__ partial, int K,
                      double* __restrict__ out) {
    __shared__ double sh[4 * AUX_THREADS];
    const SysSpan sp = spans[blockIdx.x];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int it = threadIdx.x; it < sp.count; it += AUX_THREADS) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < K) acc[k] += partial[int64_t(sp.first + it) * 4 + k];
    }
    block_sum<4, AUX_THREADS>(acc, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < K; ++k) out[blockIdx.x * K + k] = acc[k];
}

// glob layout per system (8 doubles): n_samples, mass0, mass, jx, jy, jz, rho_mean, spare
__global__ void obs_globals_kernel(const SysDev* __restrict__ sysv, int n_sys, const double* __restrict__ red4,
                                   double* __restrict__ dbar, double* __restrict__ glob, int set_mass0,
                                   int count_sample) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sys) return;
    const SysDev& S = sysv[s];
    const double sum_d = red4[s * 4 + 0];
    const double n = double(S.n_sites);
    const double mass = S.rho_c * n + sum_d;
    dbar[s] = sum_d / n;
    double* g = glob + s * 8;
    if (set_mass0) {
        g[0] = 0.0;
        g[1] = mass;
    }
    if (count_sample) g[0] += 1.0;
    g[2] = mass;
    g[3] = red4[s * 4 + 1];
    g[4] = red4[s * 4 + 2];
    g[5] = red4[s * 4 + 3];
    g[6] = mass / n;
}

__global__ void set_dbar_kernel(const SysDev* __restrict__ sysv, int n_sys, double* __restrict__ dbar) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n_sys) dbar[s] = sysv[s].rho_c;
}

__device__ __forceinline__ void add_terms(double (&t)[REC], double s, double e, double inv_v) {
    const double m = s * inv_v;
    const double E = 0.5 * e * inv_v;
    const double m2 = m * m;
    t[0] += m;
    t[1] += m2;
    t[2] += fabs(m);
    t[3] += m2 * m2;
    t[4] += E;
    t[5] += E * E;
}

// Histogram bin of a block value m: 1 + floor(t), t = (m - lo) * inv_w, with
// 0 below the range and nbins + 1 at or above it (and for NaN).  The product
// is formed from the rounded difference, as in the plain definition.
__device__ __forceinline__ int hist_bin(double m, const HistDev& H) {
    const double t = __dmul_rn(__dsub_rn(m, H.lo), H.inv_w);
    if (t >= 0.0) return t < double(H.nbins) ? 1 + int(t) : H.nbins + 1;
    return t < 0.0 ? 0 : H.nbins + 1;
}

// Per-CTA histograms in shared memory (32-bit counts; a CTA sees far fewer
// than 2^32 values), added to the 64-bit global counts at the end.
__device__ __forceinline__ void hist_clear(unsigned* sh, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) sh[k] = 0u;
}
__device__ __forceinline__ void hist_flush(const unsigned* sh, int n, unsigned long long* g) {
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        if (sh[k]) atomicAdd(g + k, (unsigned long long)sh[k]);
}

// Bottom pyramid level: block sums of phi, phi^2 straight from the sites; the
// separate single-site level (if any) is fed from the same loop.  With
// histograms on, each block value m (and each site value of the single-site
// level) is also binned.
__global__ void __launch_bounds__(OBS_THREADS)
    pyr_bottom_kernel(const SysDev* __restrict__ sysv, const LevelDev* __restrict__ lvv,
                      const ObsItem* __restrict__ items, const double* __restrict__ d,
                      const double* __restrict__ dbar, double* __restrict__ Sg, double* __restrict__ Eg,
                      double* __restrict__ rec, const HistDev H) {
    __shared__ double sh[REC * OBS_THREADS];
    extern __shared__ unsigned shist[];          // [block level | single-site level], nbins + 2 each
    const ObsItem it = items[blockIdx.x];
    const LevelDev lv = lvv[it.level];
    const SysDev& S = sysv[lv.sys];
    const double* ds = d + S.site_offset;
    const double db = dbar[lv.sys];
    const double inv_rbar = 1.0 / (S.rho_c + db);
    const double inv_v = 1.0 / (double(lv.bx) * lv.by * lv.bz);
    const int nh = H.nbins + 2;
    const bool hist = H.nbins > 0;
    const bool hist_u = hist && it.unit_level >= 0;
    if (hist) {
        hist_clear(shist, hist_u ? 2 * nh : nh);
        __syncthreads();
    }
    double tb[REC] = {0, 0, 0, 0, 0, 0};
    double tu[REC] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < BLOCKS_PER_THREAD; ++j) {
        const int64_t b = it.b0 + int64_t(j) * OBS_THREADS + threadIdx.x;
        if (b >= it.b1) break;
        const int X = int(b % lv.gx), Y = int((b / lv.gx) % lv.gy), Z = int(b / (int64_t(lv.gx) * lv.gy));
        double s = 0.0, e = 0.0;
        for (int z = 0; z < lv.bz; ++z)
            for (int y = 0; y < lv.by; ++y) {
                const int64_t row = int64_t(X) * lv.bx + int64_t(S.nx) * (int64_t(Y) * lv.by + y +
                                                                           int64_t(S.ny) * (int64_t(Z) * lv.bz + z));
                for (int x = 0; x < lv.bx; ++x) {
                    const double phi = (ds[row + x] - db) * inv_rbar;
                    s += phi;
                    e += phi * phi;
                    if (it.unit_level >= 0) add_terms(tu, phi, phi * phi, 1.0);
                    if (hist_u) atomicAdd(shist + nh + hist_bin(phi, H), 1u);
                }
            }
        Sg[lv.off + b] = s;
        Eg[lv.off + b] = e;
        add_terms(tb, s, e, inv_v);
        if (hist) atomicAdd(shist + hist_bin(s * inv_v, H), 1u);
    }
    block_sum<REC, OBS_THREADS>(tb, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < REC; ++k) rec[int64_t(it.rec) * REC + k] = tb[k];
    if (it.unit_level >= 0) {
        __syncthreads();
        block_sum<REC, OBS_THREADS>(tu, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < REC; ++k) rec[int64_t(it.rec2) * REC + k] = tu[k];
    }
    if (hist) {
        __syncthreads();
        hist_flush(shist, nh, H.counts + int64_t(it.level) * nh);
        if (hist_u) hist_flush(shist + nh, nh, H.counts + int64_t(it.unit_level) * nh);
    }
}

// One coarser level: each block sums its 2^d children of the next finer level.
__global__ void __launch_bounds__(OBS_THREADS)
    pyr_up_kernel(const LevelDev* __restrict__ lvv, const ObsItem* __restrict__ items, int dims3,
                  double* __restrict__ Sg, double* __restrict__ Eg, double* __restrict__ rec, const HistDev H) {
    __shared__ double sh[REC * OBS_THREADS];
    extern __shared__ unsigned shist[];
    const ObsItem it = items[blockIdx.x];
    const LevelDev lv = lvv[it.level];
    const LevelDev ch = lvv[lv.child];
    const double inv_v = 1.0 / (double(lv.bx) * lv.by * lv.bz);
    const int nh = H.nbins + 2;
    const bool hist = H.nbins > 0;
    if (hist) {
        hist_clear(shist, nh);
        __syncthreads();
    }
    double tb[REC] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < BLOCKS_PER_THREAD; ++j) {
        const int64_t b = it.b0 + int64_t(j) * OBS_THREADS + threadIdx.x;
        if (b >= it.b1) break;
        const int X = int(b % lv.gx), Y = int((b / lv.gx) % lv.gy), Z = int(b / (int64_t(lv.gx) * lv.gy));
        double s = 0.0, e = 0.0;
        const int nz = dims3 ? 2 : 1;
        for (int dz = 0; dz < nz; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int64_t cb = int64_t(2 * X + dx) +
                                       int64_t(ch.gx) * (int64_t(2 * Y + dy) + int64_t(ch.gy) * (int64_t(nz * Z + dz)));
                    s += Sg[ch.off + cb];
                    e += Eg[ch.off + cb];
                }
        Sg[lv.off + b] = s;
        Eg[lv.off + b] = e;
        add_terms(tb, s, e, inv_v);
        if (hist) atomicAdd(shist + hist_bin(s * inv_v, H), 1u);
    }
    block_sum<REC, OBS_THREADS>(tb, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < REC; ++k) rec[int64_t(it.rec) * REC + k] = tb[k];
    if (hist) {
        __syncthreads();
        hist_flush(shist, nh, H.counts + int64_t(it.level) * nh);
    }
}

// acc layout per level (7 doubles): n, sum m, m^2, |m|, m^4, e, e^2
__global__ void obs_accum_kernel(const LevelDev* __restrict__ lvv, int n_levels, const double* __restrict__ rec,
                                 double* __restrict__ acc, int* status) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_levels) return;
    const LevelDev lv = lvv[l];
    double t[REC] = {0, 0, 0, 0, 0, 0};
    for (int r = 0; r < lv.rec_count; ++r)
        for (int k = 0; k < REC; ++k) t[k] += rec[int64_t(lv.rec_first + r) * REC + k];
    double* a = acc + int64_t(l) * 7;
    a[0] += double(lv.nblocks);
    bool finite = true;
    for (int k = 0; k < REC; ++k) {
        a[1 + k] += t[k];
        finite = finite && isfinite(t[k]);
    }
    if (!finite) atomicOr(status, ST_NONFINITE);
}

__global__ void advance_kernel(int64_t* step, int64_t n) { *step += n; }

// Fault injection: OR bits into the device status word (as a kernel would on
// detecting the condition).
__global__ void set_status_kernel(int* status, int bits) { atomicOr(status, bits); }

// Self-test of the bounded waits: one CTA waits on an mbarrier that nothing
// arrives at; every thread must give up and the status must record it.
__global__ void selftest_wait_kernel(int* status) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
    }
    __syncthreads();
    if (mbar_wait(&bar, 0u, &abort_flag, status)) atomicOr(status, 1 << 30);   // cannot complete
}

}  // namespace

cudaError_t launch_init_noise(const SysDev* sys, const int4* items, int n_items, double amp, double* d,
                              double* partial, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    init_noise_kernel<<<n_items, AUX_THREADS, 0, st>>>(sys, items, amp, d, partial);
    return cudaGetLastError();
}

cudaError_t launch_reduce_sys(const SysSpan* spans, int n_sys, const double* partial, int K, double* out,
                              cudaStream_t st) {
    reduce_sys_kernel<<<n_sys, AUX_THREADS, 0, st>>>(spans, partial, K, out);
    return cudaGetLastError();
}

cudaError_t launch_obs_globals(const SysDev* sys, int n_sys, const double* red4, double* dbar, double* glob,
                               int set_mass0, int count_sample, cudaStream_t st) {
    obs_globals_kernel<<<(n_sys + 127) / 128, 128, 0, st>>>(sys, n_sys, red4, dbar, glob, set_mass0, count_sample);
    return cudaGetLastError();
}

cudaError_t launch_set_dbar(const SysDev* sys, int n_sys, double* dbar, cudaStream_t st) {
    set_dbar_kernel<<<(n_sys + 127) / 128, 128, 0, st>>>(sys, n_sys, dbar);
    return cudaGetLastError();
}

cudaError_t launch_pyr_bottom(const SysDev* sys, const LevelDev* lv, const ObsItem* items, int n_items,
                              const double* d, const double* dbar, double* S, double* E, double* rec,
                              const HistDev& hist, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const size_t shm = hist.nbins > 0 ? 2 * sizeof(unsigned) * (hist.nbins + 2) : 0;
    pyr_bottom_kernel<<<n_items, OBS_THREADS, shm, st>>>(sys, lv, items, d, dbar, S, E, rec, hist);
    return cudaGetLastError();
}

cudaError_t launch_pyr_up(const SysDev*, const LevelDev* lv, const ObsItem* items, int n_items, int dims3,
                          double* S, double* E, double* rec, const HistDev& hist, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const size_t shm = hist.nbins > 0 ? sizeof(unsigned) * (hist.nbins + 2) : 0;
    pyr_up_kernel<<<n_items, OBS_THREADS, shm, st>>>(lv, items, dims3, S, E, rec, hist);
    return cudaGetLastError();
}

cudaError_t launch_obs_accum(const LevelDev* lv, int n_levels_total, const double* rec, double* acc, int* status,
                             cudaStream_t st) {
    obs_accum_kernel<<<(n_levels_total + 127) / 128, 128, 0, st>>>(lv, n_levels_total, rec, acc, status);
    return cudaGetLastError();
}

cudaError_t launch_advance(int64_t* step, int64_t n, cudaStream_t st) {
    advance_kernel<<<1, 1, 0, st>>>(step, n);
    return cudaGetLastError();
}

cudaError_t launch_selftest_wait(int* status, cudaStream_t st) {
    selftest_wait_kernel<<<1, 64, 0, st>>>(status);
    return cudaGetLastError();
}

cudaError_t launch_set_status(int* status, int bits, cudaStream_t st) {
    set_status_kernel<<<1, 1, 0, st>>>(status, bits);
    return cudaGetLastError();
}

}  // namespace lbf

// Internal host-side interface between the C ABI (api.cu) and the kernel
// translation units.  Plain structs and pointers only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lb_device.cuh"

namespace lbf {

constexpr int AUX_THREADS = 256;        // threads of the auxiliary (non-step) kernels
constexpr int SITES_PER_THREAD = 4;     // sites per thread in a site-pass item

struct StepLaunch {
    const SysDev* sys;
    const void* phys;       // SysPhys<float> or SysPhys<double> per system
    const int4* tiles;
    int n_tiles;
    const void* fin;
    void* fout;
    const int64_t* step_ptr;
    int k;
    int* status;
    int tile_id;            // index into the lattice's tile-shape table
    int bgk_only;           // 0: per-mode rates; 1: one rate per system; 2: one rate, equal to 1
    int bulk_ok;            // every system allows bulk-copy staging (nx % 4 == 0, nx >= 8, sides >= 3)
    int pair_ok;            // every system has nx % 4 == 0 (the paired-site kernel can run)
};

// Step-kernel variants compiled for each lattice: (x, y, z, resident CTAs per
// SM, producer warps, staging: 0 plain loads, 1 bulk copies, sites per
// consumer thread); index = tile_id.
constexpr int kVariantCols = 7;
int tile_shapes_d2q9(int (*out)[kVariantCols], int max);
int tile_shapes_d3q19(int (*out)[kVariantCols], int max);

cudaError_t launch_step_d2q9(int coupling, int fp32, const StepLaunch& a, cudaStream_t st);
cudaError_t launch_step_d3q19(int coupling, int fp32, const StepLaunch& a, cudaStream_t st);

cudaError_t launch_init_feq_d2q9(int coupling, int fp32, const SysDev* sys, const int4* items, int n_items,
                                 const double* d, const double* dbar, void* fbuf, cudaStream_t st);
cudaError_t launch_init_feq_d3q19(int coupling, int fp32, const SysDev* sys, const int4* items, int n_items,
                                  const double* d, const double* dbar, void* fbuf, cudaStream_t st);
cudaError_t launch_gather_d2q9(int fp32, const SysDev* sys, int s, int i, int64_t n, const void* fbuf, double* out,
                               cudaStream_t st);
cudaError_t launch_gather_d3q19(int fp32, const SysDev* sys, int s, int i, int64_t n, const void* fbuf, double* out,
                                cudaStream_t st);
cudaError_t launch_scatter_d2q9(int fp32, const SysDev* sys, int s, int i, int64_t n, const double* in, void* fbuf,
                                cudaStream_t st);
cudaError_t launch_scatter_d3q19(int fp32, const SysDev* sys, int s, int i, int64_t n, const double* in, void* fbuf,
                                 cudaStream_t st);
// jout (nullable): momentum field j_a at jout + a * jstride.
cudaError_t launch_obs_site_d2q9(int fp32, const SysDev* sys, const int4* items, int n_items, const void* fbuf,
                                 double* d, double* partial, double* jout, int64_t jstride, cudaStream_t st);
cudaError_t launch_obs_site_d3q19(int fp32, const SysDev* sys, const int4* items, int n_items, const void* fbuf,
                                  double* d, double* partial, double* jout, int64_t jstride, cudaStream_t st);

// ---- lattice-independent (obs.cu) ----------------------------------------
struct SysSpan {            // items [first, first + count) of one system
    int first, count;
};

// One block level of one system, as the observable kernels see it.
struct LevelDev {
    int32_t sys;
    int32_t bx, by, bz;     // block dims
    int32_t gx, gy, gz;     // blocks per axis
    int32_t child;          // index of the next finer pyramid level (-1 at the bottom)
    int64_t nblocks;
    int64_t off;            // offset of this level's block sums in the S/E arrays (-1: unit level)
    int32_t rec_first;      // records of this level in the partial-record array
    int32_t rec_count;
};

struct ObsItem {            // a range of blocks of one level
    int32_t level;          // index into the LevelDev array
    int32_t unit_level;     // bottom items also feed the separate single-site level (-1: none)
    int64_t b0, b1;
    int32_t rec, rec2;      // partial records written (rec2 for the unit level)
};

// Order-parameter histograms: per level (nbins + 2) counts [under, bins, over]
// at counts + level * (nbins + 2); nbins = 0 disables them.
struct HistDev {
    unsigned long long* counts;
    int32_t nbins;
    double lo, inv_w;       // bin of m: floor((m - lo) * inv_w), inv_w = nbins / (hi - lo)
};

// OR status bits into the device status word (fault injection).
cudaError_t launch_set_status(int* status, int bits, cudaStream_t st);
// One CTA whose bounded wait on a barrier nothing arrives at must time out.
cudaError_t launch_selftest_wait(int* status, cudaStream_t st);

cudaError_t launch_init_noise(const SysDev* sys, const int4* items, int n_items, double amp, double* d,
                              double* partial, cudaStream_t st);
cudaError_t launch_reduce_sys(const SysSpan* spans, int n_sys, const double* partial, int K, double* out,
                              cudaStream_t st);
cudaError_t launch_obs_globals(const SysDev* sys, int n_sys, const double* red4, double* dbar, double* glob,
                               int set_mass0, int count_sample, cudaStream_t st);
cudaError_t launch_set_dbar(const SysDev* sys, int n_sys, double* dbar, cudaStream_t st);
cudaError_t launch_pyr_bottom(const SysDev* sys, const LevelDev* lv, const ObsItem* items, int n_items,
                              const double* d, const double* dbar, double* S, double* E, double* rec,
                              const HistDev& hist, cudaStream_t st);
cudaError_t launch_pyr_up(const SysDev* sys, const LevelDev* lv, const ObsItem* items, int n_items, int dims3,
                          double* S, double* E, double* rec, const HistDev& hist, cudaStream_t st);
cudaError_t launch_obs_accum(const LevelDev* lv, int n_levels_total, const double* rec, double* acc,
                             int* status, cudaStream_t st);
cudaError_t launch_advance(int64_t* step, int64_t n, cudaStream_t st);

constexpr int OBS_THREADS = 256;
constexpr int BLOCKS_PER_THREAD = 4;
constexpr int REC = 6;      // per record: sum m, m^2, |m|, m^4, e, e^2

}  // namespace lbf

namespace lbf {

// ---- structure factor (Eq. 80) -------------------------------------------------
struct SkSys {             // per system: sides, twiddle-table offsets, site offset
    int32_t nx, ny, nz;
    int32_t tw_x, tw_y, tw_z;   // offsets of W_n^j = exp(-2 pi i j / n) tables (complex)
    int64_t site_offset;
    double inv_n;               // 1 / sites
};

cudaError_t launch_sk_twiddles(double* tw, const int* sides, const int* offs, int n_tables, int max_n,
                               cudaStream_t st);
// x pass (real phi -> complex), then y and z passes (complex -> complex), then accumulate |F|^2 / N.
cudaError_t launch_sk_x(const SysDev* sys, const SkSys* sk, const int4* items, int n_items, const double* d,
                        const double* dbar, const double* tw, double* out, cudaStream_t st);
cudaError_t launch_sk_pass(const SkSys* sk, const int4* items, int n_items, int axis, const double* tw,
                           const double* in, double* out, cudaStream_t st);
// Line FFTs along `axis` for systems with equal sides 2^a 3^b (see sk.cu):
// items (system, first line, line count, 0) with line count * side <= max_elems
// <= kSkFftMaxElems; in == nullptr: real input from d (and dbar) as launch_sk_x.
constexpr int kSkFftMaxElems = 2048;
bool sk_fft_side(int n);   // n = 2^a 3^b and n <= kSkFftMaxElems
cudaError_t launch_sk_fft(const SysDev* sys, const SkSys* sk, const int4* items, int n_items, int axis,
                          const double* d, const double* dbar, const double* in, const double* tw, double* out,
                          int max_elems, cudaStream_t st);
cudaError_t launch_sk_accum(const SkSys* sk, const int4* items, int n_items, const double* F, double* acc,
                            cudaStream_t st);
// per-shell sums of the accumulated C(k) of one system (one CTA per shell)
// Momentum spectra (see sk.cu): accumulate the x, longitudinal and transverse
// spectra of the transforms F0..F2 (F2 unused in 2-D) into acc + c * stride.
cudaError_t launch_jk_accum(const SkSys* sk, const int4* items, int n_items, int dims, const double* F0,
                            const double* F1, const double* F2, double* acc, int64_t stride, cudaStream_t st);
// Guo variant: lap = Laplacian of d, then j_a += kappa rho d_a(lap) / 2 (j at jf + a * stride).
cudaError_t launch_jk_guo_force(int lattice, const SysDev* sys, const int4* items, int n_items, const double* d,
                                double* lap, double* jf, int64_t stride, cudaStream_t st);
cudaError_t launch_sk_bin(const SkSys* sk, int sys, const double* acc, int nbins, double* sums, double* counts,
                          cudaStream_t st);

}  // namespace lbf

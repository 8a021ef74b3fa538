// Structure factor C(k) = N^-1 |sum_r phi(r) exp(-i k.r)|^2 (Eq. 80), accumulated
// in FP64 over samples for every k of every system.  The discrete Fourier
// transform is taken one axis at a time (x: real -> complex, then y, z) with
// per-side twiddle tables W_n^j = exp(-2 pi i j / n).  Sides of the form
// 2^a 3^b (every workload's) are transformed by a mixed-radix (4, 2, 3)
// Stockham FFT, one CTA per group of lines in shared memory; other sides sum
// each output element's line directly in a fixed order.  Shell binning
// (j(j-1) < |n|^2 <= j(j+1)) happens only when the accumulated spectrum is read.
#include "lattice_kernels.cuh"
#include "lb_launch.h"

namespace lbf {

namespace {

__global__ void sk_twiddle_kernel(double* __restrict__ tw, const int* __restrict__ sides,
                                  const int* __restrict__ offs, int n_tables, int max_n) {
    const int t = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tables) return;
    const int n = sides[t];
    if (j >= n || j >= max_n) return;
    double s, c;
    sincospi(-2.0 * double(j) / double(n), &s, &c);
    tw[2 * (offs[t] + j)] = c;
    tw[2 * (offs[t] + j) + 1] = s;
}

// item: (system, first element, end element, unused); element e of a system
// enumerates its sites in [z][y][x] order, and names the output (k_x, y, z) etc.
// With dbar the input is phi = (d - dbar) / (rho_c + dbar); without (null) it
// is the field d itself.
__global__ void __launch_bounds__(AUX_THREADS)
    sk_x_kernel(const SysDev* __restrict__ sysv, const SkSys* __restrict__ skv, const int4* __restrict__ items,
                const double* __restrict__ d, const double* __restrict__ dbar, const double* __restrict__ tw,
                double* __restrict__ out) {
    const int4 it = items[blockIdx.x];
    const SkSys K = skv[it.x];
    const SysDev& S = sysv[it.x];
    const double db = dbar ? dbar[it.x] : 0.0;
    const double inv_rbar = dbar ? 1.0 / (S.rho_c + db) : 1.0;
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int e = it.y + j * AUX_THREADS + threadIdx.x;
        if (e >= it.z) break;
        const int kx = e % K.nx;
        const int line = e - kx;
        const double* row = d + K.site_offset + line;
        double re = 0.0, im = 0.0;
        int idx = 0;                      // (kx * x) mod nx, advanced incrementally
        for (int x = 0; x < K.nx; ++x) {
            const double phi = (row[x] - db) * inv_rbar;
            re += phi * tw[2 * (K.tw_x + idx)];
            im += phi * tw[2 * (K.tw_x + idx) + 1];
            idx += kx;
            if (idx >= K.nx) idx -= K.nx;
        }
        out[2 * (K.site_offset + e)] = re;
        out[2 * (K.site_offset + e) + 1] = im;
    }
}

__global__ void __launch_bounds__(AUX_THREADS)
    sk_pass_kernel(const SkSys* __restrict__ skv, const int4* __restrict__ items, int axis,
                   const double* __restrict__ tw, const double* __restrict__ in, double* __restrict__ out) {
    const int4 it = items[blockIdx.x];
    const SkSys K = skv[it.x];
    const int n = axis == 1 ? K.ny : K.nz;
    const int64_t stride = axis == 1 ? K.nx : int64_t(K.nx) * K.ny;
    const int toff = axis == 1 ? K.tw_y : K.tw_z;
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int e = it.y + j * AUX_THREADS + threadIdx.x;
        if (e >= it.z) break;
        const int k = int((e / stride) % n);           // output wavenumber index along the axis
        const int64_t base = e - int64_t(k) * stride;  // element with axis coordinate 0
        const double* src = in + 2 * (K.site_offset + base);
        double re = 0.0, im = 0.0;
        int idx = 0;
        for (int y = 0; y < n; ++y) {
            const double ar = src[2 * (int64_t(y) * stride)], ai = src[2 * (int64_t(y) * stride) + 1];
            const double wr = tw[2 * (toff + idx)], wi = tw[2 * (toff + idx) + 1];
            re += ar * wr - ai * wi;
            im += ar * wi + ai * wr;
            idx += k;
            if (idx >= n) idx -= n;
        }
        out[2 * (K.site_offset + e)] = re;
        out[2 * (K.site_offset + e) + 1] = im;
    }
}

__global__ void __launch_bounds__(AUX_THREADS)
    sk_accum_kernel(const SkSys* __restrict__ skv, const int4* __restrict__ items, const double* __restrict__ F,
                    double* __restrict__ acc) {
    const int4 it = items[blockIdx.x];
    const SkSys K = skv[it.x];
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int e = it.y + j * AUX_THREADS + threadIdx.x;
        if (e >= it.z) break;
        const int64_t g = K.site_offset + e;
        const double re = F[2 * g], im = F[2 * g + 1];
        acc[g] += (re * re + im * im) * K.inv_n;
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// -i a
__device__ __forceinline__ double2 cmi(double2 a) { return make_double2(a.y, -a.x); }

// Line FFT along `axis` (0 x, 1 y, 2 z) of systems with equal sides S = 2^a 3^b:
// item = (system, first line, line count, unused); line l of a system is the
// l-th line along the axis with the other two coordinates in [z][y][x] order
// (x lines: l = y + S z; y lines: l = x + S z; z lines: l = x + S y).  REAL_IN:
// the input is phi = (d - dbar)/(rho_c + dbar) (or d itself without dbar),
// else the complex field `in`.  Stockham autosort: stage with radix R after
// sub-transforms of length Ns takes, for butterfly j of a line, the R inputs
// a[j + r S/R] times W^(k r S/(Ns R)), k = j mod Ns, and writes their R-point
// DFT to b[(j / Ns) Ns R + k + s Ns]; after the last stage the line is in
// natural order.  F(k) = sum_x a(x) exp(-2 pi i k x / S), as the direct sums.
template <bool REAL_IN>
__global__ void __launch_bounds__(AUX_THREADS)
    sk_fft_kernel(const SysDev* __restrict__ sysv, const SkSys* __restrict__ skv, const int4* __restrict__ items,
                  int axis, const double* __restrict__ d, const double* __restrict__ dbar,
                  const double2* __restrict__ in, const double2* __restrict__ tw, double2* __restrict__ out) {
    extern __shared__ double2 fft_buf[];
    const int4 it = items[blockIdx.x];
    const SkSys K = skv[it.x];
    const int S = K.nx;
    const int nl = it.z, line0 = it.y;
    const int toff = axis == 0 ? K.tw_x : (axis == 1 ? K.tw_y : K.tw_z);
    double2* A = fft_buf;
    double2* B = fft_buf + nl * S;
    auto elem = [&](int line, int t) -> int64_t {
        if (axis == 0) return int64_t(line) * S + t;
        const int u = line % S, v = line / S;
        if (axis == 1) return u + int64_t(S) * (t + int64_t(S) * v);
        return u + int64_t(S) * (v + int64_t(S) * t);
    };
    // element (line l, position t) <-> index: x lines contiguous per line, the
    // other axes with consecutive lines (consecutive x) in consecutive threads
    auto lt = [&](int idx, int& l, int& t) {
        if (axis == 0) {
            l = idx / S;
            t = idx - l * S;
        } else {
            t = idx / nl;
            l = idx - t * nl;
        }
    };
    double db = 0.0, inv_rbar = 1.0;
    if constexpr (REAL_IN) {
        if (dbar) {
            db = dbar[it.x];
            inv_rbar = 1.0 / (sysv[it.x].rho_c + db);
        }
    }
    for (int idx = threadIdx.x; idx < nl * S; idx += AUX_THREADS) {
        int l, t;
        lt(idx, l, t);
        const int64_t g = K.site_offset + elem(line0 + l, t);
        if constexpr (REAL_IN) A[l * S + t] = make_double2((d[g] - db) * inv_rbar, 0.0);
        else A[l * S + t] = in[g];
    }
    __syncthreads();
    int Ns = 1;
    for (int m = S; m > 1;) {
        const int R = (m % 4 == 0) ? 4 : ((m % 2 == 0) ? 2 : 3);
        m /= R;
        const int nb = S / R, tstep = S / (Ns * R);
        for (int b = threadIdx.x; b < nl * nb; b += AUX_THREADS) {
            const int l = b / nb, j = b - l * nb, k = j % Ns;
            const double2* src = A + l * S;
            double2* dst = B + l * S + (j / Ns) * Ns * R + k;
            double2 v[4];
            v[0] = src[j];
            for (int r = 1; r < R; ++r) v[r] = cmul(src[j + r * nb], tw[toff + k * r * tstep]);
            if (R == 4) {
                const double2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
                const double2 s13 = cadd(v[1], v[3]), d13 = cmi(csub(v[1], v[3]));
                dst[0] = cadd(s02, s13);
                dst[Ns] = cadd(d02, d13);
                dst[2 * Ns] = csub(s02, s13);
                dst[3 * Ns] = csub(d02, d13);
            } else if (R == 2) {
                dst[0] = cadd(v[0], v[1]);
                dst[Ns] = csub(v[0], v[1]);
            } else {
                // w = exp(-2 pi i / 3): X1,2 = v0 - (v1 + v2)/2 -+ i (sqrt(3)/2)(v1 - v2)
                const double2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
                const double2 m0 = make_double2(v[0].x - 0.5 * t1.x, v[0].y - 0.5 * t1.y);
                const double h = 0.86602540378443864676;
                const double2 rt = make_double2(h * t2.y, -h * t2.x);      // -i (sqrt(3)/2) t2
                dst[0] = cadd(v[0], t1);
                dst[Ns] = cadd(m0, rt);
                dst[2 * Ns] = csub(m0, rt);
            }
        }
        __syncthreads();
        double2* tmp = A;
        A = B;
        B = tmp;
        Ns *= R;
    }
    for (int idx = threadIdx.x; idx < nl * S; idx += AUX_THREADS) {
        int l, t;
        lt(idx, l, t);
        out[K.site_offset + elem(line0 + l, t)] = A[l * S + t];
    }
}

__device__ __forceinline__ int wrapk(int k, int n) { return 2 * k < n ? k : k - n; }

// Momentum spectra of one sample (Eq. 69 diagnostics): from the transforms
// J_a(k) (complex, one field per component) accumulate per k
//   acc[0][k] += |J_x|^2 / N
//   acc[1][k] += |khat . J|^2 / N                       (0 at k = 0)
//   acc[2][k] += (|J|^2 - |khat . J|^2) / (N (d - 1))    (0 at k = 0)
// with khat = n / |n|, n the wrapped integer wavevector; acc[c] = acc + c * stride.
__global__ void __launch_bounds__(AUX_THREADS)
    jk_accum_kernel(const SkSys* __restrict__ skv, const int4* __restrict__ items, int dims,
                    const double* __restrict__ F0, const double* __restrict__ F1, const double* __restrict__ F2,
                    double* __restrict__ acc, int64_t stride) {
    const int4 it = items[blockIdx.x];
    const SkSys K = skv[it.x];
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int e = it.y + j * AUX_THREADS + threadIdx.x;
        if (e >= it.z) break;
        const int64_t g = K.site_offset + e;
        const int kx = e % K.nx, ky = (e / K.nx) % K.ny, kz = e / (K.nx * K.ny);
        const double a = wrapk(kx, K.nx), b = wrapk(ky, K.ny), c = dims == 3 ? wrapk(kz, K.nz) : 0;
        const double xr = F0[2 * g], xi = F0[2 * g + 1];
        const double yr = F1[2 * g], yi = F1[2 * g + 1];
        const double zr = dims == 3 ? F2[2 * g] : 0.0, zi = dims == 3 ? F2[2 * g + 1] : 0.0;
        const double jx2 = xr * xr + xi * xi;
        acc[g] += jx2 * K.inv_n;
        const double nn2 = a * a + b * b + c * c;
        if (nn2 > 0.0) {
            const double inv = 1.0 / sqrt(nn2);
            const double pr = (a * xr + b * yr + c * zr) * inv, pi = (a * xi + b * yi + c * zi) * inv;
            const double p2 = pr * pr + pi * pi;
            const double tot = jx2 + yr * yr + yi * yi + zr * zr + zi * zi;
            acc[stride + g] += p2 * K.inv_n;
            acc[2 * stride + g] += (tot - p2) * K.inv_n / double(dims - 1);
        }
    }
}

// Laplacian of the density deviation d (FP64): lap(r) = 6 sum_i t_i (d(r + c_i) - d(r)).
template <class L>
__global__ void __launch_bounds__(AUX_THREADS)
    jk_lap_kernel(const SysDev* __restrict__ sysv, const int4* __restrict__ items, const double* __restrict__ d,
                  double* __restrict__ lap) {
    const int4 it = items[blockIdx.x];
    const SysDev& S = sysv[it.x];
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const double* ds = d + S.site_offset;
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int site = it.y + j * AUX_THREADS + threadIdx.x;
        if (site >= it.z) break;
        int x, y, z;
        site_coords(site, nx, ny, x, y, z);
        const double c0 = ds[site];
        double v = 0.0;
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            const int sx = wrap1(x + L::c(i, 0), nx), sy = wrap1(y + L::c(i, 1), ny);
            const int sz = L::D == 3 ? wrap1(z + L::c(i, 2), nz) : 0;
            v += 6.0 * L::w(i) * (ds[sx + nx * (sy + ny * sz)] - c0);
        }
        lap[S.site_offset + site] = v;
    }
}

// Guo half-force: j_a(r) += (1/2) kappa rho(r) d_a lap(r), d_a X = 3 sum_i t_i c_ia X(r + c_i),
// rho = rho_c + d; the three components at j + a * stride.
template <class L>
__global__ void __launch_bounds__(AUX_THREADS)
    jk_force_kernel(const SysDev* __restrict__ sysv, const int4* __restrict__ items, const double* __restrict__ d,
                    const double* __restrict__ lap, double* __restrict__ jf, int64_t stride) {
    const int4 it = items[blockIdx.x];
    const SysDev& S = sysv[it.x];
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const double* ls = lap + S.site_offset;
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int site = it.y + j * AUX_THREADS + threadIdx.x;
        if (site >= it.z) break;
        int x, y, z;
        site_coords(site, nx, ny, x, y, z);
        double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            const int sx = wrap1(x + L::c(i, 0), nx), sy = wrap1(y + L::c(i, 1), ny);
            const int sz = L::D == 3 ? wrap1(z + L::c(i, 2), nz) : 0;
            const double v = ls[sx + nx * (sy + ny * sz)];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (L::c(i, a) != 0) g[a] += 3.0 * L::w(i) * double(L::c(i, a)) * v;
        }
        const int64_t gi = S.site_offset + site;
        const double half = 0.5 * S.kappa * (S.rho_c + d[gi]);
#pragma unroll
        for (int a = 0; a < L::D; ++a) jf[a * stride + gi] += half * g[a];
    }
}

__global__ void __launch_bounds__(AUX_THREADS)
    sk_bin_kernel(const SkSys* __restrict__ skv, int sys, const double* __restrict__ acc, double* __restrict__ sums,
                  double* __restrict__ counts) {
    __shared__ double sh[2 * AUX_THREADS];
    const SkSys K = skv[sys];
    const int bin = blockIdx.x + 1;                    // shells j = 1 .. nbins
    const int64_t n = int64_t(K.nx) * K.ny * K.nz;
    double v[2] = {0.0, 0.0};
    const int64_t lo = int64_t(bin) * (bin - 1), hi = int64_t(bin) * (bin + 1);
    for (int64_t e = threadIdx.x; e < n; e += AUX_THREADS) {
        const int kx = int(e % K.nx), ky = int((e / K.nx) % K.ny), kz = int(e / (int64_t(K.nx) * K.ny));
        const int64_t a = wrapk(kx, K.nx), b = wrapk(ky, K.ny), c = wrapk(kz, K.nz);
        const int64_t n2 = a * a + b * b + c * c;
        if (n2 > lo && n2 <= hi) {
            v[0] += acc[K.site_offset + e];
            v[1] += 1.0;
        }
    }
    block_sum<2, AUX_THREADS>(v, sh);
    if (threadIdx.x == 0) {
        sums[blockIdx.x] = v[0];
        counts[blockIdx.x] = v[1];
    }
}

}  // namespace

cudaError_t launch_sk_twiddles(double* tw, const int* sides, const int* offs, int n_tables, int max_n,
                               cudaStream_t st) {
    if (n_tables == 0) return cudaSuccess;
    dim3 grid((max_n + 255) / 256, n_tables);
    sk_twiddle_kernel<<<grid, 256, 0, st>>>(tw, sides, offs, n_tables, max_n);
    return cudaGetLastError();
}

cudaError_t launch_sk_x(const SysDev* sys, const SkSys* sk, const int4* items, int n_items, const double* d,
                        const double* dbar, const double* tw, double* out, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    sk_x_kernel<<<n_items, AUX_THREADS, 0, st>>>(sys, sk, items, d, dbar, tw, out);
    return cudaGetLastError();
}

cudaError_t launch_sk_pass(const SkSys* sk, const int4* items, int n_items, int axis, const double* tw,
                           const double* in, double* out, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    sk_pass_kernel<<<n_items, AUX_THREADS, 0, st>>>(sk, items, axis, tw, in, out);
    return cudaGetLastError();
}

bool sk_fft_side(int n) {
    if (n < 1 || n > kSkFftMaxElems) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

cudaError_t launch_sk_fft(const SysDev* sys, const SkSys* sk, const int4* items, int n_items, int axis,
                          const double* d, const double* dbar, const double* in, const double* tw, double* out,
                          int max_elems, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const size_t dyn = size_t(2) * max_elems * sizeof(double2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sk_fft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(2 * kSkFftMaxElems * sizeof(double2)));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sk_fft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(2 * kSkFftMaxElems * sizeof(double2)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const double2* tw2 = reinterpret_cast<const double2*>(tw);
    double2* out2 = reinterpret_cast<double2*>(out);
    if (in == nullptr)
        sk_fft_kernel<true><<<n_items, AUX_THREADS, dyn, st>>>(sys, sk, items, axis, d, dbar, nullptr, tw2, out2);
    else
        sk_fft_kernel<false><<<n_items, AUX_THREADS, dyn, st>>>(sys, sk, items, axis, nullptr, nullptr,
                                                                reinterpret_cast<const double2*>(in), tw2, out2);
    return cudaGetLastError();
}

cudaError_t launch_sk_accum(const SkSys* sk, const int4* items, int n_items, const double* F, double* acc,
                            cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    sk_accum_kernel<<<n_items, AUX_THREADS, 0, st>>>(sk, items, F, acc);
    return cudaGetLastError();
}

cudaError_t launch_jk_accum(const SkSys* sk, const int4* items, int n_items, int dims, const double* F0,
                            const double* F1, const double* F2, double* acc, int64_t stride, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    jk_accum_kernel<<<n_items, AUX_THREADS, 0, st>>>(sk, items, dims, F0, F1, F2, acc, stride);
    return cudaGetLastError();
}

cudaError_t launch_jk_guo_force(int lattice, const SysDev* sys, const int4* items, int n_items, const double* d,
                                double* lap, double* jf, int64_t stride, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    if (lattice == 0) {
        jk_lap_kernel<D2Q9><<<n_items, AUX_THREADS, 0, st>>>(sys, items, d, lap);
        jk_force_kernel<D2Q9><<<n_items, AUX_THREADS, 0, st>>>(sys, items, d, lap, jf, stride);
    } else {
        jk_lap_kernel<D3Q19><<<n_items, AUX_THREADS, 0, st>>>(sys, items, d, lap);
        jk_force_kernel<D3Q19><<<n_items, AUX_THREADS, 0, st>>>(sys, items, d, lap, jf, stride);
    }
    return cudaGetLastError();
}

cudaError_t launch_sk_bin(const SkSys* sk, int sys, const double* acc, int nbins, double* sums, double* counts,
                          cudaStream_t st) {
    if (nbins <= 0) return cudaSuccess;
    sk_bin_kernel<<<nbins, AUX_THREADS, 0, st>>>(sk, sys, acc, sums, counts);
    return cudaGetLastError();
}

}  // namespace lbf

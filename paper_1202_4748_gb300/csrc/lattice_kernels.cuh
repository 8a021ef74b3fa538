// Lattice-dependent auxiliary kernels: initial equilibrium, population
// gather/scatter for host I/O, and the per-site pass of the observables.
// All reductions are fixed-order (per thread sequential, then a warp-shuffle
// tree and a cross-warp stage), so results are bitwise reproducible run to run.
#pragma once

#include "lb_device.cuh"
#include "lb_launch.h"

namespace lbf {

// Work item of a site pass: (system, first site, end site, unused).
// Deterministic sum of K doubles over the CTA; result valid in thread 0.
template <int K, int NT>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sh /* >= K * NT / 32 */) {
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // within each warp: shuffle-down tree (fixed order, so the sum is reproducible)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh[k * NW + w] = v[k];
    }
    __syncthreads();
    // across warps: warp 0 reduces the NW partial sums the same way
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = lane < NW ? sh[k * NW + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
}

__device__ __forceinline__ void site_coords(int site, int nx, int ny, int& x, int& y, int& z) {
    x = site % nx;
    const int r = site / nx;
    y = r % ny;
    z = r / ny;
}

// f = f^eq(rho, u = 0, grad rho) at every site, written to the pull layout:
// buf_i(r - c_i) = f_i(r, 0).  rho = rho_c + d - dbar (d in FP64 scratch).
template <class L, int CP, class Real>
__global__ void __launch_bounds__(AUX_THREADS)
    init_feq_kernel(const SysDev* __restrict__ sysv, const int4* __restrict__ items, const double* __restrict__ d,
                    const double* __restrict__ dbar, Real* __restrict__ fbuf) {
    const int4 it = items[blockIdx.x];
    const SysDev& S = sysv[it.x];
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const int64_t N = S.n_sites;
    const double* ds = d + S.site_offset;
    const double db = dbar[it.x];
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int site = it.y + j * AUX_THREADS + threadIdx.x;
        if (site >= it.z) break;
        int x, y, z;
        site_coords(site, nx, ny, x, y, z);
        // wrapped neighbour coordinates x + d (d = -1, 0, 1) and their offsets
        const int X[3] = {wrap1(x - 1, nx), x, wrap1(x + 1, nx)};
        const int Y[3] = {wrap1(y - 1, ny) * nx, y * nx, wrap1(y + 1, ny) * nx};
        const int Z[3] = {L::D == 3 ? wrap1(z - 1, nz) * nx * ny : 0, z * nx * ny,
                          L::D == 3 ? wrap1(z + 1, nz) * nx * ny : 0};
        auto nb = [&](int i) { return ds[X[1 + L::c(i, 0)] + Y[1 + L::c(i, 1)] + Z[1 + L::c(i, 2)]] - db; };
        const double drho = ds[site] - db;
        const double rho = S.rho_c + drho;
        const double phi = drho * S.inv_rho_c;
        const double df0 = phi * (S.a + S.b * phi * phi);
        const double f0 = phi * phi * (0.5 * S.a + 0.25 * S.b * phi * phi);
        const double p0 = rho * S.inv_rho_c * df0 - f0;
        double feq[L::Q];
        double s = 0.0;
        if constexpr (CP == MODEQ && L::D == 2) {
            double gx = 0.0, gy = 0.0, lap = 0.0;
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const double rn = nb(i);
                gx += 3.0 * L::w(i) * L::c(i, 0) * rn;
                gy += 3.0 * L::w(i) * L::c(i, 1) * rn;
                lap += 6.0 * L::w(i) * (rn - drho);
            }
            const double iso = p0 - S.kappa * rho * lap;
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                feq[i] = pooley_w(i) * iso +
                         S.kappa * (pooley_wxx(i) * gx * gx + pooley_wyy(i) * gy * gy + pooley_wxy(i) * gx * gy);
                s += feq[i];
            }
        } else if constexpr (CP == MODEQ) {
            // D3Q19 modified equilibrium at rest: 3 t_i iso + kappa t_i [(9/2)(c.g)^2 - (9/2) c^2 |g|^2 + (9/2)|g|^2]
            double g[3] = {0.0, 0.0, 0.0}, lap = 0.0;
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const double rn = nb(i);
#pragma unroll
                for (int a = 0; a < 3; ++a) g[a] += 3.0 * L::w(i) * L::c(i, a) * rn;
                lap += 6.0 * L::w(i) * (rn - drho);
            }
            const double iso = p0 - S.kappa * rho * lap;
            const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const double cg = L::c(i, 0) * g[0] + L::c(i, 1) * g[1] + L::c(i, 2) * g[2];
                const double c2 = double(L::c(i, 0) * L::c(i, 0) + L::c(i, 1) * L::c(i, 1) + L::c(i, 2) * L::c(i, 2));
                feq[i] = 3.0 * L::w(i) * iso + S.kappa * L::w(i) * (4.5 * cg * cg - 4.5 * c2 * g2 + 4.5 * g2);
                s += feq[i];
            }
        } else {
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                feq[i] = 3.0 * L::w(i) * p0;
                s += feq[i];
            }
        }
        feq[0] = drho - s;
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            fbuf[S.pop_offset + int64_t(i) * N + (X[1 - L::c(i, 0)] + Y[1 - L::c(i, 1)] + Z[1 - L::c(i, 2)])] =
                Real(feq[i]);
    }
}

// out[site] = f_i(r, t) = buf_i(r - c_i) + rho_c [i == 0], one population.
template <class L, class Real>
__global__ void __launch_bounds__(AUX_THREADS)
    gather_kernel(const SysDev* __restrict__ sysv, int sys, int i, const Real* __restrict__ fbuf,
                  double* __restrict__ out) {
    const SysDev& S = sysv[sys];
    const int64_t site = int64_t(blockIdx.x) * AUX_THREADS + threadIdx.x;
    if (site >= S.n_sites) return;
    int x, y, z;
    site_coords(int(site), S.nx, S.ny, x, y, z);
    int cx = 0, cy = 0, cz = 0;
#pragma unroll
    for (int q = 0; q < L::Q; ++q)
        if (q == i) {
            cx = L::c(q, 0);
            cy = L::c(q, 1);
            cz = L::c(q, 2);
        }
    const int sx = wrapm(x - cx, S.nx), sy = wrapm(y - cy, S.ny), sz = wrapm(z - cz, S.nz);
    const double v = double(fbuf[S.pop_offset + int64_t(i) * S.n_sites + (sx + S.nx * (sy + S.ny * sz))]);
    out[site] = v + (i == 0 ? S.rho_c : 0.0);
}

// buf_i(r - c_i) = f_i(r) - rho_c [i == 0], one population.
template <class L, class Real>
__global__ void __launch_bounds__(AUX_THREADS)
    scatter_kernel(const SysDev* __restrict__ sysv, int sys, int i, const double* __restrict__ in,
                   Real* __restrict__ fbuf) {
    const SysDev& S = sysv[sys];
    const int64_t site = int64_t(blockIdx.x) * AUX_THREADS + threadIdx.x;
    if (site >= S.n_sites) return;
    int x, y, z;
    site_coords(int(site), S.nx, S.ny, x, y, z);
    int cx = 0, cy = 0, cz = 0;
#pragma unroll
    for (int q = 0; q < L::Q; ++q)
        if (q == i) {
            cx = L::c(q, 0);
            cy = L::c(q, 1);
            cz = L::c(q, 2);
        }
    const int sx = wrapm(x - cx, S.nx), sy = wrapm(y - cy, S.ny), sz = wrapm(z - cz, S.nz);
    fbuf[S.pop_offset + int64_t(i) * S.n_sites + (sx + S.nx * (sy + S.ny * sz))] =
        Real(in[site] - (i == 0 ? S.rho_c : 0.0));
}

// Compensated sum (Knuth's TwoSum): s + c carries the exact sum of the added
// values up to the rounding of c, i.e. to about eps^2 relative.
template <class Real>
struct CompSum {
    Real s = Real(0), c = Real(0);
    __device__ __forceinline__ void add(Real v) {
        const Real t = s + v;
        const Real bp = t - s;
        c += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// Observable site pass: d(r) = rho(r, t) - rho_c = sum_i delta f_i(r - c_i) and
// j(r) = sum_i c_i f_i(r - c_i), to FP64 accuracy (FP64 sums for FP64 storage;
// compensated FP32 sums for FP32 storage, which keeps the per-population work
// off the FP64 pipe).  Writes d and per-item partial sums (sum d, sum jx,
// sum jy, sum jz) in FP64, and, when jout is not null, the momentum field
// j_a(r) at jout + a * jstride (D components).
template <class L, class Real>
__global__ void __launch_bounds__(AUX_THREADS)
    obs_site_kernel(const SysDev* __restrict__ sysv, const int4* __restrict__ items, const Real* __restrict__ fbuf,
                    double* __restrict__ d, double* __restrict__ partial, double* __restrict__ jout,
                    int64_t jstride) {
    __shared__ double sh[4 * AUX_THREADS];
    const int4 it = items[blockIdx.x];
    const SysDev& S = sysv[it.x];
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const Real* fb = fbuf + S.pop_offset;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int site = it.y + j * AUX_THREADS + threadIdx.x;
        if (site >= it.z) break;
        int x, y, z;
        site_coords(site, nx, ny, x, y, z);
        CompSum<Real> r, m[3];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const int sx = wrap1(x - L::c(i, 0), nx), sy = wrap1(y - L::c(i, 1), ny);
            const int sz = L::D == 3 ? wrap1(z - L::c(i, 2), nz) : 0;
            const Real v = fb[int64_t(i) * S.n_sites + (sx + nx * (sy + ny * sz))];
            r.add(v);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (L::c(i, a) == 1) m[a].add(v);
                if (L::c(i, a) == -1) m[a].add(-v);
            }
        }
        const double rv = r.value();
        d[S.site_offset + site] = rv;
        if (jout) {
#pragma unroll
            for (int a = 0; a < L::D; ++a) jout[a * jstride + S.site_offset + site] = m[a].value();
        }
        acc[0] += rv;
        acc[1] += m[0].value();
        acc[2] += m[1].value();
        acc[3] += m[2].value();
    }
    block_sum<4, AUX_THREADS>(acc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) partial[int64_t(blockIdx.x) * 4 + k] = acc[k];
    }
}

}  // namespace lbf

// Perturbation-theory comparator (Sec. II C): the lattice sums over q != 0 of
// the self-consistent equations for r' (Eq. 36) and, below the critical point,
// v and r'_sigma (Eqs. 40, 42, 43), evaluated on the device, with the root
// finding on the host.
//
// G(q) = 1 / (m + kappa q^2) on the S^d wavevector grid, q^2 the symbol of the
// lattice Laplacian 6 sum_i t_i (1 - cos q.c_i), G = 0 at the zero mode.
//   S1   = N^-1 sum_q G(q),   S1sq = N^-1 sum_q G(q)^2,
//   S2   = N^-2 sum_{q1, q2} G(q1) G(q2) G(q1 + q2)  (zero-mode terms vanish)
//        = sum_r g(r)^3,  g = inverse DFT of G (convolution theorem); G is real
//          and even, so the forward transform the structure-factor passes take
//          equals N g, and S2 costs O(N S d) instead of O(N^2).
// Partial sums are per CTA and added on the host in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/lbfluct.h"
#include "lattice_kernels.cuh"
#include "lb_launch.h"

namespace lbf {

namespace {

constexpr int PT_ELEMS = SITES_PER_THREAD * AUX_THREADS;   // elements per CTA

template <class L>
__global__ void __launch_bounds__(AUX_THREADS)
    pt_prop_kernel(const int4* __restrict__ items, SkSys K, double m, double kappa, double* __restrict__ G,
                   double* __restrict__ partial) {
    __shared__ double sh[2 * AUX_THREADS];
    const int4 it = items[blockIdx.x];
    double acc[2] = {0.0, 0.0};
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int e = it.y + j * AUX_THREADS + threadIdx.x;
        if (e >= it.z) break;
        const int kx = e % K.nx, ky = (e / K.nx) % K.ny, kz = e / (K.nx * K.ny);
        const int n[3] = {2 * kx < K.nx ? kx : kx - K.nx, 2 * ky < K.ny ? ky : ky - K.ny,
                          2 * kz < K.nz ? kz : kz - K.nz};
        double g = 0.0;
        if (e != 0) {
            double q2 = 0.0;
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const int nc = n[0] * L::c(i, 0) + n[1] * L::c(i, 1) + (L::D == 3 ? n[2] * L::c(i, 2) : 0);
                q2 += 6.0 * L::w(i) * (1.0 - cospi(2.0 * double(nc) / double(K.nx)));
            }
            g = 1.0 / (m + kappa * q2);
        }
        G[e] = g;
        acc[0] += g;
        acc[1] += g * g;
    }
    block_sum<2, AUX_THREADS>(acc, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = acc[0];
        partial[2 * blockIdx.x + 1] = acc[1];
    }
}

__global__ void __launch_bounds__(AUX_THREADS)
    pt_cube_kernel(const int4* __restrict__ items, double inv_n, const double* __restrict__ F,
                   double* __restrict__ partial) {
    __shared__ double sh[AUX_THREADS];
    const int4 it = items[blockIdx.x];
    double acc[1] = {0.0};
    for (int j = 0; j < SITES_PER_THREAD; ++j) {
        const int e = it.y + j * AUX_THREADS + threadIdx.x;
        if (e >= it.z) break;
        const double g = F[2 * int64_t(e)] * inv_n;
        acc[0] += g * g * g;
    }
    block_sum<1, AUX_THREADS>(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc[0];
}

size_t align_pt(size_t x) { return (x + 255) & ~size_t(255); }

struct PtPlan {
    int lattice = 0, side = 0, dims = 0;
    int64_t n = 0;
    int n_items = 0;
    size_t sys, sk, items, meta, tw, G, b0, b1, part2, part1, total;
};

bool make_pt_plan(int lattice, int side, PtPlan& P) {
    if ((lattice != LB_D2Q9 && lattice != LB_D3Q19) || side < 2 || side > 65536) return false;
    P.lattice = lattice;
    P.side = side;
    P.dims = lattice == LB_D3Q19 ? 3 : 2;
    P.n = int64_t(side) * side * (P.dims == 3 ? side : 1);
    if (P.n > (int64_t(1) << 28)) return false;
    P.n_items = int((P.n + PT_ELEMS - 1) / PT_ELEMS);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_pt(off + (bytes ? bytes : 1));
        return at;
    };
    P.sys = take(sizeof(SysDev));
    P.sk = take(sizeof(SkSys));
    P.items = take(sizeof(int4) * P.n_items);
    P.meta = take(sizeof(int) * 2);
    P.tw = take(sizeof(double) * 2 * side);
    P.G = take(sizeof(double) * P.n);
    P.b0 = take(sizeof(double) * 2 * P.n);
    P.b1 = take(sizeof(double) * 2 * P.n);
    P.part2 = take(sizeof(double) * 2 * P.n_items);
    P.part1 = take(sizeof(double) * P.n_items);
    P.total = off;
    return true;
}

struct PtCtx {
    PtPlan P;
    char* ws;
    cudaStream_t st;
    std::vector<double> h2, h1;
    template <class T>
    T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
};

SkSys sk_of(const PtPlan& P) {
    SkSys K;
    std::memset(&K, 0, sizeof(K));
    K.nx = P.side;
    K.ny = P.side;
    K.nz = P.dims == 3 ? P.side : 1;
    K.tw_x = K.tw_y = K.tw_z = 0;                  // one table: every side is S
    K.site_offset = 0;
    K.inv_n = 1.0 / double(P.n);
    return K;
}

// Descriptors, work items and the twiddle table into the workspace.
cudaError_t pt_setup(PtCtx& c) {
    const PtPlan& P = c.P;
    SysDev sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.nx = P.side;
    sd.ny = P.side;
    sd.nz = P.dims == 3 ? P.side : 1;
    sd.rho_c = 1.0;
    const SkSys K = sk_of(P);
    std::vector<int4> items(P.n_items);
    for (int k = 0; k < P.n_items; ++k) {
        const int64_t a = int64_t(k) * PT_ELEMS;
        items[k] = make_int4(0, int(a), int(std::min<int64_t>(a + PT_ELEMS, P.n)), 0);
    }
    const int meta[2] = {P.side, 0};
    cudaError_t e = cudaMemcpyAsync(c.ws + P.sys, &sd, sizeof(sd), cudaMemcpyHostToDevice, c.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.ws + P.sk, &K, sizeof(K), cudaMemcpyHostToDevice, c.st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.ws + P.items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, c.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.ws + P.meta, meta, sizeof(meta), cudaMemcpyHostToDevice, c.st);
    if (e == cudaSuccess) e = launch_sk_twiddles(c.at<double>(P.tw), c.at<int>(P.meta), c.at<int>(P.meta) + 1, 1,
                                                 P.side, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);   // host arrays above go out of scope
    return e;
}

// S1, S1sq (and S2 when want_s2) at propagator mass m.
cudaError_t pt_eval(PtCtx& c, double m, double kappa, bool want_s2, double& S1, double& S1sq, double& S2) {
    const PtPlan& P = c.P;
    const SkSys K = sk_of(P);
    const int4* items = c.at<int4>(P.items);
    if (P.lattice == LB_D2Q9)
        pt_prop_kernel<D2Q9><<<P.n_items, AUX_THREADS, 0, c.st>>>(items, K, m, kappa, c.at<double>(P.G),
                                                                    c.at<double>(P.part2));
    else
        pt_prop_kernel<D3Q19><<<P.n_items, AUX_THREADS, 0, c.st>>>(items, K, m, kappa, c.at<double>(P.G),
                                                                     c.at<double>(P.part2));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && want_s2) {
        const SysDev* sys = c.at<SysDev>(P.sys);
        const SkSys* sk = c.at<SkSys>(P.sk);
        const double* tw = c.at<double>(P.tw);
        double* b0 = c.at<double>(P.b0);
        double* b1 = c.at<double>(P.b1);
        e = launch_sk_x(sys, sk, items, P.n_items, c.at<double>(P.G), nullptr, tw, b0, c.st);
        if (e == cudaSuccess) e = launch_sk_pass(sk, items, P.n_items, 1, tw, b0, b1, c.st);
        const double* fin = b1;
        if (e == cudaSuccess && P.dims == 3) {
            e = launch_sk_pass(sk, items, P.n_items, 2, tw, b1, b0, c.st);
            fin = b0;
        }
        if (e == cudaSuccess) {
            pt_cube_kernel<<<P.n_items, AUX_THREADS, 0, c.st>>>(items, 1.0 / double(P.n), fin, c.at<double>(P.part1));
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.h2.data(), c.ws + P.part2, sizeof(double) * 2 * P.n_items, cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess && want_s2)
        e = cudaMemcpyAsync(c.h1.data(), c.ws + P.part1, sizeof(double) * P.n_items, cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return e;
    double s = 0, s2 = 0, s3 = 0;
    for (int k = 0; k < P.n_items; ++k) {
        s += c.h2[2 * k];
        s2 += c.h2[2 * k + 1];
        if (want_s2) s3 += c.h1[k];
    }
    S1 = s / double(P.n);
    S1sq = s2 / double(P.n);
    S2 = want_s2 ? s3 : NAN;
    return cudaSuccess;
}

lb_status open_pt(int lattice, int side, void* ws, size_t bytes, void* stream, PtCtx& c) {
    if (!make_pt_plan(lattice, side, c.P)) return LB_ERR_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || bytes < c.P.total) return LB_ERR_WORKSPACE;
    c.ws = static_cast<char*>(ws);
    c.st = static_cast<cudaStream_t>(stream);
    c.h2.assign(2 * size_t(c.P.n_items), 0.0);
    c.h1.assign(size_t(c.P.n_items), 0.0);
    return pt_setup(c) == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

// Bisection on [lo, hi] with fn(lo) > 0 >= fn(hi) (or the reverse), as the oracle does.
template <class Fn>
lb_status bisect(Fn&& fn, double lo, double hi, double& root) {
    double flo;
    if (!fn(lo, flo)) return LB_ERR_CUDA;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        double fm;
        if (!fn(mid, fm)) return LB_ERR_CUDA;
        if ((fm > 0) == (flo > 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    root = 0.5 * (lo + hi);
    return LB_OK;
}

// smallest non-zero Laplacian symbol on the grid (at n = (1, 0, 0))
double q2_min(int lattice, int side) {
    const double c1 = 1.0 - std::cos(6.283185307179586476925286766559 / side);
    if (lattice == LB_D2Q9) return 6.0 * (2.0 / 9.0 * c1 + 4.0 / 36.0 * c1);
    return 6.0 * (2.0 / 18.0 * c1 + 8.0 / 36.0 * c1);
}

}  // namespace

}  // namespace lbf

using namespace lbf;

extern "C" {

lb_status lb_pt_workspace_bytes(int lattice, int side, size_t* bytes) {
    PtPlan P;
    if (!bytes || !make_pt_plan(lattice, side, P)) return LB_ERR_ARG;
    *bytes = P.total;
    return LB_OK;
}

lb_status lb_pt_sums(int lattice, int side, double m, double kappa, void* ws, size_t bytes, void* stream,
                     double out[3]) {
    if (!out || !(m > 0) || !(kappa >= 0) || !std::isfinite(m) || !std::isfinite(kappa)) return LB_ERR_ARG;
    PtCtx c;
    lb_status s = open_pt(lattice, side, ws, bytes, stream, c);
    if (s != LB_OK) return s;
    if (pt_eval(c, m, kappa, true, out[0], out[1], out[2]) != cudaSuccess) return LB_ERR_CUDA;
    return LB_OK;
}

lb_status lb_pt_symmetric(int lattice, int side, double r, double u, double kappa, double kT, void* ws,
                          size_t bytes, void* stream, double out[5]) {
    if (!out || !std::isfinite(r) || !(u >= 0) || !(kappa >= 0) || !(kT >= 0) || !std::isfinite(u) ||
        !std::isfinite(kappa) || !std::isfinite(kT))
        return LB_ERR_ARG;
    PtCtx c;
    lb_status s = open_pt(lattice, side, ws, bytes, stream, c);
    if (s != LB_OK) return s;
    double S1, S1sq, S2;
    auto F = [&](double m, double& f) {
        if (pt_eval(c, m, kappa, true, S1, S1sq, S2) != cudaSuccess) return false;
        f = r + 3.0 * u * kT * S1 - 6.0 * u * u * kT * kT * S2 - m;
        return true;
    };
    double hi = 1.01 * 0.5 * (std::max(r, 0.0) + std::sqrt(r * r + 12.0 * u * kT));
    if (!(hi > 0)) return LB_ERR_NO_ROOT;
    double lo = hi;
    for (;;) {
        lo *= 0.5;
        double f;
        if (!F(lo, f)) return LB_ERR_CUDA;
        if (!std::isfinite(f) || lo < 1e-300) return LB_ERR_NO_ROOT;
        if (f > 0) break;
        hi = lo;
    }
    double rp;
    s = bisect(F, lo, hi, rp);
    if (s != LB_OK) return s;
    double f;
    if (!F(rp, f)) return LB_ERR_CUDA;
    out[0] = rp;
    out[1] = 1.0 / rp;
    out[2] = std::sqrt(kappa / rp);
    out[3] = S1;
    out[4] = S2;
    return LB_OK;
}

lb_status lb_pt_broken(int lattice, int side, double r, double u, double kappa, double kT, void* ws,
                       size_t bytes, void* stream, double out[7]) {
    if (!out || !(r < 0) || !(u > 0) || !(kappa >= 0) || !(kT >= 0) || !std::isfinite(r) || !std::isfinite(u) ||
        !std::isfinite(kappa) || !std::isfinite(kT))
        return LB_ERR_ARG;
    PtCtx c;
    lb_status s = open_pt(lattice, side, ws, bytes, stream, c);
    if (s != LB_OK) return s;
    double S1, S1sq, S2;
    auto h = [&](double w, double& f) {
        if (pt_eval(c, r + 3.0 * u * w, kappa, false, S1, S1sq, S2) != cudaSuccess) return false;
        f = r + u * w + 3.0 * u * kT * S1;
        return true;
    };
    const double w_mf = -r / u;
    const double w_low = std::max(0.0, (-r - kappa * q2_min(lattice, side)) / (3.0 * u));
    double w_pos = w_mf, w = w_mf, w_neg = NAN;
    for (int it = 0; it < 200; ++it) {
        w = w_low + 0.5 * (w - w_low);
        double f;
        if (!h(w, f)) return LB_ERR_CUDA;
        if (f < 0) {
            w_neg = w;
            break;
        }
        w_pos = w;
    }
    if (std::isnan(w_neg)) return LB_ERR_NO_ROOT;
    s = bisect(h, w_neg, w_pos, w);
    if (s != LB_OK) return s;
    const double rs = r + 3.0 * u * w;
    if (pt_eval(c, rs, kappa, false, S1, S1sq, S2) != cudaSuccess) return LB_ERR_CUDA;
    const double rps = rs + kT * (-18.0 * u * u * w * kT * S1sq + 3.0 * u * S1);
    out[0] = std::sqrt(w);
    out[1] = rs;
    out[2] = rps;
    out[3] = 1.0 / rps;
    out[4] = std::sqrt(kappa / rps);
    out[5] = S1;
    out[6] = S1sq;
    return LB_OK;
}

}  // extern "C"

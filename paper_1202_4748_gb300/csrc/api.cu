// C ABI of the fluctuating lattice Boltzmann library (declared in include/lbfluct.h).
//
// Host responsibilities: validate descriptors, carve the caller's device
// workspace, build the work lists (step tiles, site chunks, observable block
// items), order the launches on the caller's stream, optionally capture step
// chunks in CUDA graphs, and move data between host and device for I/O.
// Every arithmetic step of the method runs in the kernels.
#include <array>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbfluct.h"
#include "lb_launch.h"

using namespace lbf;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct LevelHost {
    int bx, by, bz, gx, gy, gz;
    int64_t nblocks;
    bool pyramid;   // part of the halving pyramid (else: the separate single-site level)
};

struct SysHost {
    lb_system_desc d;
    int64_t n = 0, site_off = 0, pop_off = 0;
    std::vector<LevelHost> lv;
    int imax = 0;          // bottom pyramid level index
    bool unit_sep = false; // single-site level appended after the pyramid
    int lv_first = 0;      // index of level 0 in the flattened LevelDev array
};

// Byte offsets of every region inside the workspace.
struct Plan {
    size_t sys, phys, tiles, pop0, pop1, step, status, d, dbar, site_items, site_partial, spans, red4, glob, levels,
        S, E, bottom_items, up_items, rec, acc, hist, field_tmp, sk_sys, sk_tw, sk_acc, sk_b0, sk_b1, sk_bins, jk_j,
        jk_lap, jk_F, jk_acc, total;
    bool jk = false;
    int hist_bins = 0;
    double hist_range = 0.0;
    int n_tiles = 0, n_site_items = 0, n_levels = 0, n_bottom = 0, n_up = 0, n_rec = 0, max_depth = 0;
    int64_t n_sites = 0, n_blocks_pyr = 0, max_sites = 0;
    std::vector<int4> tiles_h, site_items_h;
    std::vector<SysSpan> spans_h;
    std::vector<LevelDev> levels_h;
    std::vector<ObsItem> bottom_h, up_h;
    std::vector<int> up_first;   // up items of depth u: [up_first[u-1], up_first[u])
    // structure factor
    bool sk = false;
    std::vector<SkSys> sk_h;
    std::vector<int> tw_sides, tw_offs;
    int tw_total = 0, tw_max = 0, sk_max_bins = 0;
    // line-FFT work list of the structure factor (every side 2^a 3^b), else the direct sums
    bool sk_fft = false;
    std::vector<int4> fft_items_h;
    int n_fft_items = 0, fft_max_elems = 0;
    size_t fft_items = 0;
};

int q_of(int lattice) { return lattice == LB_D2Q9 ? 9 : 19; }

lb_status validate(const lb_system_desc* s, int n, const lb_run_opts* o) {
    if (!s || n <= 0 || !o) return LB_ERR_ARG;
    if (o->precision != LB_FP64 && o->precision != LB_FP32_DEVIATION) return LB_ERR_ARG;
    if (o->obs_every < 0 || o->sk_every < 0 || o->graph_chunk < 0 || (o->graph_chunk & 1)) return LB_ERR_ARG;
    if (o->hist_bins < 0 || o->hist_bins > LB_MAX_HIST_BINS) return LB_ERR_ARG;
    if (o->jk_spectra != 0 && (o->jk_spectra != 1 || o->sk_every == 0)) return LB_ERR_ARG;
    if (o->hist_bins > 0 && !(o->hist_range > 0 && std::isfinite(o->hist_range))) return LB_ERR_ARG;
    for (int k = 0; k < n; ++k) {
        const lb_system_desc& d = s[k];
        if (d.lattice != s[0].lattice || d.coupling != s[0].coupling) return LB_ERR_ARG;
        if (d.lattice != LB_D2Q9 && d.lattice != LB_D3Q19) return LB_ERR_ARG;
        if (d.coupling != LB_MODEQ && d.coupling != LB_GUO) return LB_ERR_ARG;
        if (d.nx < 1 || d.ny < 1 || d.nz < 1) return LB_ERR_ARG;
        if (d.lattice == LB_D2Q9 && d.nz != 1) return LB_ERR_ARG;
        if (int64_t(d.nx) * d.ny * d.nz * q_of(d.lattice) >= (int64_t(1) << 31)) return LB_ERR_ARG;
        if (!(d.rho_c > 0) || !std::isfinite(d.a) || !std::isfinite(d.b) || !(d.kappa >= 0) || !(d.kT >= 0) ||
            !std::isfinite(d.kT) || !std::isfinite(d.kappa))
            return LB_ERR_ARG;
        if (d.system_id >= (1u << 24)) return LB_ERR_ARG;
        if (o->sk_every > 0 && (d.nx != d.ny || (d.lattice == LB_D3Q19 && d.nz != d.nx))) return LB_ERR_UNSUPPORTED;
        const int q = q_of(d.lattice), nc = d.lattice == LB_D2Q9 ? 3 : 4;
        for (int a = nc; a < q; ++a)
            if (!(d.tau[a] > 0.5) || !std::isfinite(d.tau[a])) return LB_ERR_ARG;
    }
    return LB_OK;
}

std::vector<LevelHost> make_levels(const lb_system_desc& d, int& imax, bool& unit_sep) {
    const bool dims3 = d.lattice == LB_D3Q19;
    std::vector<LevelHost> out;
    for (int i = 0;; ++i) {
        const int64_t p = int64_t(1) << i;
        if (d.nx % p || d.ny % p || (dims3 && d.nz % p)) break;
        LevelHost L;
        L.bx = int(d.nx / p);
        L.by = int(d.ny / p);
        L.bz = dims3 ? int(d.nz / p) : 1;
        L.gx = int(p);
        L.gy = int(p);
        L.gz = dims3 ? int(p) : 1;
        L.nblocks = int64_t(L.gx) * L.gy * L.gz;
        L.pyramid = true;
        out.push_back(L);
        if (L.bx == 1 && L.by == 1 && L.bz == 1) break;
        if (i > 30) break;
    }
    imax = int(out.size()) - 1;
    unit_sep = !(out.back().bx == 1 && out.back().by == 1 && out.back().bz == 1);
    if (unit_sep) {
        LevelHost L;
        L.bx = L.by = L.bz = 1;
        L.gx = d.nx;
        L.gy = d.ny;
        L.gz = d.nz;
        L.nblocks = int64_t(d.nx) * d.ny * d.nz;
        L.pyramid = false;
        out.push_back(L);
    }
    return out;
}

static_assert(kVariantCols == LB_VARIANT_COLS, "variant rows of the ABI");

int tile_table(int lattice, int (*t)[kVariantCols]) {
    return lattice == LB_D2Q9 ? tile_shapes_d2q9(t, 32) : tile_shapes_d3q19(t, 32);
}

// The variant given by index, else the first compiled variant matching the
// requested shape (and occupancy, if given), else the default: the first
// variant the coupling runs (row-marching strips, scheme 2, are compiled for
// the modified equilibrium only).  zm_default: the modified equilibrium on
// D3Q19 where the paired kernel cannot run (FP64, a rate other than 1, an nx
// that is not a multiple of 4) runs the radius-1 z-marching kernel whatever
// the row, so its default is the first row of the plain z-marching kernel
// (no producer warps), whose tile shape and budget suit it best (16 x 8
// columns at 6 CTAs per SM: 0.563 ms on the 160-system ensemble against
// 0.645 ms with the paired kernel's tile).
lb_status choose_tile(int lattice, int coupling, const lb_run_opts* o, int& tile_id, int tdim[3],
                      bool zm_default = false) {
    int t[32][kVariantCols];
    const int nt = tile_table(lattice, t);
    auto runs = [&](int k) { return t[k][5] != 2 || coupling == LB_MODEQ; };
    const bool defaults = o->tile[0] <= 0 && o->occupancy <= 0;
    auto preferred = [&](int k) {
        if (!defaults || !zm_default || lattice != LB_D3Q19 || coupling != LB_MODEQ) return true;
        return t[k][4] == 0 && t[k][5] == 0 && t[k][6] == 1;
    };
    tile_id = 0;
    if (o->variant < 0) return LB_ERR_ARG;
    if (o->variant > 0) {
        if (o->variant > nt || !runs(o->variant - 1)) return LB_ERR_UNSUPPORTED;
        tile_id = o->variant - 1;
    } else {
        tile_id = -1;
        for (int pass = 0; pass < 2 && tile_id < 0; ++pass)
            for (int k = 0; k < nt && tile_id < 0; ++k) {
                const bool shape = o->tile[0] <= 0 || (t[k][0] == o->tile[0] && t[k][1] == o->tile[1] &&
                                                       t[k][2] == (o->tile[2] > 0 ? o->tile[2] : 1));
                const bool occ = o->occupancy <= 0 || t[k][3] == o->occupancy;
                if (shape && occ && runs(k) && (pass == 1 || preferred(k))) tile_id = k;
            }
        if (tile_id < 0) return LB_ERR_UNSUPPORTED;
    }
    for (int k = 0; k < 3; ++k) tdim[k] = t[tile_id][k];
    return LB_OK;
}

// Number of step tiles (CTAs) of a tile shape over the ensemble.
int64_t tiles_of(const lb_system_desc* s, int n, const int tdim[3]) {
    int64_t c = 0;
    for (int k = 0; k < n; ++k)
        c += int64_t((s[k].nx + tdim[0] - 1) / tdim[0]) * ((s[k].ny + tdim[1] - 1) / tdim[1]) *
             ((s[k].nz + tdim[2] - 1) / tdim[2]);
    return c;
}

// Default variant: among the rows that differ from the default row only in
// the z-chunk, the longest chunk whose CTAs still fill the GPU at least twice
// over (resident CTAs per SM x SMs of the current device; 152 SMs when no
// device is visible), else the default row.  Longer chunks re-read fewer
// halo planes (4 per chunk; 2 for the modified equilibrium on D3Q19), but
// too few CTAs leave SMs idle in the last
// wave: on GB300 the 64-plane chunks win on the 160-system ensemble (1,184
// CTAs) and on 256^3 (1,024), the 32-plane ones on 32 systems of 64^3 (512).
void prefer_longer_chunk(const lb_system_desc* s, int n, int& tile_id, int tdim[3]) {
    int t[32][kVariantCols];
    const int nt = tile_table(s[0].lattice, t);
    int sms = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    const int* d = t[tile_id];
    int best = tile_id;
    for (int k = 0; k < nt; ++k) {
        bool same = true;
        for (int c = 0; c < kVariantCols; ++c)
            if (c != 2 && t[k][c] != d[c]) same = false;
        if (!same || t[k][2] <= t[best][2]) continue;
        const int occ = t[k][3] > 0 ? t[k][3] : 1;
        if (tiles_of(s, n, t[k]) >= int64_t(2) * occ * sms) best = k;
    }
    tile_id = best;
    for (int k = 0; k < 3; ++k) tdim[k] = t[best][k];
}

lb_status make_plan(const lb_system_desc* s, int n, const lb_run_opts* o, std::vector<SysHost>& sys, Plan& P,
                    int& tile_id) {
    lb_status st = validate(s, n, o);
    if (st != LB_OK) return st;
    int tdim[3];
    bool paired_runs = o->precision == LB_FP32_DEVIATION;
    for (int k = 0; k < n; ++k) {
        if (s[k].nx % 4 != 0) paired_runs = false;
        for (int a = s[k].lattice == LB_D2Q9 ? 3 : 4; a < q_of(s[k].lattice); ++a)
            if (s[k].tau[a] != 1.0) paired_runs = false;
    }
    st = choose_tile(s[0].lattice, s[0].coupling, o, tile_id, tdim, !paired_runs);
    if (st != LB_OK) return st;
    if (o->variant == 0 && o->tile[0] <= 0 && o->occupancy <= 0) prefer_longer_chunk(s, n, tile_id, tdim);
    const int q = q_of(s[0].lattice);
    const size_t es = o->precision == LB_FP64 ? 8 : 4;
    sys.assign(n, SysHost());
    int64_t site_off = 0;
    int lv_count = 0;
    for (int k = 0; k < n; ++k) {
        SysHost& h = sys[k];
        h.d = s[k];
        h.n = int64_t(s[k].nx) * s[k].ny * s[k].nz;
        h.site_off = site_off;
        h.pop_off = site_off * q;
        site_off += h.n;
        h.lv = make_levels(s[k], h.imax, h.unit_sep);
        h.lv_first = lv_count;
        lv_count += int(h.lv.size());
        P.max_sites = std::max(P.max_sites, h.n);
    }
    P.n_sites = site_off;
    P.n_levels = lv_count;

    // step tiles, system by system; then the longest z-chunks first, so that
    // the last wave of CTAs holds the shortest ones (the tiles are independent)
    for (int k = 0; k < n; ++k) {
        const lb_system_desc& d = s[k];
        for (int z = 0; z < d.nz; z += tdim[2])
            for (int y = 0; y < d.ny; y += tdim[1])
                for (int x = 0; x < d.nx; x += tdim[0]) P.tiles_h.push_back(make_int4(k, x, y, z));
    }
    {
        auto planes = [&](const int4& t) { return std::min(tdim[2], s[t.x].nz - t.w); };
        std::stable_sort(P.tiles_h.begin(), P.tiles_h.end(),
                         [&](const int4& a, const int4& b) { return planes(a) > planes(b); });
    }
    P.n_tiles = int(P.tiles_h.size());

    // site chunks
    const int chunk = AUX_THREADS * SITES_PER_THREAD;
    for (int k = 0; k < n; ++k) {
        SysSpan sp{int(P.site_items_h.size()), 0};
        for (int64_t b = 0; b < sys[k].n; b += chunk)
            P.site_items_h.push_back(make_int4(k, int(b), int(std::min<int64_t>(b + chunk, sys[k].n)), 0));
        sp.count = int(P.site_items_h.size()) - sp.first;
        P.spans_h.push_back(sp);
    }
    P.n_site_items = int(P.site_items_h.size());

    // observable levels, items and records
    const int bchunk = OBS_THREADS * BLOCKS_PER_THREAD;
    int64_t blk_off = 0;
    P.levels_h.resize(lv_count);
    for (int k = 0; k < n; ++k) {
        SysHost& h = sys[k];
        for (size_t l = 0; l < h.lv.size(); ++l) {
            const LevelHost& L = h.lv[l];
            LevelDev& D = P.levels_h[h.lv_first + l];
            D.sys = k;
            D.bx = L.bx;
            D.by = L.by;
            D.bz = L.bz;
            D.gx = L.gx;
            D.gy = L.gy;
            D.gz = L.gz;
            D.nblocks = L.nblocks;
            D.child = (L.pyramid && int(l) < h.imax) ? h.lv_first + int(l) + 1 : -1;
            D.off = L.pyramid ? blk_off : -1;
            if (L.pyramid) blk_off += L.nblocks;
            D.rec_first = 0;
            D.rec_count = 0;
        }
    }
    P.n_blocks_pyr = blk_off;
    int rec = 0;
    // bottom items (records of the bottom level, then of the unit level)
    for (int k = 0; k < n; ++k) {
        SysHost& h = sys[k];
        LevelDev& B = P.levels_h[h.lv_first + h.imax];
        const int first = int(P.bottom_h.size());
        for (int64_t b = 0; b < B.nblocks; b += bchunk) {
            ObsItem it;
            it.level = h.lv_first + h.imax;
            it.unit_level = h.unit_sep ? h.lv_first + h.imax + 1 : -1;
            it.b0 = b;
            it.b1 = std::min<int64_t>(b + bchunk, B.nblocks);
            it.rec = -1;
            it.rec2 = -1;
            P.bottom_h.push_back(it);
        }
        const int cnt = int(P.bottom_h.size()) - first;
        B.rec_first = rec;
        B.rec_count = cnt;
        for (int j = 0; j < cnt; ++j) P.bottom_h[first + j].rec = rec + j;
        rec += cnt;
        if (h.unit_sep) {
            LevelDev& U = P.levels_h[h.lv_first + h.imax + 1];
            U.rec_first = rec;
            U.rec_count = cnt;
            for (int j = 0; j < cnt; ++j) P.bottom_h[first + j].rec2 = rec + j;
            rec += cnt;
        }
    }
    // up items grouped by depth u = 1..max_depth (level imax - u of each system)
    int max_depth = 0;
    for (auto& h : sys) max_depth = std::max(max_depth, h.imax);
    P.max_depth = max_depth;
    P.up_first.push_back(0);
    for (int u = 1; u <= max_depth; ++u) {
        for (int k = 0; k < n; ++k) {
            SysHost& h = sys[k];
            const int l = h.imax - u;
            if (l < 0) continue;
            LevelDev& D = P.levels_h[h.lv_first + l];
            D.rec_first = rec;
            for (int64_t b = 0; b < D.nblocks; b += bchunk) {
                ObsItem it;
                it.level = h.lv_first + l;
                it.unit_level = -1;
                it.b0 = b;
                it.b1 = std::min<int64_t>(b + bchunk, D.nblocks);
                it.rec = rec++;
                it.rec2 = -1;
                P.up_h.push_back(it);
            }
            D.rec_count = rec - D.rec_first;
        }
        P.up_first.push_back(int(P.up_h.size()));
    }
    P.n_bottom = int(P.bottom_h.size());
    P.n_up = int(P.up_h.size());
    P.n_rec = rec;

    // structure factor tables
    P.sk = o->sk_every > 0;
    if (P.sk) {
        auto table_of = [&](int n) {
            for (size_t t = 0; t < P.tw_sides.size(); ++t)
                if (P.tw_sides[t] == n) return P.tw_offs[t];
            P.tw_sides.push_back(n);
            P.tw_offs.push_back(P.tw_total);
            P.tw_total += n;
            P.tw_max = std::max(P.tw_max, n);
            return P.tw_offs.back();
        };
        for (auto& h : sys) {
            SkSys k;
            k.nx = h.d.nx;
            k.ny = h.d.ny;
            k.nz = h.d.nz;
            k.tw_x = table_of(h.d.nx);
            k.tw_y = table_of(h.d.ny);
            k.tw_z = table_of(h.d.nz);
            k.site_offset = h.site_off;
            k.inv_n = 1.0 / double(h.n);
            P.sk_h.push_back(k);
            const int side = h.d.nx;
            P.sk_max_bins = std::max(P.sk_max_bins, int(std::ceil(std::sqrt(3.0) * side / 2.0)) + 2);
        }
        P.sk_fft = true;
        for (auto& h : sys)
            if (!sk_fft_side(h.d.nx)) P.sk_fft = false;
        if (P.sk_fft) {
            for (int k = 0; k < n; ++k) {
                const int side = sys[k].d.nx;
                const int lines = int(sys[k].n / side);
                const int per = std::max(1, kSkFftMaxElems / side);
                for (int l = 0; l < lines; l += per) {
                    const int cnt = std::min(per, lines - l);
                    P.fft_items_h.push_back(make_int4(k, l, cnt, 0));
                    P.fft_max_elems = std::max(P.fft_max_elems, cnt * side);
                }
            }
            P.n_fft_items = int(P.fft_items_h.size());
        }
    }

    // byte layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + std::max<size_t>(bytes, 1));
        return at;
    };
    P.sys = take(sizeof(SysDev) * n);
    P.phys = take(sizeof(SysPhys<double>) * n);
    P.tiles = take(sizeof(int4) * P.n_tiles);
    P.pop0 = take(es * q * P.n_sites);
    P.pop1 = take(es * q * P.n_sites);
    P.step = take(sizeof(int64_t));
    P.status = take(sizeof(int));
    P.d = take(sizeof(double) * P.n_sites);
    P.dbar = take(sizeof(double) * n);
    P.site_items = take(sizeof(int4) * P.n_site_items);
    P.site_partial = take(sizeof(double) * 4 * P.n_site_items);
    P.spans = take(sizeof(SysSpan) * n);
    P.red4 = take(sizeof(double) * 4 * n);
    P.glob = take(sizeof(double) * 8 * n);
    P.levels = take(sizeof(LevelDev) * P.n_levels);
    P.S = take(sizeof(double) * P.n_blocks_pyr);
    P.E = take(sizeof(double) * P.n_blocks_pyr);
    P.bottom_items = take(sizeof(ObsItem) * P.n_bottom);
    P.up_items = take(sizeof(ObsItem) * P.n_up);
    P.rec = take(sizeof(double) * REC * P.n_rec);
    P.acc = take(sizeof(double) * 7 * P.n_levels);
    P.hist_bins = o->hist_bins;
    P.hist_range = o->hist_range;
    P.hist = take(sizeof(uint64_t) * (P.hist_bins > 0 ? (P.hist_bins + 2) * int64_t(P.n_levels) : 0));
    P.field_tmp = take(sizeof(double) * P.max_sites);
    const int64_t skn = P.sk ? P.n_sites : 0;
    P.sk_sys = take(sizeof(SkSys) * (P.sk ? n : 0));
    P.sk_tw = take(sizeof(double) * 2 * P.tw_total);
    P.fft_items = take(sizeof(int4) * P.n_fft_items);
    P.sk_acc = take(sizeof(double) * skn);
    P.sk_b0 = take(sizeof(double) * 2 * skn);
    P.sk_b1 = take(sizeof(double) * 2 * skn);
    P.sk_bins = take(sizeof(double) * 2 * P.sk_max_bins);
    // momentum spectra: j (3 fields), Laplacian scratch (Guo), transforms (3 complex fields), accumulators
    P.jk = P.sk && o->jk_spectra == 1;
    const int64_t jkn = P.jk ? P.n_sites : 0;
    P.jk_j = take(sizeof(double) * 3 * jkn);
    P.jk_lap = take(sizeof(double) * jkn);
    P.jk_F = take(sizeof(double) * 6 * jkn);
    P.jk_acc = take(sizeof(double) * 3 * jkn);
    P.total = off;
    return LB_OK;
}

template <class Real>
SysPhys<Real> to_phys(const SysDev& s, int q) {
    SysPhys<Real> p;
    std::memset(&p, 0, sizeof(p));
    p.rho_c = Real(s.rho_c);
    p.inv_rho_c = Real(s.inv_rho_c);
    p.a = Real(s.a);
    p.b = Real(s.b);
    p.kappa = Real(s.kappa);
    p.kT = Real(s.kT);
    p.nu = Real(s.nu);
    p.lam_bgk = Real(s.lam_bgk);
    p.g_pair = Real(s.g_pair);
    for (int a = 0; a < q; ++a) {
        p.lam[a] = Real(s.lam[a]);
        p.g_diag[a] = Real(s.g_diag[a]);
        p.namp[a] = Real(s.namp[a]);
    }
    return p;
}

SysDev to_dev(const SysHost& h) {
    SysDev s;
    std::memset(&s, 0, sizeof(s));
    const lb_system_desc& d = h.d;
    const int q = q_of(d.lattice), nc = d.lattice == LB_D2Q9 ? 3 : 4;
    const int H = d.coupling == LB_GUO ? 2 : 1;
    s.nx = d.nx;
    s.ny = d.ny;
    s.nz = d.nz;
    s.small = (d.nx < H + 1 || d.ny < H + 1 || (d.lattice == LB_D3Q19 && d.nz < H + 1)) ? 1 : 0;
    s.ns = int32_t(h.n);
    s.n_sites = h.n;
    s.site_offset = h.site_off;
    s.pop_offset = h.pop_off;
    s.rho_c = d.rho_c;
    s.a = d.a;
    s.b = d.b;
    s.kappa = d.kappa;
    s.kT = d.kT;
    s.inv_rho_c = 1.0 / d.rho_c;
    // kinematic viscosity of the Holdych term: tau of the c_x^2 - c_y^2 (D2Q9)
    // or c_y^2 - c_z^2 (D3Q19) shear mode
    s.nu = (d.tau[d.lattice == LB_D2Q9 ? 4 : 6] - 0.5) / 3.0;
    double gamma[LB_MAX_Q];
    for (int a = 0; a < q; ++a) {
        s.lam[a] = a < nc ? 0.0 : 1.0 / d.tau[a];
        gamma[a] = 1.0 - s.lam[a];
        s.g_diag[a] = 1.0 - gamma[a] * gamma[a];
    }
    const int P = d.lattice == LB_D2Q9 ? 3 : 4, R = d.lattice == LB_D2Q9 ? 8 : 16;
    s.g_pair = 1.0 - gamma[P] * gamma[R];
    for (int a = 0; a < q; ++a) {
        const double Na = d.lattice == LB_D2Q9 ? norm2<D2Q9>(a) : norm2<D3Q19>(a);
        s.namp[a] = std::sqrt(Na * s.g_diag[a]);
    }
    s.bgk = 1;
    for (int a = nc; a < q; ++a)
        if (s.lam[a] != s.lam[nc]) s.bgk = 0;
    s.lam_bgk = s.lam[nc];
    s.seed_lo = uint32_t(d.seed & 0xffffffffu);
    s.seed_hi = uint32_t(d.seed >> 32);
    s.system_id = d.system_id;
    return s;
}

}  // namespace

struct lb_ctx {
    int lattice = 0, coupling = 0, fp32 = 0, q = 9, n_sys = 0, tile_id = 0, bgk_only = 0, bulk_ok = 0,
        pair_ok = 0;
    lb_run_opts opts{};
    std::vector<SysHost> sys;
    Plan P;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    int64_t step = 0;
    bool has_state = false;
    lb_status sticky = LB_OK;
    // graph cache: [parity], with the number of kernel nodes of each
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_kernels[2] = {0, 0};
    int64_t launches = 0;       // kernels launched (host-side count)
    int fault_kind = 0;         // armed fault (lb_inject_fault), fires once
    int64_t fault_step = -1;

    template <class T>
    T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
    void* pop(int k) const { return ws + (k ? P.pop1 : P.pop0); }
};

namespace {

#define LB_CHECK(expr)                                   \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return LB_ERR_CUDA;       \
    } while (0)

cudaError_t launch_step_any(lb_ctx* c, const StepLaunch& a) {
    return c->lattice == LB_D2Q9 ? launch_step_d2q9(c->coupling, c->fp32, a, c->stream)
                                 : launch_step_d3q19(c->coupling, c->fp32, a, c->stream);
}

size_t hist_bytes(const Plan& P) {
    return P.hist_bins > 0 ? sizeof(uint64_t) * (P.hist_bins + 2) * size_t(P.n_levels) : 0;
}

// Observable sample of the state held in population buffer `buf`.
// With want_j the site pass also writes the momentum field (for the momentum spectra).
cudaError_t sample_obs(lb_ctx* c, int buf, bool set_mass0, bool count, bool want_j = false) {
    const Plan& P = c->P;
    cudaError_t e;
    const SysDev* sys = c->at<SysDev>(P.sys);
    double* jout = want_j && P.jk ? c->at<double>(P.jk_j) : nullptr;
    e = c->lattice == LB_D2Q9
            ? launch_obs_site_d2q9(c->fp32, sys, c->at<int4>(P.site_items), P.n_site_items, c->pop(buf),
                                   c->at<double>(P.d), c->at<double>(P.site_partial), jout, P.n_sites, c->stream)
            : launch_obs_site_d3q19(c->fp32, sys, c->at<int4>(P.site_items), P.n_site_items, c->pop(buf),
                                    c->at<double>(P.d), c->at<double>(P.site_partial), jout, P.n_sites, c->stream);
    if (e != cudaSuccess) return e;
    e = launch_reduce_sys(c->at<SysSpan>(P.spans), c->n_sys, c->at<double>(P.site_partial), 4, c->at<double>(P.red4),
                          c->stream);
    if (e != cudaSuccess) return e;
    e = launch_obs_globals(sys, c->n_sys, c->at<double>(P.red4), c->at<double>(P.dbar), c->at<double>(P.glob),
                           set_mass0 ? 1 : 0, count ? 1 : 0, c->stream);
    c->launches += 3;
    if (e != cudaSuccess || !count) return e;
    c->launches += 2 + P.max_depth;
    HistDev H;
    H.counts = c->at<unsigned long long>(P.hist);
    H.nbins = P.hist_bins;
    H.lo = -P.hist_range;
    H.inv_w = P.hist_bins > 0 ? double(P.hist_bins) / (P.hist_range - (-P.hist_range)) : 0.0;
    e = launch_pyr_bottom(sys, c->at<LevelDev>(P.levels), c->at<ObsItem>(P.bottom_items), P.n_bottom,
                          c->at<double>(P.d), c->at<double>(P.dbar), c->at<double>(P.S), c->at<double>(P.E),
                          c->at<double>(P.rec), H, c->stream);
    if (e != cudaSuccess) return e;
    for (int u = 1; u <= P.max_depth; ++u) {
        const int first = P.up_first[u - 1], cnt = P.up_first[u] - first;
        e = launch_pyr_up(sys, c->at<LevelDev>(P.levels), c->at<ObsItem>(P.up_items) + first, cnt,
                          c->lattice == LB_D3Q19 ? 1 : 0, c->at<double>(P.S), c->at<double>(P.E),
                          c->at<double>(P.rec), H, c->stream);
        if (e != cudaSuccess) return e;
    }
    return launch_obs_accum(c->at<LevelDev>(P.levels), P.n_levels, c->at<double>(P.rec), c->at<double>(P.acc),
                            c->at<int>(P.status), c->stream);
}

// Momentum spectra of the momentum field the site pass just wrote: Guo
// half-force, then per component x, y (and z) transforms, then accumulation.
cudaError_t sample_jk(lb_ctx* c) {
    const Plan& P = c->P;
    cudaError_t e;
    const SysDev* sys = c->at<SysDev>(P.sys);
    const SkSys* sk = c->at<SkSys>(P.sk_sys);
    const int4* items = c->at<int4>(P.site_items);
    const int n_items = P.n_site_items;
    const int64_t ns = P.n_sites;
    double* j = c->at<double>(P.jk_j);
    double* F = c->at<double>(P.jk_F);
    double* b0 = c->at<double>(P.sk_b0);
    double* b1 = c->at<double>(P.sk_b1);
    const double* tw = c->at<double>(P.sk_tw);
    const bool d3 = c->lattice == LB_D3Q19;
    const int dims = d3 ? 3 : 2;
    if (c->coupling == LB_GUO) {
        e = launch_jk_guo_force(d3 ? 1 : 0, sys, items, n_items, c->at<double>(P.d), c->at<double>(P.jk_lap), j, ns,
                                c->stream);
        if (e != cudaSuccess) return e;
        c->launches += 2;
    }
    for (int a = 0; a < dims; ++a) {
        double* Fa = F + 2 * ns * a;
        if (P.sk_fft) {
            const int4* fi = c->at<int4>(P.fft_items);
            e = launch_sk_fft(sys, sk, fi, P.n_fft_items, 0, j + ns * a, nullptr, nullptr, tw, b0, P.fft_max_elems,
                              c->stream);
            if (e != cudaSuccess) return e;
            e = launch_sk_fft(sys, sk, fi, P.n_fft_items, 1, nullptr, nullptr, b0, tw, d3 ? b1 : Fa,
                              P.fft_max_elems, c->stream);
            if (e != cudaSuccess) return e;
            c->launches += 2;
            if (d3) {
                e = launch_sk_fft(sys, sk, fi, P.n_fft_items, 2, nullptr, nullptr, b1, tw, Fa, P.fft_max_elems,
                                  c->stream);
                if (e != cudaSuccess) return e;
                c->launches += 1;
            }
            continue;
        }
        e = launch_sk_x(sys, sk, items, n_items, j + ns * a, nullptr, tw, b0, c->stream);
        if (e != cudaSuccess) return e;
        e = launch_sk_pass(sk, items, n_items, 1, tw, b0, d3 ? b1 : Fa, c->stream);
        if (e != cudaSuccess) return e;
        c->launches += 2;
        if (d3) {
            e = launch_sk_pass(sk, items, n_items, 2, tw, b1, Fa, c->stream);
            if (e != cudaSuccess) return e;
            c->launches += 1;
        }
    }
    c->launches += 1;
    return launch_jk_accum(sk, items, n_items, dims, F, F + 2 * ns, d3 ? F + 4 * ns : nullptr,
                           c->at<double>(P.jk_acc), ns, c->stream);
}

// Structure-factor sample of the state in buffer `buf`; `have_d` when the
// observable pass of the same step has already filled d and dbar (and, with
// momentum spectra on, the momentum field).
cudaError_t sample_sk(lb_ctx* c, int buf, bool have_d) {
    const Plan& P = c->P;
    cudaError_t e;
    if (!have_d) {
        e = sample_obs(c, buf, false, false, true);
        if (e != cudaSuccess) return e;
    }
    const SysDev* sys = c->at<SysDev>(P.sys);
    const SkSys* sk = c->at<SkSys>(P.sk_sys);
    const int4* items = c->at<int4>(P.site_items);
    double* b0 = c->at<double>(P.sk_b0);
    double* b1 = c->at<double>(P.sk_b1);
    const double* tw = c->at<double>(P.sk_tw);
    const double* fin = b1;
    if (P.sk_fft) {
        const int4* fi = c->at<int4>(P.fft_items);
        e = launch_sk_fft(sys, sk, fi, P.n_fft_items, 0, c->at<double>(P.d), c->at<double>(P.dbar), nullptr, tw, b0,
                          P.fft_max_elems, c->stream);
        if (e != cudaSuccess) return e;
        e = launch_sk_fft(sys, sk, fi, P.n_fft_items, 1, nullptr, nullptr, b0, tw, b1, P.fft_max_elems, c->stream);
        if (e != cudaSuccess) return e;
        c->launches += 2;
        if (c->lattice == LB_D3Q19) {
            e = launch_sk_fft(sys, sk, fi, P.n_fft_items, 2, nullptr, nullptr, b1, tw, b0, P.fft_max_elems,
                              c->stream);
            if (e != cudaSuccess) return e;
            fin = b0;
            c->launches += 1;
        }
    } else {
        e = launch_sk_x(sys, sk, items, P.n_site_items, c->at<double>(P.d), c->at<double>(P.dbar), tw, b0,
                        c->stream);
        if (e != cudaSuccess) return e;
        e = launch_sk_pass(sk, items, P.n_site_items, 1, tw, b0, b1, c->stream);
        if (e != cudaSuccess) return e;
        c->launches += 2;
        if (c->lattice == LB_D3Q19) {
            e = launch_sk_pass(sk, items, P.n_site_items, 2, tw, b1, b0, c->stream);
            if (e != cudaSuccess) return e;
            fin = b0;
            c->launches += 1;
        }
    }
    c->launches += 1;
    e = launch_sk_accum(sk, items, P.n_site_items, fin, c->at<double>(P.sk_acc), c->stream);
    if (e != cudaSuccess || !P.jk) return e;
    return sample_jk(c);
}

// Launch `n` steps starting at host step c->step (device counter must equal it).
cudaError_t launch_steps(lb_ctx* c, int64_t n) {
    const Plan& P = c->P;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t t = c->step + k;
        StepLaunch a;
        a.sys = c->at<SysDev>(P.sys);
        a.phys = c->ws + P.phys;
        a.tiles = c->at<int4>(P.tiles);
        a.n_tiles = P.n_tiles;
        a.fin = c->pop(int(t & 1));
        a.fout = c->pop(int((t + 1) & 1));
        a.step_ptr = c->at<int64_t>(P.step);
        a.k = int(k);
        a.status = c->at<int>(P.status);
        a.tile_id = c->tile_id;
        a.bgk_only = c->bgk_only;
        a.bulk_ok = c->bulk_ok;
        a.pair_ok = c->pair_ok;
        cudaError_t e = launch_step_any(c, a);
        if (e != cudaSuccess) return e;
        c->launches += 1;
        const int64_t t1 = t + 1;
        const bool obs_due = c->opts.obs_every > 0 && t1 % c->opts.obs_every == 0;
        if (c->fault_kind != 0 && t1 == c->fault_step) {
            static const int bits[5] = {0, ST_RHO, ST_NOISE, ST_NONFINITE, ST_TIMEOUT};
            e = launch_set_status(c->at<int>(P.status), bits[c->fault_kind], c->stream);
            c->fault_kind = 0;
            if (e != cudaSuccess) return e;
        }
        const bool sk_due = c->opts.sk_every > 0 && t1 % c->opts.sk_every == 0;
        if (obs_due) {
            e = sample_obs(c, int(t1 & 1), false, true, sk_due);
            if (e != cudaSuccess) return e;
        }
        if (sk_due) {
            e = sample_sk(c, int(t1 & 1), obs_due);
            if (e != cudaSuccess) return e;
        }
    }
    c->launches += 1;
    return launch_advance(c->at<int64_t>(P.step), n, c->stream);
}

lb_status read_status(lb_ctx* c) {
    int st = 0;
    if (cudaMemcpyAsync(&st, c->at<int>(c->P.status), sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return LB_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LB_ERR_CUDA;
    if (st & ST_RHO) return LB_ERR_NONPOSITIVE_DENSITY;
    if (st & ST_NOISE) return LB_ERR_NOISE_NOT_PD;
    if (st & ST_NONFINITE) return LB_ERR_NONFINITE;
    if (st & ST_TIMEOUT) return LB_ERR_TIMEOUT;
    return LB_OK;
}

lb_status sync_and_check(lb_ctx* c) {
    lb_status s = read_status(c);
    if (s != LB_OK && c->sticky == LB_OK) c->sticky = s;
    return c->sticky != LB_OK ? c->sticky : s;
}

void drop_graphs(lb_ctx* c) {
    for (auto& g : c->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

lb_status reset_accumulators(lb_ctx* c) {
    const Plan& P = c->P;
    LB_CHECK(cudaMemsetAsync(c->ws + P.acc, 0, sizeof(double) * 7 * P.n_levels, c->stream));
    if (P.hist_bins > 0) LB_CHECK(cudaMemsetAsync(c->ws + P.hist, 0, hist_bytes(P), c->stream));
    LB_CHECK(cudaMemsetAsync(c->ws + P.glob, 0, sizeof(double) * 8 * c->n_sys, c->stream));
    LB_CHECK(cudaMemsetAsync(c->ws + P.status, 0, sizeof(int), c->stream));
    if (P.sk) LB_CHECK(cudaMemsetAsync(c->ws + P.sk_acc, 0, sizeof(double) * P.n_sites, c->stream));
    if (P.jk) LB_CHECK(cudaMemsetAsync(c->ws + P.jk_acc, 0, sizeof(double) * 3 * P.n_sites, c->stream));
    return LB_OK;
}

}  // namespace

extern "C" {

const char* lb_version(void) { return "lbfluct 0.1 (sm_103a)"; }

const char* lb_status_string(lb_status s) {
    switch (s) {
        case LB_OK: return "ok";
        case LB_ERR_ARG: return "invalid argument";
        case LB_ERR_CUDA: return "CUDA error";
        case LB_ERR_WORKSPACE: return "workspace too small or misaligned";
        case LB_ERR_NONPOSITIVE_DENSITY: return "non-positive density";
        case LB_ERR_NOISE_NOT_PD: return "noise covariance not positive definite";
        case LB_ERR_NONFINITE: return "non-finite observable";
        case LB_ERR_UNSUPPORTED: return "unsupported combination";
        case LB_ERR_STATE: return "invalid state (sticky error or missing initialisation)";
        case LB_ERR_IO: return "checkpoint I/O error";
        case LB_ERR_NO_ROOT: return "no solution of the self-consistency equation";
        case LB_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    }
    return "unknown status";
}

lb_status lb_workspace_bytes(const lb_system_desc* systems, int n_systems, const lb_run_opts* opts, size_t* bytes) {
    if (!bytes) return LB_ERR_ARG;
    std::vector<SysHost> sys;
    Plan P;
    int tile_id;
    lb_status st = make_plan(systems, n_systems, opts, sys, P, tile_id);
    if (st != LB_OK) return st;
    *bytes = P.total;
    return LB_OK;
}

lb_status lb_create(const lb_system_desc* systems, int n_systems, const lb_run_opts* opts, void* d_workspace,
                    size_t bytes, void* stream, lb_ctx** out) {
    if (!out) return LB_ERR_ARG;
    *out = nullptr;
    lb_ctx* c = new lb_ctx();
    lb_status st = make_plan(systems, n_systems, opts, c->sys, c->P, c->tile_id);
    if (st != LB_OK) {
        delete c;
        return st;
    }
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) || bytes < c->P.total) {
        delete c;
        return LB_ERR_WORKSPACE;
    }
    c->lattice = systems[0].lattice;
    c->coupling = systems[0].coupling;
    c->fp32 = opts->precision == LB_FP32_DEVIATION ? 1 : 0;
    c->q = q_of(c->lattice);
    c->n_sys = n_systems;
    c->opts = *opts;
    c->stream = static_cast<cudaStream_t>(stream);
    c->ws = static_cast<char*>(d_workspace);
    c->ws_bytes = bytes;
    const Plan& P = c->P;
    std::vector<SysDev> sd;
    for (auto& h : c->sys) sd.push_back(to_dev(h));
    // collision specialisation: 2 = one rate, equal to 1 everywhere; 1 = one rate per system; 0 = per mode
    c->bgk_only = 2;
    for (auto& s : sd) {
        if (!s.bgk) c->bgk_only = 0;
        else if (s.lam_bgk != 1.0 && c->bgk_only == 2) c->bgk_only = 1;
    }
    // bulk-copy staging: 16-byte aligned rows (nx % 4 == 0, so every system's
    // populations start 16-byte aligned too), at most 4 seam pieces per staged
    // row (nx >= 8) and single periodic wraps (every side >= 3)
    c->bulk_ok = 1;
    for (auto& s : sd)
        if (s.nx % 4 != 0 || s.nx < 8 || s.small) c->bulk_ok = 0;
    // paired-site kernel: its producers pull aligned quads of x-adjacent sites
    // and its consumers store aligned pairs, which needs every nx to be a
    // multiple of 4 (every population array then starts 16-byte aligned)
    c->pair_ok = 1;
    for (auto& s : sd)
        if (s.nx % 4 != 0) c->pair_ok = 0;
    bool ok = cudaMemcpyAsync(c->ws + P.sys, sd.data(), sizeof(SysDev) * sd.size(), cudaMemcpyHostToDevice,
                              c->stream) == cudaSuccess;
    // physics in the step kernel's precision (staged on the host, copied synchronously)
    if (c->fp32) {
        std::vector<SysPhys<float>> ph;
        for (auto& s : sd) ph.push_back(to_phys<float>(s, c->q));
        ok = ok && cudaMemcpy(c->ws + P.phys, ph.data(), sizeof(SysPhys<float>) * ph.size(),
                              cudaMemcpyHostToDevice) == cudaSuccess;
    } else {
        std::vector<SysPhys<double>> ph;
        for (auto& s : sd) ph.push_back(to_phys<double>(s, c->q));
        ok = ok && cudaMemcpy(c->ws + P.phys, ph.data(), sizeof(SysPhys<double>) * ph.size(),
                              cudaMemcpyHostToDevice) == cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(c->ws + P.tiles, P.tiles_h.data(), sizeof(int4) * P.n_tiles, cudaMemcpyHostToDevice,
                               c->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(c->ws + P.site_items, P.site_items_h.data(), sizeof(int4) * P.n_site_items,
                               cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(c->ws + P.spans, P.spans_h.data(), sizeof(SysSpan) * P.spans_h.size(),
                               cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(c->ws + P.levels, P.levels_h.data(), sizeof(LevelDev) * P.n_levels,
                               cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    if (P.n_bottom)
        ok = ok && cudaMemcpyAsync(c->ws + P.bottom_items, P.bottom_h.data(), sizeof(ObsItem) * P.n_bottom,
                                   cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    if (P.n_up)
        ok = ok && cudaMemcpyAsync(c->ws + P.up_items, P.up_h.data(), sizeof(ObsItem) * P.n_up,
                                   cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    if (P.sk) {
        ok = ok && cudaMemcpyAsync(c->ws + P.sk_sys, P.sk_h.data(), sizeof(SkSys) * P.sk_h.size(),
                                   cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
        // twiddle tables: sides and offsets staged through the bin scratch (ints fit in it)
        std::vector<int> meta(P.tw_sides);
        meta.insert(meta.end(), P.tw_offs.begin(), P.tw_offs.end());
        int* dmeta = reinterpret_cast<int*>(c->ws + P.field_tmp);
        ok = ok && cudaMemcpyAsync(dmeta, meta.data(), sizeof(int) * meta.size(), cudaMemcpyHostToDevice,
                                   c->stream) == cudaSuccess;
        ok = ok && launch_sk_twiddles(c->at<double>(P.sk_tw), dmeta, dmeta + P.tw_sides.size(),
                                      int(P.tw_sides.size()), P.tw_max, c->stream) == cudaSuccess;
        if (P.n_fft_items)
            ok = ok && cudaMemcpyAsync(c->ws + P.fft_items, P.fft_items_h.data(), sizeof(int4) * P.n_fft_items,
                                       cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    }
    ok = ok && cudaMemsetAsync(c->ws + P.step, 0, sizeof(int64_t), c->stream) == cudaSuccess;
    ok = ok && reset_accumulators(c) == LB_OK;
    ok = ok && cudaStreamSynchronize(c->stream) == cudaSuccess;
    if (!ok) {
        delete c;
        return LB_ERR_CUDA;
    }
    *out = c;
    return LB_OK;
}

lb_status lb_stripe_density(const lb_system_desc* s, int n, double* out) {
    if (!s || n < 1 || !out) return LB_ERR_ARG;
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
        const lb_system_desc& d = s[k];
        if (d.nx < 1 || d.ny < 1 || d.nz < 1) return LB_ERR_ARG;
        if (!(d.a < 0) || !(d.b > 0) || !(d.kappa >= 0) || !std::isfinite(d.a) || !std::isfinite(d.b))
            return LB_ERR_ARG;
        const double phi0 = std::sqrt(-d.a / d.b), w = std::sqrt(-2.0 * d.kappa / d.a);
        const double x1 = 0.25 * d.nx, x2 = 0.75 * d.nx;
        for (int x = 0; x < d.nx; ++x) {
            const double t = w > 0 ? std::tanh((x - x1) / w) - std::tanh((x - x2) / w) - 1.0
                                   : (x >= x1 && x < x2 ? 1.0 : -1.0);
            const double rho = d.rho_c + phi0 * t;
            for (int z = 0; z < d.nz; ++z)
                for (int y = 0; y < d.ny; ++y) out[off + (size_t(z) * d.ny + y) * d.nx + x] = rho;
        }
        off += size_t(d.nx) * d.ny * d.nz;
    }
    return LB_OK;
}

lb_status lb_init(lb_ctx* c, int mode, double amplitude, const double* h_rho) {
    if (!c) return LB_ERR_ARG;
    if (mode != LB_INIT_UNIFORM_NOISE && mode != LB_INIT_FROM_RHO && mode != LB_INIT_TANH_STRIPE &&
        mode != LB_INIT_FROM_DEVICE_RHO)
        return LB_ERR_ARG;
    if ((mode == LB_INIT_FROM_RHO || mode == LB_INIT_FROM_DEVICE_RHO) && !h_rho) return LB_ERR_ARG;
    std::vector<double> stripe;
    if (mode == LB_INIT_TANH_STRIPE) {
        std::vector<lb_system_desc> desc;
        for (auto& h : c->sys) desc.push_back(h.d);
        stripe.resize(size_t(c->P.n_sites));
        const lb_status st = lb_stripe_density(desc.data(), int(desc.size()), stripe.data());
        if (st != LB_OK) return st;
        h_rho = stripe.data();          // then exactly the LB_INIT_FROM_RHO path
        mode = LB_INIT_FROM_RHO;
    }
    if (mode == LB_INIT_UNIFORM_NOISE && !(amplitude >= 0 && std::isfinite(amplitude))) return LB_ERR_ARG;
    const Plan& P = c->P;
    const SysDev* sys = c->at<SysDev>(P.sys);
    // the cached step graphs stay valid: they read the step counter on the
    // device and address only the context's fixed workspace regions, and a
    // chunk's schedule of observable passes depends on the step only modulo
    // the chunk length
    c->step = 0;
    LB_CHECK(cudaMemsetAsync(c->ws + P.step, 0, sizeof(int64_t), c->stream));
    if (reset_accumulators(c) != LB_OK) return LB_ERR_CUDA;
    if (mode == LB_INIT_UNIFORM_NOISE) {
        LB_CHECK(launch_init_noise(sys, c->at<int4>(P.site_items), P.n_site_items, amplitude, c->at<double>(P.d),
                                   c->at<double>(P.site_partial), c->stream));
        LB_CHECK(launch_reduce_sys(c->at<SysSpan>(P.spans), c->n_sys, c->at<double>(P.site_partial), 4,
                                   c->at<double>(P.red4), c->stream));
        // dbar = sum d / n via the globals kernel (its mass fields are overwritten below)
        LB_CHECK(launch_obs_globals(sys, c->n_sys, c->at<double>(P.red4), c->at<double>(P.dbar),
                                    c->at<double>(P.glob), 1, 0, c->stream));
    } else {
        LB_CHECK(cudaMemcpyAsync(c->at<double>(P.d), h_rho, sizeof(double) * P.n_sites,
                                 mode == LB_INIT_FROM_DEVICE_RHO ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 c->stream));
        LB_CHECK(launch_set_dbar(sys, c->n_sys, c->at<double>(P.dbar), c->stream));
    }
    LB_CHECK(c->lattice == LB_D2Q9
                 ? launch_init_feq_d2q9(c->coupling, c->fp32, sys, c->at<int4>(P.site_items), P.n_site_items,
                                        c->at<double>(P.d), c->at<double>(P.dbar), c->pop(0), c->stream)
                 : launch_init_feq_d3q19(c->coupling, c->fp32, sys, c->at<int4>(P.site_items), P.n_site_items,
                                         c->at<double>(P.d), c->at<double>(P.dbar), c->pop(0), c->stream));
    LB_CHECK(sample_obs(c, 0, true, false));
    LB_CHECK(cudaStreamSynchronize(c->stream));
    c->sticky = LB_OK;
    c->has_state = true;
    return LB_OK;
}

lb_status lb_step(lb_ctx* c, int64_t nsteps) {
    if (!c) return LB_ERR_ARG;
    if (nsteps < 0) return LB_ERR_ARG;
    if (!c->has_state || c->sticky != LB_OK) return LB_ERR_STATE;
    if (nsteps == 0) return LB_OK;
    const int C = c->opts.graph_chunk;
    int64_t left = nsteps;
    struct Range {   // NVTX range over the enqueue of these steps (profiler timelines)
        Range() { nvtxRangePushA("lb_step"); }
        ~Range() { nvtxRangePop(); }
    } range;
    while (left > 0) {
        const bool aligned = C > 0 && c->fault_kind == 0 && c->step % C == 0 && left >= C &&
                             (c->opts.obs_every == 0 || C % c->opts.obs_every == 0) &&
                             (c->opts.sk_every == 0 || C % c->opts.sk_every == 0);
        if (!aligned) {
            // plain launches up to the next chunk boundary (or all remaining)
            int64_t n = left;
            if (C > 0) {
                const int64_t to_boundary = (C - c->step % C) % C;
                n = to_boundary > 0 ? std::min(left, to_boundary) : left;
                if (n >= C) n = left;   // never reached: aligned handles it
            }
            if (c->fault_kind == LB_FAULT_LAUNCH && c->fault_step <= c->step + n) {
                // the step that would end at fault_step is not launched
                n = c->fault_step - 1 - c->step;
                if (n == 0) {
                    c->fault_kind = 0;
                    return LB_ERR_CUDA;
                }
            }
            if (launch_steps(c, n) != cudaSuccess) return LB_ERR_CUDA;
            c->step += n;
            left -= n;
            continue;
        }
        const int parity = int(c->step & 1);
        if (!c->graph[parity]) {
            cudaStream_t cap;
            if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return LB_ERR_CUDA;
            cudaStream_t saved = c->stream;
            c->stream = cap;
            cudaGraph_t g = nullptr;
            const int64_t before = c->launches;
            bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            ok = ok && launch_steps(c, C) == cudaSuccess;
            c->graph_kernels[parity] = c->launches - before;
            c->launches = before;
            ok = (cudaStreamEndCapture(cap, &g) == cudaSuccess) && ok;
            c->stream = saved;
            ok = ok && cudaGraphInstantiate(&c->graph[parity], g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cap);
            if (!ok) return LB_ERR_CUDA;
        }
        if (cudaGraphLaunch(c->graph[parity], c->stream) != cudaSuccess) return LB_ERR_CUDA;
        c->launches += c->graph_kernels[parity];
        c->step += C;
        left -= C;
    }
    return LB_OK;
}

lb_status lb_sync(lb_ctx* c) {
    if (!c) return LB_ERR_ARG;
    return sync_and_check(c);
}

lb_status lb_get_step(lb_ctx* c, int64_t* step) {
    if (!c || !step) return LB_ERR_ARG;
    *step = c->step;
    return LB_OK;
}

lb_status lb_observables(lb_ctx* c, int sys, lb_obs_level* h_levels, int max_levels, int* n_levels,
                         lb_obs_global* h_global) {
    if (!c || sys < 0 || sys >= c->n_sys || (!h_levels && max_levels > 0)) return LB_ERR_ARG;
    const SysHost& h = c->sys[sys];
    const int nl = int(h.lv.size());
    std::vector<double> acc(7 * nl), glob(8);
    LB_CHECK(cudaMemcpyAsync(acc.data(), c->at<double>(c->P.acc) + 7 * h.lv_first, sizeof(double) * 7 * nl,
                             cudaMemcpyDeviceToHost, c->stream));
    LB_CHECK(cudaMemcpyAsync(glob.data(), c->at<double>(c->P.glob) + 8 * sys, sizeof(double) * 8,
                             cudaMemcpyDeviceToHost, c->stream));
    lb_status s = sync_and_check(c);
    if (n_levels) *n_levels = nl;
    for (int l = 0; l < nl && l < max_levels; ++l) {
        lb_obs_level& o = h_levels[l];
        o.bx = h.lv[l].bx;
        o.by = h.lv[l].by;
        o.bz = h.lv[l].bz;
        o.pad = 0;
        o.n = acc[7 * l + 0];
        o.sum_m = acc[7 * l + 1];
        o.sum_m2 = acc[7 * l + 2];
        o.sum_abs_m = acc[7 * l + 3];
        o.sum_m4 = acc[7 * l + 4];
        o.sum_e = acc[7 * l + 5];
        o.sum_e2 = acc[7 * l + 6];
    }
    if (h_global) {
        h_global->step = c->step;
        h_global->n_samples = int64_t(glob[0]);
        h_global->mass0 = glob[1];
        h_global->mass = glob[2];
        h_global->momentum[0] = glob[3];
        h_global->momentum[1] = glob[4];
        h_global->momentum[2] = glob[5];
        h_global->rho_mean = glob[6];
    }
    return s;
}

lb_status lb_observables_all(lb_ctx* c, lb_obs_level* h_levels, int max_levels, int* level_first,
                             lb_obs_global* h_globals) {
    if (!c || !level_first) return LB_ERR_ARG;
    const Plan& P = c->P;
    int total = 0;
    for (int k = 0; k < c->n_sys; ++k) {
        level_first[k] = total;
        total += int(c->sys[k].lv.size());
    }
    level_first[c->n_sys] = total;
    if (h_levels && max_levels < total) return LB_ERR_ARG;
    std::vector<double> acc(7 * size_t(P.n_levels)), glob(8 * size_t(c->n_sys));
    LB_CHECK(cudaMemcpyAsync(acc.data(), c->ws + P.acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost,
                             c->stream));
    LB_CHECK(cudaMemcpyAsync(glob.data(), c->ws + P.glob, sizeof(double) * glob.size(), cudaMemcpyDeviceToHost,
                             c->stream));
    lb_status s = sync_and_check(c);
    for (int k = 0; k < c->n_sys && h_levels; ++k) {
        const SysHost& h = c->sys[k];
        for (size_t l = 0; l < h.lv.size(); ++l) {
            const double* a = acc.data() + 7 * (size_t(h.lv_first) + l);
            lb_obs_level& o = h_levels[level_first[k] + int(l)];
            o.bx = h.lv[l].bx;
            o.by = h.lv[l].by;
            o.bz = h.lv[l].bz;
            o.pad = 0;
            o.n = a[0];
            o.sum_m = a[1];
            o.sum_m2 = a[2];
            o.sum_abs_m = a[3];
            o.sum_m4 = a[4];
            o.sum_e = a[5];
            o.sum_e2 = a[6];
        }
    }
    for (int k = 0; k < c->n_sys && h_globals; ++k) {
        const double* g = glob.data() + 8 * size_t(k);
        lb_obs_global& o = h_globals[k];
        o.step = c->step;
        o.n_samples = int64_t(g[0]);
        o.mass0 = g[1];
        o.mass = g[2];
        o.momentum[0] = g[3];
        o.momentum[1] = g[4];
        o.momentum[2] = g[5];
        o.rho_mean = g[6];
    }
    return s;
}

lb_status lb_derive(const lb_obs_level* L, double kT, double out[6]) {
    if (!L || !out || !(L->n > 0) || !(kT > 0)) return LB_ERR_ARG;
    const double n = L->n, v = double(L->bx) * L->by * L->bz;
    const double m = L->sum_m / n, m2 = L->sum_m2 / n, am = L->sum_abs_m / n, m4 = L->sum_m4 / n;
    const double e = L->sum_e / n, e2 = L->sum_e2 / n;
    out[0] = am;
    out[1] = v / kT * (m2 - m * m);
    out[2] = v / kT * (m2 - am * am);
    out[3] = v / kT * (e2 - e * e);
    out[4] = m2 > 0 ? 1.0 - m4 / (3.0 * m2 * m2) : NAN;
    out[5] = m;
    return LB_OK;
}

lb_status lb_histogram(lb_ctx* c, int sys, int level, uint64_t* h_counts, int n_counts, double* lo, double* hi) {
    if (!c || sys < 0 || sys >= c->n_sys) return LB_ERR_ARG;
    const Plan& P = c->P;
    if (P.hist_bins == 0) return LB_ERR_UNSUPPORTED;
    const SysHost& h = c->sys[sys];
    if (level < 0 || level >= int(h.lv.size()) || !h_counts || n_counts != P.hist_bins + 2) return LB_ERR_ARG;
    const int nh = P.hist_bins + 2;
    LB_CHECK(cudaMemcpyAsync(h_counts, c->at<uint64_t>(P.hist) + int64_t(h.lv_first + level) * nh,
                             sizeof(uint64_t) * nh, cudaMemcpyDeviceToHost, c->stream));
    if (lo) *lo = -P.hist_range;
    if (hi) *hi = P.hist_range;
    return sync_and_check(c);
}

lb_status lb_histogram_estimates(const uint64_t* counts, int nbins, double lo, double hi, double vol, double kT,
                                 double m_cut, double frac, double out[LB_HIST_EST]) {
    if (!counts || !out || nbins < 2 || !(hi > 0) || lo != -hi || !std::isfinite(hi) || !(vol > 0) || !(kT > 0) ||
        !(frac > 0 && frac < 1) || !(m_cut >= 0))
        return LB_ERR_ARG;
    for (int k = 0; k < LB_HIST_EST; ++k) out[k] = NAN;
    const double w = (hi - lo) / nbins;
    std::vector<double> mc(nbins), cnt(nbins), ps(nbins);
    double n_all = double(counts[0]) + double(counts[nbins + 1]);
    for (int k = 0; k < nbins; ++k) {
        mc[k] = lo + (k + 0.5) * w;
        cnt[k] = std::fabs(mc[k]) < m_cut ? 0.0 : double(counts[1 + k]);
        n_all += cnt[k];
    }
    for (int k = 0; k < nbins; ++k) ps[k] = 0.5 * (cnt[k] + cnt[nbins - 1 - k]);
    out[6] = 0;
    out[10] = n_all;
    const int k_in = nbins / 2;       // innermost bin with centre >= 0
    int ks = k_in;
    for (int k = k_in + 1; k < nbins; ++k)
        if (ps[k] > ps[ks]) ks = k;
    double kept = 0, s_abs = 0, s_m2 = 0;
    for (int k = 0; k < nbins; ++k) {
        kept += cnt[k];
        s_abs += std::fabs(mc[k]) * cnt[k];
        s_m2 += mc[k] * mc[k] * cnt[k];
    }
    if (kept > 0) {
        out[8] = s_abs / kept;
        out[9] = s_m2 / kept;
    }
    if (!(n_all > 0) || !(ps[ks] > 0)) return LB_OK;
    const bool central = ks == k_in;
    out[0] = mc[ks];
    out[1] = ps[ks] / (n_all * w);
    constexpr double kPi = 3.14159265358979323846;
    out[2] = vol / ((central ? 2.0 : 8.0) * kPi * kT * out[1] * out[1]);
    out[7] = central ? 1.0 : 0.0;
    // fit window: contiguous bins around k* at or above frac of the peak
    const double floor_v = frac * ps[ks];
    const int kmin = central ? 0 : k_in;
    int a = ks, b = ks;
    while (a - 1 >= kmin && ps[a - 1] >= floor_v) --a;
    while (b + 1 < nbins && ps[b + 1] >= floor_v) ++b;
    const int nfit = b - a + 1;
    out[6] = nfit;
    if (nfit >= 3) {
        // weighted normal equations for y = c0 + c1 x + c2 x^2, x centred on the peak
        // for conditioning (the fitted curve is the same)
        const double x0 = mc[ks];
        double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, r[3] = {0, 0, 0};
        for (int k = a; k <= b; ++k) {
            const double x = mc[k] - x0, y = std::log(ps[k]), wt = ps[k];
            const double v[3] = {1.0, x, x * x};
            for (int i = 0; i < 3; ++i) {
                r[i] += wt * v[i] * y;
                for (int j = 0; j < 3; ++j) A[i][j] += wt * v[i] * v[j];
            }
        }
        // Gaussian elimination with partial pivoting on the 3 x 3 system
        double M[3][4];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) M[i][j] = A[i][j];
            M[i][3] = r[i];
        }
        bool ok = true;
        for (int col = 0; col < 3 && ok; ++col) {
            int best = col;
            for (int i = col + 1; i < 3; ++i)
                if (std::fabs(M[i][col]) > std::fabs(M[best][col])) best = i;
            if (!(std::fabs(M[best][col]) > 0)) ok = false;
            if (!ok) break;
            if (best != col)
                for (int j = 0; j < 4; ++j) std::swap(M[col][j], M[best][j]);
            for (int i = col + 1; i < 3; ++i) {
                const double f = M[i][col] / M[col][col];
                for (int j = col; j < 4; ++j) M[i][j] -= f * M[col][j];
            }
        }
        if (ok) {
            double cf[3];
            for (int i = 2; i >= 0; --i) {
                double t = M[i][3];
                for (int j = i + 1; j < 3; ++j) t -= M[i][j] * cf[j];
                cf[i] = t / M[i][i];
            }
            if (cf[2] < 0) {
                out[4] = -0.5 / cf[2];
                out[3] = x0 - cf[1] / (2.0 * cf[2]);
                out[5] = vol * out[4] / kT;
            }
        }
    }
    return LB_OK;
}

lb_status lb_structure_factor(lb_ctx* c, int sys, double* h_sum, int64_t* h_count, int nbins, int64_t* n_samples) {
    if (!c || sys < 0 || sys >= c->n_sys || nbins < 0 || (nbins > 0 && (!h_sum || !h_count))) return LB_ERR_ARG;
    const Plan& P = c->P;
    if (!P.sk) return LB_ERR_UNSUPPORTED;
    if (nbins > P.sk_max_bins) return LB_ERR_ARG;
    double* bins = c->at<double>(P.sk_bins);
    LB_CHECK(launch_sk_bin(c->at<SkSys>(P.sk_sys), sys, c->at<double>(P.sk_acc), nbins, bins, bins + P.sk_max_bins,
                           c->stream));
    std::vector<double> hb(2 * size_t(P.sk_max_bins));
    if (nbins > 0)
        LB_CHECK(cudaMemcpyAsync(hb.data(), bins, sizeof(double) * 2 * P.sk_max_bins, cudaMemcpyDeviceToHost,
                                 c->stream));
    lb_status s = sync_and_check(c);
    for (int j = 0; j < nbins; ++j) {
        h_sum[j] = hb[j];
        h_count[j] = int64_t(hb[P.sk_max_bins + j]);
    }
    if (n_samples) *n_samples = c->step / c->opts.sk_every;
    return s;
}

lb_status lb_momentum_spectra(lb_ctx* c, int sys, double* h_sum, int64_t* h_count, int nbins, int64_t* n_samples) {
    if (!c || sys < 0 || sys >= c->n_sys || nbins < 0 || (nbins > 0 && (!h_sum || !h_count))) return LB_ERR_ARG;
    const Plan& P = c->P;
    if (!P.jk) return LB_ERR_UNSUPPORTED;
    if (nbins > P.sk_max_bins) return LB_ERR_ARG;
    double* bins = c->at<double>(P.sk_bins);
    std::vector<double> hb(2 * size_t(P.sk_max_bins));
    for (int comp = 0; comp < 3 && nbins > 0; ++comp) {
        LB_CHECK(launch_sk_bin(c->at<SkSys>(P.sk_sys), sys, c->at<double>(P.jk_acc) + int64_t(comp) * P.n_sites,
                               nbins, bins, bins + P.sk_max_bins, c->stream));
        LB_CHECK(cudaMemcpyAsync(hb.data(), bins, sizeof(double) * 2 * P.sk_max_bins, cudaMemcpyDeviceToHost,
                                 c->stream));
        LB_CHECK(cudaStreamSynchronize(c->stream));
        for (int j = 0; j < nbins; ++j) {
            h_sum[int64_t(comp) * nbins + j] = hb[j];
            h_count[j] = int64_t(hb[P.sk_max_bins + j]);
        }
    }
    lb_status st = sync_and_check(c);
    if (n_samples) *n_samples = c->step / c->opts.sk_every;
    return st;
}

lb_status lb_oz_fit(int lattice, int side, const double* h_sum, const int64_t* h_count, int kmax, int64_t n_samples,
                    double kT, double out[5]) {
    if ((lattice != LB_D2Q9 && lattice != LB_D3Q19) || side < 2 || !h_sum || !h_count || !out || kmax < 2 ||
        n_samples <= 0 || !(kT > 0))
        return LB_ERR_ARG;
    // shell means of the Laplacian symbol, enumerating the k grid of the lattice
    const bool d3 = lattice == LB_D3Q19;
    static const int c2[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    std::vector<std::array<int, 3>> vel;
    std::vector<double> wt;
    if (d3) {
        for (int x = -1; x <= 1; ++x)
            for (int y = -1; y <= 1; ++y)
                for (int z = -1; z <= 1; ++z) {
                    const int n2 = x * x + y * y + z * z;
                    if (n2 == 1 || n2 == 2) {
                        vel.push_back({x, y, z});
                        wt.push_back(n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                    }
                }
    } else {
        for (int i = 1; i < 9; ++i) {
            vel.push_back({c2[i][0], c2[i][1], c2[i][2]});
            wt.push_back(i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    }
    std::vector<double> ksum(kmax, 0.0);
    std::vector<int64_t> kcnt(kmax, 0);
    const int nzk = d3 ? side : 1;
    const double two_pi = 6.283185307179586476925286766559;
    for (int kz = 0; kz < nzk; ++kz)
        for (int ky = 0; ky < side; ++ky)
            for (int kx = 0; kx < side; ++kx) {
                const int64_t a = 2 * kx < side ? kx : kx - side, b = 2 * ky < side ? ky : ky - side,
                              cz = d3 ? (2 * kz < side ? kz : kz - side) : 0;
                const int64_t n2 = a * a + b * b + cz * cz;
                if (n2 == 0) continue;
                int64_t j = int64_t(std::floor(std::sqrt(double(n2))));
                while (j * (j + 1) < n2) ++j;
                while (j > 0 && j * (j - 1) >= n2) --j;
                if (j < 1 || j > kmax) continue;
                double sym = 0.0;
                for (size_t i = 0; i < vel.size(); ++i) {
                    const double kc = two_pi * (double(a) * vel[i][0] + double(b) * vel[i][1] + double(cz) * vel[i][2]) /
                                      side;
                    sym += 6.0 * wt[i] * (1.0 - std::cos(kc));
                }
                ksum[j - 1] += sym;
                kcnt[j - 1] += 1;
            }
    double A00 = 0, A01 = 0, A11 = 0, r0 = 0, r1 = 0;
    int used = 0;
    for (int j = 0; j < kmax; ++j) {
        if (h_count[j] != kcnt[j]) return LB_ERR_ARG;
        if (kcnt[j] == 0) continue;
        const double C = h_sum[j] / (double(h_count[j]) * double(n_samples));
        if (!(C > 0)) return LB_ERR_ARG;
        const double x = ksum[j] / double(kcnt[j]), y = 1.0 / C, w = double(h_count[j]) * C * C;
        A00 += w;
        A01 += w * x;
        A11 += w * x * x;
        r0 += w * y;
        r1 += w * x * y;
        ++used;
    }
    if (used < 2) return LB_ERR_ARG;
    const double det = A00 * A11 - A01 * A01;
    if (!(det != 0)) return LB_ERR_ARG;
    const double a = (r0 * A11 - r1 * A01) / det, b = (A00 * r1 - A01 * r0) / det;
    out[0] = 1.0 / (kT * a);
    out[1] = (a > 0 && b >= 0) ? std::sqrt(b / a) : NAN;
    out[2] = a;
    out[3] = b;
    out[4] = used;
    return LB_OK;
}

lb_status lb_read_fields(lb_ctx* c, int sys, double* h_f) {
    if (!c || !h_f || sys < 0 || sys >= c->n_sys) return LB_ERR_ARG;
    if (!c->has_state) return LB_ERR_STATE;
    const SysHost& h = c->sys[sys];
    const int buf = int(c->step & 1);
    double* tmp = c->at<double>(c->P.field_tmp);
    for (int i = 0; i < c->q; ++i) {
        LB_CHECK(c->lattice == LB_D2Q9
                     ? launch_gather_d2q9(c->fp32, c->at<SysDev>(c->P.sys), sys, i, h.n, c->pop(buf), tmp, c->stream)
                     : launch_gather_d3q19(c->fp32, c->at<SysDev>(c->P.sys), sys, i, h.n, c->pop(buf), tmp,
                                           c->stream));
        LB_CHECK(cudaMemcpyAsync(h_f + int64_t(i) * h.n, tmp, sizeof(double) * h.n, cudaMemcpyDeviceToHost,
                                 c->stream));
    }
    LB_CHECK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_write_fields(lb_ctx* c, int sys, const double* h_f) {
    if (!c || !h_f || sys < 0 || sys >= c->n_sys) return LB_ERR_ARG;
    const SysHost& h = c->sys[sys];
    const int buf = int(c->step & 1);
    double* tmp = c->at<double>(c->P.field_tmp);
    for (int i = 0; i < c->q; ++i) {
        LB_CHECK(cudaMemcpyAsync(tmp, h_f + int64_t(i) * h.n, sizeof(double) * h.n, cudaMemcpyHostToDevice,
                                 c->stream));
        LB_CHECK(c->lattice == LB_D2Q9
                     ? launch_scatter_d2q9(c->fp32, c->at<SysDev>(c->P.sys), sys, i, h.n, tmp, c->pop(buf), c->stream)
                     : launch_scatter_d3q19(c->fp32, c->at<SysDev>(c->P.sys), sys, i, h.n, tmp, c->pop(buf),
                                            c->stream));
    }
    LB_CHECK(cudaMemsetAsync(c->ws + c->P.status, 0, sizeof(int), c->stream));
    LB_CHECK(cudaStreamSynchronize(c->stream));
    c->sticky = LB_OK;
    c->has_state = true;
    return LB_OK;
}

// Checkpoint file: header, descriptors, populations (raw), accumulators,
// globals, histogram counts, C(k) and momentum-spectrum accumulators.
struct CkptHeader {
    char magic[8];
    int32_t version, lattice, coupling, fp32, n_sys, q;
    int64_t step, n_sites, n_levels;
    int32_t hist_bins, sk_every;
    double hist_range;
    int32_t jk, pad;
};

namespace {

size_t spectra_doubles(const Plan& P) { return (P.sk ? size_t(P.n_sites) : 0) + (P.jk ? 3 * size_t(P.n_sites) : 0); }

// C(k) accumulators then momentum-spectrum accumulators, between host and device.
cudaError_t copy_spectra(lb_ctx* c, double* h, bool to_device) {
    const Plan& P = c->P;
    const size_t nk = P.sk ? size_t(P.n_sites) : 0, nj = P.jk ? 3 * size_t(P.n_sites) : 0;
    const auto kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (nk) e = to_device ? cudaMemcpyAsync(c->ws + P.sk_acc, h, sizeof(double) * nk, kind, c->stream)
                          : cudaMemcpyAsync(h, c->ws + P.sk_acc, sizeof(double) * nk, kind, c->stream);
    if (e == cudaSuccess && nj)
        e = to_device ? cudaMemcpyAsync(c->ws + P.jk_acc, h + nk, sizeof(double) * nj, kind, c->stream)
                      : cudaMemcpyAsync(h + nk, c->ws + P.jk_acc, sizeof(double) * nj, kind, c->stream);
    return e;
}

}  // namespace

lb_status lb_save(lb_ctx* c, const char* path) {
    if (!c || !path) return LB_ERR_ARG;
    if (!c->has_state) return LB_ERR_STATE;
    const Plan& P = c->P;
    const size_t es = c->fp32 ? 4 : 8;
    std::vector<char> pop(es * c->q * P.n_sites);
    std::vector<double> acc(7 * P.n_levels), glob(8 * c->n_sys);
    std::vector<uint64_t> hist(hist_bytes(P) / sizeof(uint64_t));
    std::vector<double> spec(spectra_doubles(P));
    LB_CHECK(cudaMemcpyAsync(pop.data(), c->pop(int(c->step & 1)), pop.size(), cudaMemcpyDeviceToHost, c->stream));
    LB_CHECK(copy_spectra(c, spec.data(), false));
    if (!hist.empty())
        LB_CHECK(cudaMemcpyAsync(hist.data(), c->ws + P.hist, hist_bytes(P), cudaMemcpyDeviceToHost, c->stream));
    LB_CHECK(cudaMemcpyAsync(acc.data(), c->ws + P.acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost,
                             c->stream));
    LB_CHECK(cudaMemcpyAsync(glob.data(), c->ws + P.glob, sizeof(double) * glob.size(), cudaMemcpyDeviceToHost,
                             c->stream));
    LB_CHECK(cudaStreamSynchronize(c->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return LB_ERR_IO;
    CkptHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "LBFLUCT2", 8);
    hd.version = 2;
    hd.hist_bins = P.hist_bins;
    hd.hist_range = P.hist_range;
    hd.sk_every = c->opts.sk_every;
    hd.jk = P.jk ? 1 : 0;
    hd.lattice = c->lattice;
    hd.coupling = c->coupling;
    hd.fp32 = c->fp32;
    hd.n_sys = c->n_sys;
    hd.q = c->q;
    hd.step = c->step;
    hd.n_sites = P.n_sites;
    hd.n_levels = P.n_levels;
    bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1;
    for (auto& h : c->sys) ok = ok && std::fwrite(&h.d, sizeof(lb_system_desc), 1, fp) == 1;
    ok = ok && std::fwrite(pop.data(), 1, pop.size(), fp) == pop.size();
    ok = ok && std::fwrite(acc.data(), sizeof(double), acc.size(), fp) == acc.size();
    ok = ok && std::fwrite(glob.data(), sizeof(double), glob.size(), fp) == glob.size();
    ok = ok && std::fwrite(hist.data(), sizeof(uint64_t), hist.size(), fp) == hist.size();
    ok = ok && std::fwrite(spec.data(), sizeof(double), spec.size(), fp) == spec.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LB_OK : LB_ERR_IO;
}

lb_status lb_load(lb_ctx* c, const char* path) {
    if (!c || !path) return LB_ERR_ARG;
    const Plan& P = c->P;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return LB_ERR_IO;
    CkptHeader hd;
    bool ok = std::fread(&hd, sizeof(hd), 1, fp) == 1 && std::memcmp(hd.magic, "LBFLUCT2", 8) == 0 &&
              hd.version == 2 && hd.lattice == c->lattice && hd.coupling == c->coupling && hd.fp32 == c->fp32 &&
              hd.n_sys == c->n_sys && hd.q == c->q && hd.n_sites == P.n_sites && hd.n_levels == P.n_levels &&
              hd.hist_bins == P.hist_bins && hd.hist_range == P.hist_range && hd.sk_every == c->opts.sk_every &&
              hd.jk == (P.jk ? 1 : 0);
    for (int k = 0; ok && k < c->n_sys; ++k) {
        lb_system_desc d;
        ok = std::fread(&d, sizeof(d), 1, fp) == 1 && std::memcmp(&d, &c->sys[k].d, sizeof(d)) == 0;
    }
    const size_t es = c->fp32 ? 4 : 8;
    std::vector<char> pop(es * c->q * P.n_sites);
    std::vector<double> acc(7 * P.n_levels), glob(8 * c->n_sys);
    std::vector<uint64_t> hist(hist_bytes(P) / sizeof(uint64_t));
    ok = ok && std::fread(pop.data(), 1, pop.size(), fp) == pop.size();
    ok = ok && std::fread(acc.data(), sizeof(double), acc.size(), fp) == acc.size();
    ok = ok && std::fread(glob.data(), sizeof(double), glob.size(), fp) == glob.size();
    ok = ok && std::fread(hist.data(), sizeof(uint64_t), hist.size(), fp) == hist.size();
    std::vector<double> spec(spectra_doubles(P));
    ok = ok && std::fread(spec.data(), sizeof(double), spec.size(), fp) == spec.size();
    std::fclose(fp);
    if (!ok) return LB_ERR_IO;
    drop_graphs(c);
    c->step = hd.step;
    LB_CHECK(cudaMemcpyAsync(c->pop(int(c->step & 1)), pop.data(), pop.size(), cudaMemcpyHostToDevice, c->stream));
    LB_CHECK(cudaMemcpyAsync(c->ws + P.acc, acc.data(), sizeof(double) * acc.size(), cudaMemcpyHostToDevice,
                             c->stream));
    LB_CHECK(cudaMemcpyAsync(c->ws + P.glob, glob.data(), sizeof(double) * glob.size(), cudaMemcpyHostToDevice,
                             c->stream));
    if (!hist.empty())
        LB_CHECK(cudaMemcpyAsync(c->ws + P.hist, hist.data(), hist_bytes(P), cudaMemcpyHostToDevice, c->stream));
    LB_CHECK(copy_spectra(c, spec.data(), true));
    LB_CHECK(cudaMemcpyAsync(c->ws + P.step, &c->step, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    LB_CHECK(cudaMemsetAsync(c->ws + P.status, 0, sizeof(int), c->stream));
    LB_CHECK(cudaStreamSynchronize(c->stream));
    c->sticky = LB_OK;
    c->has_state = true;
    return LB_OK;
}

lb_status lb_inject_fault(lb_ctx* c, int kind, int64_t at_step) {
    if (!c || kind < LB_FAULT_NONE || kind > LB_FAULT_LAUNCH || (kind != LB_FAULT_NONE && at_step <= c->step))
        return LB_ERR_ARG;
    c->fault_kind = kind;
    c->fault_step = kind == LB_FAULT_NONE ? -1 : at_step;
    return LB_OK;
}

lb_status lb_selftest_wait_timeout(int* d_status, void* stream) {
    if (!d_status) return LB_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int h = 0;
    if (cudaMemsetAsync(d_status, 0, sizeof(int), st) != cudaSuccess) return LB_ERR_CUDA;
    if (launch_selftest_wait(d_status, st) != cudaSuccess) return LB_ERR_CUDA;
    if (cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LB_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LB_ERR_CUDA;
    if (h & (1 << 30)) return LB_ERR_STATE;
    return (h & ST_TIMEOUT) ? LB_ERR_TIMEOUT : LB_ERR_STATE;
}

lb_status lb_kernel_variant(lb_ctx* ctx, int* row) {
    if (!ctx || !row) return LB_ERR_ARG;
    *row = ctx->tile_id;
    return LB_OK;
}

int lb_kernel_variants(int lattice, int32_t* out, int max_rows) {
    if (lattice != LB_D2Q9 && lattice != LB_D3Q19) return int(LB_ERR_ARG);
    int t[32][kVariantCols];
    const int nt = tile_table(lattice, t);
    for (int r = 0; r < nt && r < max_rows && out; ++r)
        for (int k = 0; k < kVariantCols; ++k) out[kVariantCols * r + k] = t[r][k];
    return nt;
}

lb_status lb_kernel_launches(lb_ctx* c, int64_t* count) {
    if (!c || !count) return LB_ERR_ARG;
    *count = c->launches;
    return LB_OK;
}

void lb_destroy(lb_ctx* c) {
    if (!c) return;
    drop_graphs(c);
    delete c;
}

}  // extern "C"

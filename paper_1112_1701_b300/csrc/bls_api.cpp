// bls_api.cpp -- C ABI of the BLS library: plans, argument checks, input staging,
// batching of curves into launches, and the batched search (Sec. 2.2.2 of the paper:
// many light curves, every trial period, every box duration and phase, best kept).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include <nvtx3/nvToolsExt.h>

#include "bls_plan.h"

using namespace blsgpu;

static_assert(kSumFixed == BLS_SUM_FIXED && kSumF32 == BLS_SUM_F32 && kSumKahan == BLS_SUM_KAHAN,
              "internal sum modes are the ABI's values");

namespace blsgpu {

static thread_local std::string g_last_error;

bls_status set_error(bls_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

unsigned long long handoff_limit_ns()
{
    if (const char* v = getenv("BLS_HANDOFF_LIMIT_US")) {
        const long long us = atoll(v);
        if (us > 0) return (unsigned long long)us * 1000ull;
    }
    return 30ull * 1000000000ull;
}

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }
void NvtxRange::next(const char* name)
{
    nvtxRangePop();
    nvtxRangePushA(name);
}

bls_status cuda_fail(cudaError_t e, const char* what)
{
    return set_error(e == cudaErrorMemoryAllocation ? BLS_ERR_NOMEM : BLS_ERR_CUDA,
                     "%s: %s", what, cudaGetErrorString(e));
}

cudaError_t DevBuf::ensure(size_t need)
{
    if (need <= bytes && p) return cudaSuccess;
    release();
    size_t sz = need + need / 4 + 256;
    cudaError_t e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) { p = nullptr; bytes = 0; return e; }
    bytes = sz;
    return cudaSuccess;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

cudaError_t HostBuf::ensure(size_t need)
{
    if (need <= bytes && p) return cudaSuccess;
    release();
    size_t sz = need + need / 4 + 256;
    cudaError_t e = cudaMallocHost(&p, sz);
    if (e != cudaSuccess) { p = nullptr; bytes = 0; return e; }
    bytes = sz;
    return cudaSuccess;
}

void HostBuf::release()
{
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
}

// Where an input lives: 0 pageable host, 1 pinned host, 2 device (or managed).
int ptr_kind(const void* p)
{
    if (!p) return 0;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) { cudaGetLastError(); return 0; }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 2;
    return a.type == cudaMemoryTypeHost ? 1 : 0;
}

static bool is_device_ptr(const void* p) { return ptr_kind(p) == 2; }

static bls_status kminmax_impl(int nb, double qmin, double qmax, int* kmin, int* kmax)
{
    if (nb < 2 || !(qmin > 0.0) || !(qmax >= qmin) || !(qmax < 1.0))
        return set_error(BLS_ERR_INVALID, "need nb >= 2 and 0 < qmin <= qmax < 1 (nb=%d qmin=%g qmax=%g)",
                         nb, qmin, qmax);
    int lo = (int)std::floor(qmin * nb + 1e-9);
    int hi = (int)std::ceil(qmax * nb - 1e-9);
    lo = std::max(lo, 1);
    hi = std::min(hi, nb - 1);
    hi = std::max(hi, lo);
    *kmin = lo;
    *kmax = hi;
    return BLS_OK;
}

bls_status resolve_curve(const bls_plan_impl* P, const bls_curve* c, int index, CurveSpec* o,
                         const int* kinds, bool scan_values)
{
    if (!c) return set_error(BLS_ERR_INVALID, "curve %d: NULL descriptor", index);
    if (c->n < 2) return set_error(BLS_ERR_INVALID, "curve %d: n = %d, need n >= 2", index, c->n);
    if (c->nf < 1) return set_error(BLS_ERR_INVALID, "curve %d: nf = %d, need nf >= 1", index, c->nf);
    if (!c->t || !c->y) return set_error(BLS_ERR_INVALID, "curve %d: NULL t or y", index);
    o->t = c->t; o->y = c->y; o->dy = c->dy; o->freqs = c->freqs;
    o->n = c->n; o->nf = c->nf;
    o->fmin = c->fmin; o->df = c->df;
    if (!c->freqs) {
        if (!(c->fmin > 0.0) || !std::isfinite(c->fmin) || !(c->df >= 0.0) || !std::isfinite(c->df))
            return set_error(BLS_ERR_INVALID, "curve %d: uniform grid needs fmin > 0 and df >= 0 (fmin=%g df=%g)",
                             index, c->fmin, c->df);
        double fmax = c->fmin + (double)(c->nf - 1) * c->df;
        if (!std::isfinite(fmax)) return set_error(BLS_ERR_INVALID, "curve %d: grid overflows", index);
    }
    o->nb = c->nb > 0 ? c->nb : P->d.nb;
    double qmin = c->qmin > 0.0 ? c->qmin : P->d.qmin;
    double qmax = c->qmax > 0.0 ? c->qmax : P->d.qmax;
    if (o->nb < 2) return set_error(BLS_ERR_INVALID, "curve %d: nb = %d, need nb >= 2", index, o->nb);
    if (c->nb <= 0 && c->qmin <= 0.0 && c->qmax <= 0.0 && P->d.kmin > 0) {
        o->kmin = P->d.kmin;
        o->kmax = P->d.kmax;
        if (o->kmin < 1 || o->kmax < o->kmin || o->kmax > o->nb)
            return set_error(BLS_ERR_INVALID, "kmin/kmax %d/%d invalid for nb = %d", o->kmin, o->kmax, o->nb);
    } else {
        bls_status s = kminmax_impl(o->nb, qmin, qmax, &o->kmin, &o->kmax);
        if (s != BLS_OK) return set_error(s, "curve %d: %s", index, bls_last_error());
    }
    if (o->nb > 4096) return set_error(BLS_ERR_INVALID, "curve %d: nb = %d exceeds 4096", index, o->nb);
    const int kt = kinds ? kinds[0] : ptr_kind(c->t);
    const int ky = kinds ? kinds[1] : ptr_kind(c->y);
    const int kd = c->dy ? (kinds ? kinds[2] : ptr_kind(c->dy)) : 2;
    const int kf = c->freqs ? (kinds ? kinds[3] : ptr_kind(c->freqs)) : 2;
    o->t_dev = kt == 2;
    o->y_dev = ky == 2;
    o->dy_dev = c->dy ? kd == 2 : false;
    o->f_dev = c->freqs ? kf == 2 : false;
    o->capturable = kt != 0 && ky != 0 && kd != 0 && kf != 0;   // no pageable host copies
    // host values are checked here (unless the caller's prep kernel checks them after the
    // copy); device values by the prep kernel
    if (!scan_values) return BLS_OK;
    if (!o->t_dev)
        for (int i = 0; i < c->n; ++i)
            if (!std::isfinite(c->t[i])) return set_error(BLS_ERR_INVALID, "curve %d: t[%d] is not finite", index, i);
    if (!o->y_dev)
        for (int i = 0; i < c->n; ++i)
            if (!std::isfinite(c->y[i])) return set_error(BLS_ERR_INVALID, "curve %d: y[%d] is not finite", index, i);
    if (c->dy && !o->dy_dev)
        for (int i = 0; i < c->n; ++i)
            if (!(c->dy[i] > 0.0f) || !std::isfinite(c->dy[i]))
                return set_error(BLS_ERR_INVALID, "curve %d: dy[%d] = %g, need finite dy > 0", index, i, (double)c->dy[i]);
    if (c->freqs && !o->f_dev)
        for (int j = 0; j < c->nf; ++j)
            if (!(c->freqs[j] > 0.0) || !std::isfinite(c->freqs[j]))
                return set_error(BLS_ERR_INVALID, "curve %d: freqs[%d] = %g, need finite f > 0", index, j, c->freqs[j]);
    return BLS_OK;
}

bls_status fold_geometry(const bls_plan_impl* P, int nb, int kmin, int kmax, FoldGeom* g)
{
    const int sums = P->d.sum;
    const size_t esz = hist_entry_bytes(sums);
    const int maxT = fold_sweep_max_threads();
    // chunk: a multiple of 16 points; by default the larger of 512/256 that leaves the
    // block size (frequencies per block) as large as 256 allows.  tmax: the most columns
    // (a multiple of 16) whose block fits in shared memory.
    auto tmax = [&](int chunk) {
        const size_t stage = (size_t)2 * chunk * 24;
        const size_t avail = P->smem_optin > stage + kFoldSmemReserve ? P->smem_optin - stage - kFoldSmemReserve : 0;
        int T = (int)std::min<size_t>(avail / ((size_t)nb * esz), (size_t)maxT) & ~15;
        while (T >= 16 && fold_smem_bytes(T, (T + 15) & ~15, nb, chunk, sums) + kFoldSmemReserve > P->smem_optin) T -= 16;
        return T;
    };
    // histogram stride: the warp-specialised kernel packs its columns at any multiple of 8,
    // the one-group kernel rounds up to 16
    auto stride_of = [&](int T) {
        return fold_ws_mode(T, sums, nb, kmin, kmax, P->d.fold_kernel) ? (T + 7) & ~7 : (T + 15) & ~15;
    };
    auto fits = [&](int T, int chunk) {
        return fold_smem_bytes(T, stride_of(T), nb, chunk, sums) + kFoldSmemReserve <= P->smem_optin;
    };
    // (at least 32 points: the staging buffers then also hold the sweep's 2 x 256 partial
    // maxima at the end of a tile)
    const bool chunk_given = P->d.point_chunk > 0, width_given = P->d.freqs_per_block > 0;
    if (chunk_given) g->chunk = std::max(32, (P->d.point_chunk + 15) & ~15);
    else g->chunk = tmax(512) >= tmax(256) ? 512 : 256;
    int T = width_given ? P->d.freqs_per_block
                        : fold_preferred_cols(tmax(g->chunk), sums, nb, kmin, kmax, P->d.fold_kernel);
    if (T > maxT) T = maxT;
    if (width_given && !chunk_given && !fits(T, g->chunk)) {
        // the largest chunk (a multiple of 16, at least 32) with which the given width fits
        int c = g->chunk;
        while (c > 32 && !fits(T, c)) c -= 16;
        g->chunk = c;
    } else if (!width_given && T % 16 == 0 && T + 8 <= 128 &&
               fold_ws_mode(T, sums, nb, kmin, kmax, P->d.fold_kernel) &&
               fold_ws_mode(T + 8, sums, nb, kmin, kmax, P->d.fold_kernel)) {
        // eight more columns in the warp-specialised kernel where a staging chunk of 256 or
        // more points (the one given, else the largest) leaves room: fewer tiles per curve
        // outweigh shorter chunks (survey sweep, nb = 256: 104 columns with 336-point chunks
        // 416 ms per 512 curves, against 444 ms at 96 columns with 512-point chunks)
        for (int c = g->chunk; c >= (chunk_given ? g->chunk : 256); c -= 16)
            if (fits(T + 8, c)) {
                T += 8;
                g->chunk = c;
                break;
            }
    }
    if (T < 8 || (T < 16 && !width_given)) return set_error(BLS_ERR_INVALID, "nb = %d needs more shared memory than a block has", nb);
    g->T = T;
    g->ws = fold_ws_mode(T, sums, nb, kmin, kmax, P->d.fold_kernel);
    g->stride = stride_of(T);
    if (!g->ws && T % 16 != 0)   // the one-group kernel runs 2 T threads: whole warps
        return set_error(BLS_ERR_INVALID, "freqs_per_block = %d: the one-group kernel needs a multiple of 16", T);
    g->smem = fold_smem_bytes(T, g->stride, nb, g->chunk, sums);
    if (g->smem + kFoldSmemReserve > P->smem_optin)
        return set_error(BLS_ERR_INVALID, "nb = %d with %d frequencies per block needs %zu B of shared memory (> %zu)",
                         nb, T, g->smem, P->smem_optin);
    return BLS_OK;
}

void order_by_cost(const std::vector<CurveSpec>& cs, const std::vector<int>& idx,
                   std::vector<int>* out)
{
    *out = idx;
    std::stable_sort(out->begin(), out->end(), [&](int a, int b) {
        double ca = (double)cs[a].n * cs[a].nf, cb = (double)cs[b].n * cs[b].nf;
        return ca > cb;
    });
}

void to_peak(const DevPeak& s, bls_peak* d)
{
    d->best_j = s.j;
    d->i1 = s.i1;
    d->k = s.k;
    d->pad_ = 0;
    d->freq = s.freq;
    d->period = s.period;
    d->epoch = s.epoch;
    d->duration = s.duration;
    d->depth = s.depth;
    d->snr = s.snr;
    d->sr = s.sr;
    d->power = s.power;
    d->sde = s.sde;
}

}  // namespace blsgpu

// ------------------------------------------------------------------------------ search

namespace {

struct Copy {
    void* dst;
    const void* src;
    size_t bytes;
};

// Merge copies whose sources and destinations both continue the previous copy.
void push_copy(std::vector<Copy>& v, void* dst, const void* src, size_t bytes)
{
    if (!v.empty()) {
        Copy& b = v.back();
        if ((const char*)b.src + b.bytes == (const char*)src && (char*)b.dst + b.bytes == (char*)dst) {
            b.bytes += bytes;
            return;
        }
    }
    v.push_back({dst, src, bytes});
}

size_t curve_bytes(const bls_plan_impl* P, const CurveSpec& c, bool host_spec)
{
    size_t n2 = (size_t)((c.n + 1) & ~1);
    size_t b = n2 * (16 + 8) + (size_t)c.nf * 8 + sizeof(CurveDesc) + 64;
    if (!c.t_dev) b += (size_t)c.n * 8;
    if (!c.y_dev) b += (size_t)c.n * 4;
    if (c.dy && !c.dy_dev) b += (size_t)c.n * 4;
    if (c.freqs && !c.f_dev) b += (size_t)c.nf * 8;
    if (host_spec) b += (size_t)c.nf * 4;
    if (P->d.algo == BLS_ALGO_PLAIN_F64) b += n2 * 16;
    if (P->d.algo == BLS_ALGO_UNBINNED) b += (size_t)c.nf * sizeof(int2);
    return b;
}


// One launch group: curves [g0, g1) of `specs`.  Writes peaks to out (host), optionally the
// SR spectra, and (diagnostics) the per-frequency powers into res_dump.
//
// All buffers are sized first; then every stream operation of the group (input copies,
// descriptor and work-list copies, prep, fold-sweep, reduce, result copies) is issued by
// one routine.  When every input is device or pinned host memory, that routine is captured
// into a CUDA graph; while the group's signature (curve descriptors, buffers, options)
// repeats, the graph is replayed with a single launch.
bls_status run_group(bls_plan_impl* P, const std::vector<CurveSpec>& specs, int g0, int g1,
                     const std::vector<long long>& spec_off, bls_peak* out, float* spectrum,
                     bool spectrum_dev, float* res_dump, const ShapeReq* shape)
{
    const int nc = g1 - g0;
    const int topk = P->d.topk;
    cudaStream_t st = P->stream;
    cudaError_t e;
    const bool tiled = P->d.algo == BLS_ALGO_TILED;
    const bool unbinned = P->d.algo == BLS_ALGO_UNBINNED;

    // ---- layout
    std::vector<long long> pt_off(nc), res_off(nc), raw_off(nc), f_off(nc);
    long long npts = 0, nres = 0, nraw = 0, nfr = 0;
    bool any_dy = false, capturable = true;
    size_t plain_hist = 0;
    for (int c = 0; c < nc; ++c) {
        const CurveSpec& s = specs[g0 + c];
        pt_off[c] = npts;
        npts += (s.n + 1) & ~1;
        res_off[c] = nres;
        nres += s.nf;
        raw_off[c] = nraw;
        nraw += s.n;
        f_off[c] = nfr;
        if (s.freqs && !s.f_dev) nfr += s.nf;
        any_dy = any_dy || s.dy;
        capturable = capturable && s.capturable;
        plain_hist = std::max(plain_hist, (size_t)2 * s.nb * s.nf * 8);
    }
    npts += 2;  // slack so a staged chunk never reads past the pool
    int nmax = 2;
    for (int c = 0; c < nc; ++c) nmax = std::max(nmax, specs[g0 + c].n);
    if (unbinned && nmax > kUblsMaxPoints)
        return set_error(BLS_ERR_INVALID, "the unbinned search takes up to %d points per curve (got %d)",
                         kUblsMaxPoints, nmax);

    // fold classes (block size per nb)
    std::vector<FoldGeom> geoms;
    std::vector<std::vector<int>> cls;
    std::vector<int> cls_of(nc, 0);
    if (tiled) {
        for (int c = 0; c < nc; ++c) {
            FoldGeom g;
            bls_status s = fold_geometry(P, specs[g0 + c].nb, specs[g0 + c].kmin, specs[g0 + c].kmax, &g);
            if (s != BLS_OK) return s;
            int k = -1;
            for (size_t q = 0; q < geoms.size(); ++q)
                if (geoms[q].T == g.T && geoms[q].stride == g.stride && geoms[q].chunk == g.chunk &&
                    geoms[q].ws == g.ws) { k = (int)q; break; }
            if (k < 0) { geoms.push_back(g); cls.emplace_back(); k = (int)geoms.size() - 1; }
            else geoms[k].smem = std::max(geoms[k].smem, g.smem);
            cls[k].push_back(c);
            cls_of[c] = k;
        }
    }
    const size_t nr = (size_t)nc;

    // ---- buffers (all before any capture)
#define BLS_ENSURE(buf, bytes, what) \
    if ((e = (buf).ensure(bytes)) != cudaSuccess) return cuda_fail(e, what);
    BLS_ENSURE(P->pts, (size_t)npts * sizeof(float4), "allocating points")
    BLS_ENSURE(P->dt64, (size_t)npts * sizeof(double), "allocating dt")
    BLS_ENSURE(P->res, (size_t)nres * sizeof(float), "allocating results")
    BLS_ENSURE(P->raw_t, (size_t)nraw * 8, "allocating staging")
    BLS_ENSURE(P->raw_y, (size_t)nraw * 4, "allocating staging")
    if (any_dy) BLS_ENSURE(P->raw_dy, (size_t)nraw * 4, "allocating staging")
    if (nfr) BLS_ENSURE(P->raw_f, (size_t)nfr * 8, "allocating staging")
    BLS_ENSURE(P->cdesc, (size_t)nc * sizeof(CurveDesc), "allocating descriptors")
    BLS_ENSURE(P->peaks, (size_t)nc * topk * sizeof(DevPeak), "allocating peaks")
    BLS_ENSURE(P->err, 64, "allocating error word")
    if (spectrum && !spectrum_dev) BLS_ENSURE(P->spec, (size_t)nres * 4, "allocating spectrum")
    BLS_ENSURE(P->h_cdesc, (size_t)nc * sizeof(CurveDesc), "pinned descriptors")
    BLS_ENSURE(P->h_peaks, (size_t)nc * topk * sizeof(DevPeak), "pinned peaks")
    BLS_ENSURE(P->h_err, 64, "pinned error word")
    if (shape) {
        BLS_ENSURE(P->shapes, (size_t)nc * topk * sizeof(DevShape), "allocating shape fits")
        BLS_ENSURE(P->h_shapes, (size_t)nc * topk * sizeof(DevShape), "pinned shape fits")
    }
    if (tiled) {
        BLS_ENSURE(P->ranges, nr * sizeof(TileRange), "allocating work list")
        BLS_ENSURE(P->prefix, (nr + cls.size()) * sizeof(long long), "allocating work list")
        BLS_ENSURE(P->counter, cls.size() * sizeof(int) + 64, "allocating counters")
        BLS_ENSURE(P->h_ranges, nr * sizeof(TileRange), "pinned work list")
        BLS_ENSURE(P->h_prefix, (nr + cls.size()) * sizeof(long long), "pinned work list")
    } else if (unbinned) {
        BLS_ENSURE(P->prefix, (nr + 1) * sizeof(long long), "allocating work list")
        BLS_ENSURE(P->h_prefix, (nr + 1) * sizeof(long long), "pinned work list")
    } else {
        BLS_ENSURE(P->w64, (size_t)npts * 8, "allocating w64")
        BLS_ENSURE(P->wx64, (size_t)npts * 8, "allocating wx64")
        BLS_ENSURE(P->plain_hist, plain_hist, "allocating baseline histograms")
    }
#undef BLS_ENSURE

    // ---- host side: descriptors, input copies (merged when contiguous), work lists
    std::vector<Copy> copies, cy, cdy, cf;   // one list per array so contiguous runs merge
    CurveDesc* hd = P->h_cdesc.as<CurveDesc>();
    for (int c = 0; c < nc; ++c) {
        const CurveSpec& s = specs[g0 + c];
        CurveDesc d;
        memset(&d, 0, sizeof(d));
        if (s.t_dev) d.t = s.t;
        else { d.t = P->raw_t.as<double>() + raw_off[c]; push_copy(copies, (void*)d.t, s.t, (size_t)s.n * 8); }
        if (s.y_dev) d.y = s.y;
        else { d.y = P->raw_y.as<float>() + raw_off[c]; push_copy(cy, (void*)d.y, s.y, (size_t)s.n * 4); }
        if (!s.dy) d.dy = nullptr;
        else if (s.dy_dev) d.dy = s.dy;
        else { d.dy = P->raw_dy.as<float>() + raw_off[c]; push_copy(cdy, (void*)d.dy, s.dy, (size_t)s.n * 4); }
        if (!s.freqs) d.freqs = nullptr;
        else if (s.f_dev) d.freqs = s.freqs;
        else { d.freqs = P->raw_f.as<double>() + f_off[c]; push_copy(cf, (void*)d.freqs, s.freqs, (size_t)s.nf * 8); }
        d.pts = P->pts.as<float4>() + pt_off[c];
        d.dt64 = P->dt64.as<double>() + pt_off[c];
        d.res = P->res.as<float>() + res_off[c];
        d.pt_off = pt_off[c];
        d.spec_off = spectrum_dev ? spec_off[g0 + c] : res_off[c];
        d.fmin = s.fmin;
        d.df = s.df;
        d.n = s.n; d.nf = s.nf; d.nb = s.nb; d.kmin = s.kmin; d.kmax = s.kmax;
        d.T = tiled ? geoms[cls_of[c]].T : 0;
        hd[c] = d;
    }
    copies.insert(copies.end(), cy.begin(), cy.end());
    copies.insert(copies.end(), cdy.begin(), cdy.end());
    copies.insert(copies.end(), cf.begin(), cf.end());

    std::vector<size_t> r0(cls.size()), p0(cls.size());
    std::vector<long long> totals(cls.size());
    size_t pp = 0;
    if (tiled) {
        TileRange* hr = P->h_ranges.as<TileRange>();
        long long* hp = P->h_prefix.as<long long>();
        size_t rr = 0;
        std::vector<CurveSpec> local(specs.begin() + g0, specs.begin() + g1);
        for (size_t q = 0; q < cls.size(); ++q) {
            std::vector<int> ord;
            order_by_cost(local, cls[q], &ord);
            r0[q] = rr;
            p0[q] = pp;
            long long acc = 0;
            for (int c : ord) {
                hr[rr++] = TileRange{c, 0};
                hp[pp++] = acc;
                acc += (local[c].nf + geoms[q].T - 1) / geoms[q].T;
            }
            hp[pp++] = acc;
            totals[q] = acc;
        }
    }
    long long utiles = 0;
    UblsParams up = {};
    if (unbinned) {
        long long* hp = P->h_prefix.as<long long>();
        for (int c = 0; c < nc; ++c) {
            hp[c] = utiles;
            utiles += (specs[g0 + c].nf + ubls_tile() - 1) / ubls_tile();
        }
        hp[nc] = utiles;
        pp = (size_t)nc + 1;
        up.curves = P->cdesc.as<CurveDesc>();
        up.ncurves = nc;
        up.tile_prefix = P->prefix.as<long long>();
        up.res_base = P->res.as<float>();
        up.peaks = P->peaks.as<DevPeak>();
        up.spectrum = spectrum ? (spectrum_dev ? spectrum : P->spec.as<float>()) : nullptr;
        up.topk = topk;
        up.sign = P->d.sign;
        up.qmin = P->d.qmin;
        up.qmax = P->d.qmax;
        up.err = P->err.as<int>();
        up.nmax = nmax;
        up.M = 1;
        while (up.M < nmax) up.M <<= 1;
        up.nitems = utiles;
        // curves too long for a block's shared memory work in a global slice per block
        const size_t wb = ubls_work_bytes(nmax);
        if (wb > P->smem_optin) {
            up.grid = (int)std::min<long long>(utiles, (long long)P->sm_count);
            up.scratch_stride = (wb + 255) & ~(size_t)255;
            if ((e = P->ubls_scratch.ensure(up.scratch_stride * (size_t)up.grid)) != cudaSuccess)
                return cuda_fail(e, "allocating the unbinned working arrays");
            up.scratch = P->ubls_scratch.as<unsigned char>();
        }
    }
    std::vector<int> grids(cls.size());
    for (size_t q = 0; q < cls.size(); ++q) {
        const int bps = fold_blocks_per_sm(geoms[q].T, geoms[q].smem, P->d.phase,
                                           P->d.sum, P->d.sign, geoms[q].ws);
        long long grid = std::min<long long>((long long)P->sm_count * bps, totals[q]);
        grids[q] = (int)std::max<long long>(grid, 1);
    }
    ReduceParams rp;
    rp.curves = P->cdesc.as<CurveDesc>();
    rp.slots = nullptr;
    rp.peaks = P->peaks.as<DevPeak>();
    rp.topk = topk;
    rp.sign = P->d.sign;
    rp.phase = P->d.phase;
    rp.sums = P->d.sum;
    {
        int nbmax = 2;
        for (int c = 0; c < nc; ++c) nbmax = std::max(nbmax, specs[g0 + c].nb);
        rp.smem_bytes = reduce_smem_bytes(nbmax, topk, rp.sums);
        rp.err = P->err.as<int>();
    }
    rp.spectrum = spectrum ? (spectrum_dev ? spectrum : P->spec.as<float>()) : nullptr;
    const bool prof = P->ev[0] != nullptr;
    uint64_t launches = 0, fold_launches = 0;

    // ---- every stream operation of the group
    // inside a capture, an event record becomes a graph node only with the external flag
    // (which is rejected outside a capture)
    bool capturing = false;
    auto record = [&](cudaEvent_t ev) {
        if (capturing) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
        else cudaEventRecord(ev, st);
    };
    const unsigned long long wait_ns = handoff_limit_ns();
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t x;
        launches = 0;
        fold_launches = 0;
        for (const Copy& cp : copies)
            if ((x = cudaMemcpyAsync(cp.dst, cp.src, cp.bytes, cudaMemcpyDefault, st)) != cudaSuccess) return x;
        if ((x = cudaMemcpyAsync(P->cdesc.p, hd, (size_t)nc * sizeof(CurveDesc), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return x;
        if ((x = cudaMemsetAsync(P->err.p, 0, 64, st)) != cudaSuccess) return x;
        if (prof) record(P->ev[0]);
        NvtxRange r_prep("bls.prep");   // then fold_sweep, reduce (host enqueue spans)
        // (the unbinned kernels read FP32 weights)
        if ((x = launch_prep(P->cdesc.as<CurveDesc>(), nullptr, nc, P->err.as<int>(),
                             unbinned ? kPhaseFX64 : P->d.phase, unbinned ? kSumF32 : P->d.sum,
                             st)) != cudaSuccess)
            return x;
        ++launches;
        if (prof) record(P->ev[1]);
        r_prep.next("bls.fold_sweep");
        if (tiled) {
            if ((x = cudaMemcpyAsync(P->ranges.p, P->h_ranges.p, nr * sizeof(TileRange), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (x = cudaMemcpyAsync(P->prefix.p, P->h_prefix.p, pp * sizeof(long long), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (x = cudaMemsetAsync(P->counter.p, 0, cls.size() * sizeof(int), st)) != cudaSuccess)
                return x;
            for (size_t q = 0; q < cls.size(); ++q) {
                FoldParams fp;
                fp.curves = P->cdesc.as<CurveDesc>();
                fp.ranges = P->ranges.as<TileRange>() + r0[q];
                fp.prefix = P->prefix.as<long long>() + p0[q];
                fp.nranges = (int)cls[q].size();
                fp.total = totals[q];
                fp.counter = P->counter.as<int>() + q;
                fp.err = P->err.as<int>();
                fp.chunk = geoms[q].chunk;
                fp.stride = geoms[q].stride;
                fp.wait_ns = wait_ns;
                if ((x = launch_fold_sweep(fp, geoms[q].T, grids[q], P->d.phase, P->d.sum,
                                           geoms[q].ws, P->d.sign, geoms[q].smem, st)) != cudaSuccess)
                    return x;
                ++launches;
                ++fold_launches;
            }
        } else if (unbinned) {
            if ((x = cudaMemcpyAsync(P->prefix.p, P->h_prefix.p, pp * sizeof(long long), cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return x;
            if ((x = launch_ubls(up, st)) != cudaSuccess) return x;
            ++launches;
            ++fold_launches;
        } else {
            if ((x = launch_prep_f64(P->cdesc.as<CurveDesc>(), nc, P->w64.as<double>(), P->wx64.as<double>(), st)) != cudaSuccess)
                return x;
            ++launches;
            for (int c = 0; c < nc; ++c) {
                if ((x = launch_plain_f64(P->cdesc.as<CurveDesc>() + c, P->w64.as<double>(), P->wx64.as<double>(),
                                          specs[g0 + c].nf, P->plain_hist.as<double>(), P->d.sign, st)) != cudaSuccess)
                    return x;
                ++launches;
                ++fold_launches;
            }
        }
        if (prof) record(P->ev[2]);
        r_prep.next("bls.reduce");
        if ((x = unbinned ? launch_ubls_reduce(up, st) : launch_reduce(rp, nc, st)) != cudaSuccess) return x;
        ++launches;
        if (shape) {
            ShapeParams sp;
            sp.curves = P->cdesc.as<CurveDesc>();
            sp.peaks = P->peaks.as<DevPeak>();
            sp.out = P->shapes.as<DevShape>();
            sp.topk = topk;
            sp.nc = shape->nc; sp.nw = shape->nw; sp.na = shape->na;
            sp.wlo = shape->wlo; sp.whi = shape->whi; sp.amax = shape->amax;
            if ((x = launch_shape(sp, nc, st)) != cudaSuccess) return x;
            ++launches;
            if ((x = cudaMemcpyAsync(P->h_shapes.p, P->shapes.p, (size_t)nc * topk * sizeof(DevShape),
                                     cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return x;
        }
        if (prof) record(P->ev[3]);
        if ((x = cudaMemcpyAsync(P->h_peaks.p, P->peaks.p, (size_t)nc * topk * sizeof(DevPeak),
                                 cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return x;
        if (spectrum && !spectrum_dev)
            if ((x = cudaMemcpyAsync(spectrum + spec_off[g0], P->spec.p, (size_t)nres * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return x;
        if (res_dump)
            if ((x = cudaMemcpyAsync(res_dump, P->res.p, (size_t)nres * sizeof(float), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return x;
        return cudaMemcpyAsync(P->h_err.p, P->err.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    };

    // ---- graph replay / capture, or direct launch
    bool launched = false;
    const bool graphable = P->graphs && capturable && !res_dump && (!spectrum || spectrum_dev ||
                                                                   ptr_kind(spectrum) == 1);
    if (graphable) {
        std::string sig;
        auto put = [&](const void* p, size_t n) { sig.append(static_cast<const char*>(p), n); };
        put(&nc, sizeof(nc));
        put(hd, (size_t)nc * sizeof(CurveDesc));
        for (const Copy& cp : copies) put(&cp, sizeof(cp));
        put(&spectrum, sizeof(spectrum));
        put(&P->d, sizeof(P->d));
        put(&wait_ns, sizeof(wait_ns));
        const int shp[3] = {shape ? shape->nc : 0, shape ? shape->nw : 0, shape ? shape->na : 0};
        const double shd[3] = {shape ? shape->wlo : 0.0, shape ? shape->whi : 0.0, shape ? shape->amax : 0.0};
        put(shp, sizeof(shp));
        put(shd, sizeof(shd));
        put(&pp, sizeof(pp));
        if (tiled) {
            put(P->h_ranges.p, nr * sizeof(TileRange));
            put(P->h_prefix.p, pp * sizeof(long long));
        }
        if (unbinned) put(P->h_prefix.p, pp * sizeof(long long));
        void* bufs[] = {P->pts.p, P->res.p, P->peaks.p, P->spec.p, P->err.p, P->h_peaks.p, P->h_err.p, P->ranges.p,
                        P->shapes.p, P->h_shapes.p, P->prefix.p, P->ubls_scratch.p};
        put(bufs, sizeof(bufs));
        if (P->graph && sig == P->graph_sig) {
            if ((e = cudaGraphLaunch(P->graph, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
            launches = P->graph_launches;
            fold_launches = P->graph_fold_launches;
            P->prof.graph_replays += 1;
            launched = true;
        } else {
            if (P->graph) { cudaGraphExecDestroy(P->graph); P->graph = nullptr; P->graph_sig.clear(); }
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                capturing = true;
                cudaError_t x = enqueue();
                capturing = false;
                cudaError_t y = cudaStreamEndCapture(st, &g);
                if (x == cudaSuccess && y == cudaSuccess && g &&
                    cudaGraphInstantiate(&P->graph, g, 0) == cudaSuccess) {
                    P->graph_sig = sig;
                    P->graph_launches = launches;
                    P->graph_fold_launches = fold_launches;
                    P->prof.graph_captures += 1;
                    if ((e = cudaGraphLaunch(P->graph, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
                    launched = true;
                } else {
                    P->graph = nullptr;
                    P->graphs = false;   // not capturable here: launch directly from now on
                }
                if (g) cudaGraphDestroy(g);
            } else {
                P->graphs = false;
            }
            cudaGetLastError();   // a failed capture leaves no sticky error; launch directly
        }
    }
    if (!launched && (e = enqueue()) != cudaSuccess) return cuda_fail(e, "search launch");

    // ---- results
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "search");
    if (prof) {
        float a = 0.f, b = 0.f, c = 0.f;
        cudaEventElapsedTime(&a, P->ev[0], P->ev[1]);
        cudaEventElapsedTime(&b, P->ev[1], P->ev[2]);
        cudaEventElapsedTime(&c, P->ev[2], P->ev[3]);
        cudaGetLastError();
        P->prof.prep_ms += a;
        P->prof.fold_ms += b;
        P->prof.reduce_ms += c;
    }
    P->prof.searches += 1;
    P->prof.kernel_launches += launches;
    P->prof.fold_launches += fold_launches;
    int errw = *P->h_err.as<int>();
    if (errw & kErrInput)
        return set_error(BLS_ERR_INVALID, "a curve has a non-finite time or flux, a non-positive or non-finite error, "
                                          "or a non-positive frequency (device check)");
    if (errw & kErrTimeout)
        return set_error(BLS_ERR_INTERNAL, "a bounded wait between the fold-sweep kernel's warp groups gave up "
                                           "(code %d)", errw);
    if (errw) return set_error(BLS_ERR_INTERNAL, "device consistency check failed (code %d)", errw);
    const DevPeak* hpk = P->h_peaks.as<DevPeak>();
    for (int c = 0; c < nc; ++c)
        for (int q = 0; q < topk; ++q) to_peak(hpk[(size_t)c * topk + q], &out[(size_t)(g0 + c) * topk + q]);
    if (shape) {
        static_assert(sizeof(DevShape) == sizeof(bls_shape), "DevShape mirrors bls_shape");
        memcpy(shape->out + (size_t)g0 * topk, P->h_shapes.p, (size_t)nc * topk * sizeof(bls_shape));
    }
    return BLS_OK;
}

bls_status search_impl(bls_plan_impl* P, const bls_curve* curves, int ncurves, bls_peak* out,
                       float* spectrum, float* res_dump, const ShapeReq* shape = nullptr)
{
    if (ncurves < 0) return set_error(BLS_ERR_INVALID, "ncurves = %d", ncurves);
    if (ncurves == 0) return BLS_OK;
    if (!curves || !out) return set_error(BLS_ERR_INVALID, "NULL curves or out");
    cudaError_t e = cudaSetDevice(P->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    // memory kind of every input array, queried once per contiguous run of curves
    std::vector<CurveSpec> specs(ncurves);
    const void* run_end[4] = {nullptr, nullptr, nullptr, nullptr};
    int run_kind[4] = {0, 0, 0, 0};
    for (int c = 0; c < ncurves; ++c) {
        const bls_curve& cv = curves[c];
        const void* ptrs[4] = {cv.t, cv.y, cv.dy, cv.freqs};
        const size_t sz[4] = {8, 4, 4, 8};
        const long long cnt[4] = {cv.n, cv.n, cv.n, cv.nf};
        int kinds[4];
        for (int a = 0; a < 4; ++a) {
            if (!ptrs[a]) { kinds[a] = 2; continue; }
            if (ptrs[a] != run_end[a]) run_kind[a] = ptr_kind(ptrs[a]);
            kinds[a] = run_kind[a];
            run_end[a] = static_cast<const char*>(ptrs[a]) + (cnt[a] > 0 ? cnt[a] : 0) * sz[a];
        }
        // values are checked by the prep kernel on the device copies (one pass over the
        // points on the device instead of three on the host)
        bls_status s = resolve_curve(P, &cv, c, &specs[c], kinds, false);
        if (s != BLS_OK) return s;
    }
    const bool spec_dev = spectrum && is_device_ptr(spectrum);
    std::vector<long long> spec_off(ncurves + 1, 0);
    for (int c = 0; c < ncurves; ++c) spec_off[c + 1] = spec_off[c] + specs[c].nf;
    // launch groups by memory budget and curve cap
    const int cap = P->d.max_curves_per_launch > 0 ? P->d.max_curves_per_launch : ncurves;
    int g0 = 0;
    while (g0 < ncurves) {
        size_t bytes = 0;
        int g1 = g0;
        while (g1 < ncurves && g1 - g0 < cap) {
            size_t b = curve_bytes(P, specs[g1], spectrum && !spec_dev);
            if (g1 > g0 && bytes + b > P->budget) break;
            bytes += b;
            ++g1;
        }
        if (bytes > P->budget)
            return set_error(BLS_ERR_NOMEM, "curve %d needs %zu B, over the plan's device budget of %zu B", g0,
                             bytes, P->budget);
        bls_status s = run_group(P, specs, g0, g1, spec_off, out, spectrum, spec_dev,
                                 res_dump ? res_dump + spec_off[g0] : nullptr, shape);
        if (s != BLS_OK) return s;
        g0 = g1;
    }
    return BLS_OK;
}

}  // namespace

namespace blsgpu {
bls_status search_one_locked(bls_plan_impl* P, const bls_curve* curve, bls_peak* out)
{
    std::lock_guard<std::mutex> lk(P->mu);
    return search_impl(P, curve, 1, out, nullptr, nullptr);
}
}  // namespace blsgpu

// ------------------------------------------------------------------------------ C ABI

extern "C" {

const char* bls_last_error(void) { return g_last_error.c_str(); }

bls_status bls_moments_of(const float* sr, long long n, bls_moments* out)
{
    if (!out || n < 0 || (n > 0 && !sr)) return set_error(BLS_ERR_INVALID, "bad argument");
    *out = bls_moments{0, 0.0, 0.0};
    if (n == 0) return BLS_OK;
    std::vector<float> host;
    const float* v = sr;
    if (ptr_kind(sr) == 2) {
        try {
            host.resize((size_t)n);
        } catch (const std::bad_alloc&) {
            return set_error(BLS_ERR_NOMEM, "host copy of the spectrum");
        }
        cudaError_t e = cudaMemcpy(host.data(), sr, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "copying the spectrum");
        v = host.data();
    }
    double s = 0.0;
    for (long long i = 0; i < n; ++i) s += (double)v[i];
    const double m = s / (double)n;
    double m2 = 0.0;
    for (long long i = 0; i < n; ++i) {
        const double d = (double)v[i] - m;
        m2 += d * d;
    }
    *out = bls_moments{n, m, m2};
    return BLS_OK;
}

bls_status bls_moments_merge(const bls_moments* parts, int nparts, bls_moments* out)
{
    if (!out || nparts < 0 || (nparts > 0 && !parts)) return set_error(BLS_ERR_INVALID, "bad argument");
    long long n = 0;
    double m = 0.0, m2 = 0.0;
    for (int q = 0; q < nparts; ++q) {
        const bls_moments& b = parts[q];
        if (b.count < 0) return set_error(BLS_ERR_INVALID, "parts[%d].count = %lld", q, b.count);
        if (b.count == 0) continue;
        const double d = b.mean - m;
        const double tot = (double)(n + b.count);
        m = m + d * (double)b.count / tot;
        m2 = m2 + b.m2 + d * d * (double)n * (double)b.count / tot;
        n += b.count;
    }
    *out = bls_moments{n, m, m2};
    return BLS_OK;
}

bls_status bls_sde(double sr, const bls_moments* m, double* sde)
{
    if (!m || !sde || m->count < 0) return set_error(BLS_ERR_INVALID, "bad argument");
    const double sd = m->count > 0 ? sqrt(m->m2 / (double)m->count) : 0.0;
    *sde = sd > 0.0 ? (sr - m->mean) / sd : 0.0;
    return BLS_OK;
}

bls_status bls_kminmax(int nb, double qmin, double qmax, int* kmin, int* kmax)
{
    if (!kmin || !kmax) return set_error(BLS_ERR_INVALID, "NULL output");
    return kminmax_impl(nb, qmin, qmax, kmin, kmax);
}

bls_status bls_plan_create(const bls_plan_desc* desc, void* cuda_stream, bls_plan** out)
{
    if (!desc || !out) return set_error(BLS_ERR_INVALID, "NULL descriptor or output");
    *out = nullptr;
    bls_plan_desc d = *desc;
    if (d.nb < 2) return set_error(BLS_ERR_INVALID, "nb = %d, need nb >= 2", d.nb);
    if (d.kmin > 0 || d.kmax > 0) {
        if (d.kmin < 1 || d.kmax < d.kmin || d.kmax > d.nb)
            return set_error(BLS_ERR_INVALID, "need 1 <= kmin <= kmax <= nb (kmin=%d kmax=%d nb=%d)", d.kmin, d.kmax, d.nb);
    } else {
        int a, b;
        bls_status s = kminmax_impl(d.nb, d.qmin, d.qmax, &a, &b);
        if (s != BLS_OK) return s;
    }
    if (d.topk < 1 || d.topk > kMaxTopK) return set_error(BLS_ERR_INVALID, "topk = %d, need 1..%d", d.topk, kMaxTopK);
    if (d.phase < 0 || d.phase > 3) return set_error(BLS_ERR_INVALID, "phase = %d", d.phase);
    if (d.sum < 0 || d.sum > 2) return set_error(BLS_ERR_INVALID, "sum = %d", d.sum);
    if (d.sign < 0 || d.sign > 1) return set_error(BLS_ERR_INVALID, "sign = %d", d.sign);
    if (d.algo < 0 || d.algo > 2) return set_error(BLS_ERR_INVALID, "algo = %d", d.algo);
    if (d.freqs_per_block < 0 || d.freqs_per_block > fold_sweep_max_threads() || (d.freqs_per_block % 8) != 0)
        return set_error(BLS_ERR_INVALID, "freqs_per_block = %d, need a multiple of 8 up to %d", d.freqs_per_block,
                         fold_sweep_max_threads());
    if (d.point_chunk < 0 || d.point_chunk > 4096) return set_error(BLS_ERR_INVALID, "point_chunk = %d", d.point_chunk);
    if (d.fold_kernel < BLS_FOLD_AUTO || d.fold_kernel > BLS_FOLD_ONE_GROUP)
        return set_error(BLS_ERR_INVALID, "fold_kernel = %d", d.fold_kernel);
    if (d.max_curves_per_launch < 0 || d.max_active_requests < 0 || d.step_point_freqs < 0)
        return set_error(BLS_ERR_INVALID, "negative limit");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int sms = 0, optin = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "device attributes");
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return cuda_fail(e, "device attributes");
    bls_plan* P = new (std::nothrow) bls_plan();
    if (!P) return set_error(BLS_ERR_NOMEM, "plan allocation");
    P->d = d;
    P->device = dev;
    P->sm_count = sms;
    P->smem_optin = (size_t)optin - 1024;   // static shared memory of the kernels
    if (const char* g = getenv("BLS_NO_GRAPHS")) P->graphs = atoi(g) == 0;
    if (cuda_stream) {
        P->stream = (cudaStream_t)cuda_stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking)) != cudaSuccess) {
            delete P;
            return cuda_fail(e, "stream creation");
        }
        P->own_stream = true;
    }
    if (d.max_device_bytes > 0) {
        P->budget = d.max_device_bytes;
    } else {
        size_t fr = 0, tot = 0;
        if ((e = cudaMemGetInfo(&fr, &tot)) != cudaSuccess) {
            if (P->own_stream) cudaStreamDestroy(P->stream);
            delete P;
            return cuda_fail(e, "cudaMemGetInfo");
        }
        P->budget = fr / 2;
    }
    for (int q = 0; q < 4; ++q)
        if (cudaEventCreate(&P->ev[q]) != cudaSuccess) { cudaGetLastError(); P->ev[0] = nullptr; break; }
    if (d.algo == BLS_ALGO_TILED) {
        FoldGeom g;
        int kmin = 1, kmax = 1;
        bls_status s = bls_kminmax(d.nb, d.qmin, d.qmax, &kmin, &kmax);
        if (s == BLS_OK) s = fold_geometry(P, d.nb, kmin, kmax, &g);
        if (s != BLS_OK) {
            if (P->own_stream) cudaStreamDestroy(P->stream);
            delete P;
            return s;
        }
    }
    *out = P;
    return BLS_OK;
}

void bls_plan_destroy(bls_plan* P)
{
    if (!P) return;
    server_destroy(P);
    cudaSetDevice(P->device);
    if (P->stream) cudaStreamSynchronize(P->stream);
    DevBuf* bufs[] = {&P->raw_t, &P->raw_y, &P->raw_dy, &P->raw_f, &P->pts, &P->dt64, &P->w64,
                      &P->wx64, &P->cdesc, &P->ranges, &P->prefix, &P->counter, &P->err, &P->res,
                      &P->peaks, &P->spec, &P->plain_hist, &P->jsbuf, &P->binsbuf, &P->shapes,
                      &P->ubls_scratch};
    for (DevBuf* b : bufs) b->release();
    HostBuf* hb[] = {&P->h_cdesc, &P->h_ranges, &P->h_prefix, &P->h_peaks, &P->h_err, &P->h_shapes};
    for (HostBuf* b : hb) b->release();
    for (int q = 0; q < 4; ++q)
        if (P->ev[q]) cudaEventDestroy(P->ev[q]);
    if (P->graph) cudaGraphExecDestroy(P->graph);
    if (P->own_stream) cudaStreamDestroy(P->stream);
    delete P;
}

bls_status bls_profile_get(bls_plan* P, bls_profile* out, int reset)
{
    if (!P || !out) return set_error(BLS_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(P->mu);
    *out = P->prof;
    if (reset) P->prof = bls_profile{};
    return BLS_OK;
}

bls_status bls_search(bls_plan* P, const bls_curve* curves, int ncurves, bls_peak* out, float* spectrum)
{
    if (!P) return set_error(BLS_ERR_INVALID, "NULL plan");
    NvtxRange r("bls.search");
    std::lock_guard<std::mutex> lk(P->mu);
    return search_impl(P, curves, ncurves, out, spectrum, nullptr);
}

// Fine-grid re-search around every peak: the frequencies of peak q of curve c are
// f_q + (i - half*oversample) * step, i = 0 .. 2*half*oversample (FP64, one rounded product
// and one rounded sum each, non-positive ones dropped), step = the curve's grid spacing
// divided by oversample (explicit grids: half the distance between best_j's neighbours).
bls_status bls_refine(bls_plan* P, const bls_curve* curves, int ncurves, const bls_peak* coarse,
                      int oversample, int half, bls_peak* out)
{
    if (!P || !curves || !coarse || !out) return set_error(BLS_ERR_INVALID, "NULL argument");
    if (ncurves < 0) return set_error(BLS_ERR_INVALID, "ncurves = %d", ncurves);
    if (oversample < 1 || half < 1 || (long long)2 * half * oversample + 1 > (1 << 24))
        return set_error(BLS_ERR_INVALID, "oversample = %d, half = %d", oversample, half);
    std::lock_guard<std::mutex> lk(P->mu);
    const int K = P->d.topk;
    const int nfine = 2 * half * oversample + 1;
    std::vector<bls_curve> fc;
    std::vector<int> slot;                 // output slot of every fine search
    std::vector<std::vector<double>> grids;
    for (int c = 0; c < ncurves; ++c) {
        const bls_curve& cv = curves[c];
        for (int q = 0; q < K; ++q) {
            const bls_peak& pk = coarse[(size_t)c * K + q];
            bls_peak& o = out[(size_t)c * K + q];
            memset(&o, 0, sizeof(o));
            o.best_j = -1;
            if (pk.best_j < 0) continue;
            if (pk.best_j >= cv.nf || cv.nf < 1)
                return set_error(BLS_ERR_INVALID, "curve %d peak %d: best_j = %d outside the grid", c, q, pk.best_j);
            double step;
            if (!cv.freqs) {
                step = cv.df / (double)oversample;
            } else {
                const int a = pk.best_j > 0 ? pk.best_j - 1 : pk.best_j;
                const int b = pk.best_j + 1 < cv.nf ? pk.best_j + 1 : pk.best_j;
                const double span = b > a ? (cv.freqs[b] - cv.freqs[a]) / (double)(b - a) : 0.0;
                step = span / (double)oversample;
            }
            std::vector<double> g;
            g.reserve(nfine);
            for (int i = 0; i < nfine; ++i) {
                const double f = pk.freq + (double)(i - half * oversample) * step;
                if (f > 0.0) g.push_back(f);
            }
            if (g.empty() || !(step > 0.0)) g.assign(1, pk.freq);
            grids.push_back(std::move(g));
            bls_curve f2 = cv;
            f2.nf = (int)grids.back().size();
            slot.push_back(c * K + q);
            fc.push_back(f2);
        }
    }
    for (size_t i = 0; i < fc.size(); ++i) fc[i].freqs = grids[i].data();
    if (fc.empty()) return BLS_OK;
    std::vector<bls_peak> tmp(fc.size() * (size_t)K);
    bls_status s = search_impl(P, fc.data(), (int)fc.size(), tmp.data(), nullptr, nullptr);
    if (s != BLS_OK) return s;
    for (size_t i = 0; i < fc.size(); ++i) out[slot[i]] = tmp[i * (size_t)K];
    return BLS_OK;
}

bls_status bls_search_shapes(bls_plan* P, const bls_curve* curves, int ncurves, bls_peak* out,
                             float* spectrum, const bls_shape_grid* grid, bls_shape* shapes)
{
    if (!P || !shapes) return set_error(BLS_ERR_INVALID, "NULL plan or shapes");
    if (P->d.algo == BLS_ALGO_UNBINNED)
        return set_error(BLS_ERR_INVALID, "the trapezoid refit starts from binned boxes (plan algo is unbinned)");
    ShapeReq r;
    r.nc = grid && grid->ncentre ? grid->ncentre : 17;
    r.nw = grid && grid->nwidth ? grid->nwidth : 13;
    r.na = grid && grid->ningress ? grid->ningress : 6;
    r.wlo = grid && grid->width_lo != 0.0 ? grid->width_lo : 0.5;
    r.whi = grid && grid->width_hi != 0.0 ? grid->width_hi : 2.0;
    r.amax = grid && grid->ingress_max >= 0.0 ? grid->ingress_max : 0.5;
    r.out = shapes;
    if (r.nc < 1 || r.nw < 1 || r.na < 1 || (long long)r.nc * r.nw * r.na > (1 << 20))
        return set_error(BLS_ERR_INVALID, "shape grid %d x %d x %d", r.nc, r.nw, r.na);
    if (!(r.wlo > 0.0) || !(r.whi >= r.wlo) || !(r.amax >= 0.0 && r.amax <= 0.5))
        return set_error(BLS_ERR_INVALID, "shape grid widths %g..%g, ingress %g", r.wlo, r.whi, r.amax);
    std::lock_guard<std::mutex> lk(P->mu);
    return search_impl(P, curves, ncurves, out, spectrum, nullptr, &r);
}

bls_status bls_debug_powers(bls_plan* P, const bls_curve* curve, float* power_out, int* i1_out, int* k_out)
{
    if (!P || !curve || !power_out || !i1_out || !k_out) return set_error(BLS_ERR_INVALID, "NULL argument");
    if (curve->nf < 1) return set_error(BLS_ERR_INVALID, "nf = %d", curve->nf);
    std::lock_guard<std::mutex> lk(P->mu);
    std::vector<bls_peak> pk((size_t)P->d.topk);
    bls_status s = search_impl(P, curve, 1, pk.data(), nullptr, power_out);
    if (s != BLS_OK) return s;
    // the best box of every frequency, recomputed with the exact tie-break on the curve the
    // search just prepared (its descriptor is still the first one on the device)
    const int nf = curve->nf;
    int nb = curve->nb > 0 ? curve->nb : P->d.nb;
    cudaError_t e;
    if ((e = P->jsbuf.ensure((size_t)nf * 12)) != cudaSuccess) return cuda_fail(e, "allocating");
    float* dP = P->jsbuf.as<float>();
    int* di1 = reinterpret_cast<int*>(dP + nf);
    int* dk = di1 + nf;
    if ((e = launch_argmax(P->cdesc.as<CurveDesc>(), nb, nf, P->d.phase, P->d.sum,
                           P->d.sign, dP, di1, dk, P->stream)) != cudaSuccess)
        return cuda_fail(e, "best-box launch");
    if ((e = cudaMemcpyAsync(i1_out, di1, (size_t)nf * 4, cudaMemcpyDeviceToHost, P->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(k_out, dk, (size_t)nf * 4, cudaMemcpyDeviceToHost, P->stream)) != cudaSuccess)
        return cuda_fail(e, "copy");
    if ((e = cudaStreamSynchronize(P->stream)) != cudaSuccess) return cuda_fail(e, "best box");
    return BLS_OK;
}

bls_status bls_tile_shape(bls_plan* P, int nb, int* cols, int* chunk, int* ws)
{
    if (!P || !cols || !chunk || !ws) return set_error(BLS_ERR_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(P->mu);
    if (P->d.algo != BLS_ALGO_TILED) return set_error(BLS_ERR_INVALID, "the plan's search has no tiles");
    const bool own = nb == 0;
    if (own) nb = P->d.nb;
    if (nb < 2 || nb > 4096) return set_error(BLS_ERR_INVALID, "nb = %d, need 2..4096", nb);
    // the widths as bls_search resolves them for a curve with this nb and the plan's q range
    int kmin = P->d.kmin, kmax = P->d.kmax;
    if (!(own && kmin > 0)) {
        bls_status st = kminmax_impl(nb, P->d.qmin, P->d.qmax, &kmin, &kmax);
        if (st != BLS_OK) return st;
    }
    FoldGeom g;
    bls_status st = fold_geometry(P, nb, kmin, kmax, &g);
    if (st != BLS_OK) return st;
    *cols = g.T;
    *chunk = g.chunk;
    *ws = g.ws;
    return BLS_OK;
}

bls_status bls_debug_fold(bls_plan* P, const bls_curve* curve, const int* js, int nj, int* bins_out)
{
    if (!P || !curve || !js || !bins_out || nj < 1) return set_error(BLS_ERR_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(P->mu);
    cudaError_t e = cudaSetDevice(P->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    CurveSpec s;
    bls_status st = resolve_curve(P, curve, 0, &s);
    if (st != BLS_OK) return st;
    for (int q = 0; q < nj; ++q)
        if (js[q] < 0 || js[q] >= s.nf) return set_error(BLS_ERR_INVALID, "js[%d] = %d out of range", q, js[q]);
    // prepare the curve exactly as a search does, then fold with the search's device code
    std::vector<CurveSpec> specs{s};
    std::vector<long long> off{0, s.nf};
    std::vector<bls_peak> pk((size_t)P->d.topk);
    bls_plan_desc saved = P->d;
    st = run_group(P, specs, 0, 1, off, pk.data(), nullptr, false, nullptr, nullptr);
    P->d = saved;
    if (st != BLS_OK) return st;
    if ((e = P->jsbuf.ensure((size_t)nj * 4)) != cudaSuccess) return cuda_fail(e, "allocating");
    if ((e = P->binsbuf.ensure((size_t)nj * s.n * 4)) != cudaSuccess) return cuda_fail(e, "allocating");
    if ((e = cudaMemcpyAsync(P->jsbuf.p, js, (size_t)nj * 4, cudaMemcpyHostToDevice, P->stream)) != cudaSuccess)
        return cuda_fail(e, "copy");
    // the tile width the search used for this curve (the incremental fold's reference
    // column depends on it)
    FoldGeom g;
    if (P->d.algo == BLS_ALGO_TILED) {
        if ((st = fold_geometry(P, s.nb, s.kmin, s.kmax, &g)) != BLS_OK) return st;
    } else {
        g.T = 1;   // no tiles: the incremental fold is not used
    }
    if ((e = launch_debug_fold(P->cdesc.as<CurveDesc>(), P->jsbuf.as<int>(), nj, P->d.phase, g.T,
                               P->d.algo == BLS_ALGO_TILED ? P->d.sum : kSumKahan,
                               P->binsbuf.as<int>(), P->stream)) != cudaSuccess)
        return cuda_fail(e, "debug fold launch");
    if ((e = cudaMemcpyAsync(bins_out, P->binsbuf.p, (size_t)nj * s.n * 4, cudaMemcpyDeviceToHost, P->stream)) != cudaSuccess)
        return cuda_fail(e, "copy");
    if ((e = cudaStreamSynchronize(P->stream)) != cudaSuccess) return cuda_fail(e, "debug fold");
    return BLS_OK;
}

}  // extern "C"

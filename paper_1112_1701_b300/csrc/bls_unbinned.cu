// bls_unbinned.cu -- unbinned (edge-to-edge) BLS: the box edges sit on data points.
//
// At every trial frequency the points are ordered by phase and every cyclic run of
// consecutive points whose phase extent lies in [qmin, qmax] is a box, scored with the
// binned search's statistic (r = sum w, s = sum w x over the run, P = s^2/(r(1-r)), dips
// only by default).  Phases are 64-bit fixed-point fractions: with DT = RN_int(dt 2^s)
// (written by the prep kernel in the fixed-point layout) and F = RN_int(f 2^(64-s)), a
// point's key is the high word of (DT F) mod 2^64, three integer multiply-adds.  The order
// is (key, point index); a run's extent is (key_last - key_first) mod 2^32, compared with
// QMIN = ceil(qmin 2^32) and QMAX = floor(qmax 2^32).  Ordering and extents are therefore
// exact integer decisions, the same in every implementation.
//
// Search kernel: one block per (curve, tile of kTile frequencies).  For each frequency the
// block forms the keys (key << 32 | index) in shared memory, sorts them with a bitonic
// network, and builds prefix sums of (w, w x) in phase order (FP64, stored as double-float
// pairs).  Each thread takes a range of run starts; the admissible ends of a start (extent
// within [QMIN, QMAX]) only move right as the start does, so two pointers give them, and
// every run's sums are independent prefix differences.  The largest P wins (ties to the
// smaller start, then the shorter run); a block argmax gives P(f_j) and its run.
//
// Reduce kernel: one block per curve: the top-k local maxima of P(f_j) (as in the binned
// search), the signal detection efficiency, and for each kept frequency the run's FP64
// refit -- keys and order recomputed exactly, r and s summed in run order in FP64.
#include <cfloat>

#include "bls_internal.h"

namespace blsgpu {
namespace {

constexpr int kUThreads = 512;
constexpr int kTile = 16;

__host__ __device__ __forceinline__ int shift_of(double dtmax)
{
    int L = 0;
    if (dtmax > 0.0) L = ilogb(dtmax) + 1;
    int s = 34 - (L + 1) / 2;
    if (s > 62 - L) s = 62 - L;
    return s < 1 ? 1 : s;
}

__device__ __forceinline__ unsigned long long fixed_freq(double f, double dtmax)
{
    return __double2ull_rn(ldexp(f, 64 - shift_of(dtmax)));
}

// Phase keys (key << 32 | point) of a curve at F, bitonic-sorted ascending in `keys`
// (M = the power of two >= n; the tail holds all-ones sentinels).
__device__ void sorted_keys(const CurveDesc& cd, unsigned long long F, unsigned long long* keys, int M)
{
    const unsigned Flo = (unsigned)F, Fhi = (unsigned)(F >> 32);
    const int n = cd.n;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        unsigned long long k = ~0ull;
        if (i < n) {
            const float4 A = cd.pts[(i >> 1) * 2];
            const unsigned lo = __float_as_uint((i & 1) ? A.y : A.x);
            const unsigned hi = __float_as_uint((i & 1) ? A.w : A.z);
            const unsigned q = __umulhi(lo, Flo) + lo * Fhi + hi * Flo;
            k = ((unsigned long long)q << 32) | (unsigned)i;
        }
        keys[i] = k;
    }
    __syncthreads();
    for (int size = 2; size <= M; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (M >> 1); t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = keys[lo], b = keys[hi];
                if ((a > b) == up) { keys[lo] = b; keys[hi] = a; }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ void point_weights(const CurveDesc& cd, int i, float& w, float& wx)
{
    const float4 B = cd.pts[(i >> 1) * 2 + 1];
    w = (i & 1) ? B.z : B.x;
    wx = (i & 1) ? B.w : B.y;
}

// (P, start, len) order: larger P, then smaller start, then shorter run.
__device__ __forceinline__ bool run_ahead(float pa, int sa, int la, float pb, int sb, int lb)
{
    return pa > pb || (pa == pb && (sa < sb || (sa == sb && la < lb)));
}

// Double-float value (hi + lo) of an FP64 number.
__device__ __forceinline__ float2 split_df(double v)
{
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(__dsub_rn(v, (double)hi)));
}

// Error-free sum of two floats (Knuth's two-sum): hi + lo == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& hi, float& lo)
{
    hi = a + b;
    const float bb = hi - a;
    lo = (a - (hi - bb)) + (b - bb);
}

// Score of one run with sums (r, s): P = s^2 / (r(1-r)), dips only unless sign; 0 if the
// run does not count.  An approximate division suffices: P only ranks the runs of a
// frequency (the kept run is refitted in FP64).
__device__ __forceinline__ float run_score(float r, float s, int sign)
{
    const float d = fmaf(-r, r, r);
    if (!(d > 0.0f) || (!sign && !(s < 0.0f))) return 0.0f;
    return __fdividef(s * s, d);
}

__global__ void __launch_bounds__(kUThreads) ubls_kernel(UblsParams p)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ float sP[kUThreads / 32];
    __shared__ int sS[kUThreads / 32], sL[kUThreads / 32];
    __shared__ double sred[2 * kUThreads];
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(dsm);
    float4* C = reinterpret_cast<float4*>(keys + p.M);      // n + 1 prefix entries
    // work item -> (curve, tile)
    const long long it = blockIdx.x;
    int lo = 0, hi = p.ncurves;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (p.tile_prefix[mid] <= it) lo = mid; else hi = mid;
    }
    const CurveDesc& cd = p.curves[lo];
    const int n = cd.n;
    const int j0 = (int)(it - p.tile_prefix[lo]) * kTile;
    int M = 1;
    while (M < n) M <<= 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = blockDim.x;
    const int ch = (n + nt - 1) / nt;                 // positions per thread
    const int q0 = min(n, (int)threadIdx.x * ch), q1 = min(n, q0 + ch);
    for (int j = j0; j < min(j0 + kTile, cd.nf); ++j) {
        const double f = cd.freqs ? cd.freqs[j] : __dadd_rn(cd.fmin, __dmul_rn((double)j, cd.df));
        sorted_keys(cd, fixed_freq(f, cd.dtmax), keys, M);
        // prefix sums in phase order: FP64 over each thread's positions, a scan of the
        // thread totals, then double-float values in shared memory
        double tw = 0.0, tx = 0.0;
        for (int q = q0; q < q1; ++q) {
            float w, wx;
            point_weights(cd, (int)(keys[q] & 0xffffffffu), w, wx);
            tw = __dadd_rn(tw, (double)w);
            tx = __dadd_rn(tx, (double)wx);
        }
        // exclusive scan of the thread totals: inclusive scans within warps (shuffles),
        // then the warp totals in order
        double iw = tw, ix = tx;
        for (int o = 1; o < 32; o <<= 1) {
            const double uw = __shfl_up_sync(0xffffffffu, iw, o);
            const double ux = __shfl_up_sync(0xffffffffu, ix, o);
            if (lane >= o) { iw = __dadd_rn(iw, uw); ix = __dadd_rn(ix, ux); }
        }
        if (lane == 31) { sred[warp] = iw; sred[nt + warp] = ix; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double aw = 0.0, ax = 0.0;
            for (int w = 0; w < nt / 32; ++w) {
                const double vw = sred[w], vx = sred[nt + w];
                sred[w] = aw;
                sred[nt + w] = ax;
                aw = __dadd_rn(aw, vw);
                ax = __dadd_rn(ax, vx);
            }
            const float2 W = split_df(aw), X = split_df(ax);
            C[n] = make_float4(W.x, W.y, X.x, X.y);
        }
        __syncthreads();
        const double base_w = __dsub_rn(__dadd_rn(sred[warp], iw), tw);
        const double base_x = __dsub_rn(__dadd_rn(sred[nt + warp], ix), tx);
        __syncthreads();
        {
            double aw = base_w, ax = base_x;
            for (int q = q0; q < q1; ++q) {
                const float2 W = split_df(aw), X = split_df(ax);
                C[q] = make_float4(W.x, W.y, X.x, X.y);
                float w, wx;
                point_weights(cd, (int)(keys[q] & 0xffffffffu), w, wx);
                aw = __dadd_rn(aw, (double)w);
                ax = __dadd_rn(ax, (double)wx);
            }
        }
        __syncthreads();
        const float4 T = C[n];
        // runs: starts dealt round-robin to the threads (phases clump, so contiguous ranges
        // would leave the threads unevenly loaded); the ends [emin, emax] of a start
        // (unwrapped positions; extents within [QMIN, QMAX], at most n - 1 points) by
        // binary search, extents growing with the end.  Run sums are prefix differences;
        // runs past the end add the totals with an error-free sum, so both cases keep
        // double-float accuracy.
        float bp = 0.0f;
        int bs = 0x7fffffff, bl = 0x7fffffff;
        for (int a = threadIdx.x; a < n; a += nt) {
            const unsigned k0 = (unsigned)(keys[a] >> 32);
            auto ext = [&](int e) { return (unsigned)(keys[e < n ? e : e - n] >> 32) - k0; };
            // largest e in [a, a + n - 2] with ext(e) <= QMAX (ext(a) = 0)
            int lo2 = a, hi2 = a + n - 1;            // ext(lo2) <= QMAX; hi2 out of range
            while (hi2 - lo2 > 1) {
                const int mid = (lo2 + hi2) >> 1;
                if (ext(mid) <= p.QMAX) lo2 = mid; else hi2 = mid;
            }
            const int emax = lo2;
            // smallest e in [a, emax] with ext(e) >= QMIN
            int lo1 = a - 1, hi1 = emax + 1;          // ext(hi1) >= QMIN or hi1 past emax
            while (hi1 - lo1 > 1) {
                const int mid = (lo1 + hi1) >> 1;
                if (ext(mid) >= p.QMIN) hi1 = mid; else lo1 = mid;
            }
            const int emin = hi1;
            const float4 ca = C[a];
            const int e1 = min(emax, n - 1);
#pragma unroll 4
            for (int e = emin; e <= e1; ++e) {            // runs inside [a, n)
                const float4 cb = C[e + 1];
                const float r = (cb.x - ca.x) + (cb.y - ca.y);
                const float s = (cb.z - ca.z) + (cb.w - ca.w);
                const float P = run_score(r, s, p.sign);
                if (P > bp) { bp = P; bs = a; bl = e - a + 1; }
            }
            for (int e = max(emin, n); e <= emax; ++e) {  // runs that wrap past the end
                const float4 c = C[e + 1 - n];
                float wh, wl, xh, xl;
                two_sum(T.x, c.x, wh, wl);
                two_sum(T.z, c.z, xh, xl);
                const float r = (wh - ca.x) + ((wl + T.y + c.y) - ca.y);
                const float s = (xh - ca.z) + ((xl + T.w + c.w) - ca.w);
                const float P = run_score(r, s, p.sign);
                if (P > bp) { bp = P; bs = a; bl = e - a + 1; }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float op = __shfl_xor_sync(0xffffffffu, bp, o);
            const int os = __shfl_xor_sync(0xffffffffu, bs, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (run_ahead(op, os, ol, bp, bs, bl)) { bp = op; bs = os; bl = ol; }
        }
        if (lane == 0) { sP[warp] = bp; sS[warp] = bs; sL[warp] = bl; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (run_ahead(sP[w], sS[w], sL[w], sP[0], sS[0], sL[0])) { sP[0] = sP[w]; sS[0] = sS[w]; sL[0] = sL[w]; }
            const long long o = cd.res - p.res_base;
            cd.res[j] = sP[0];
            p.runs[o + j] = make_int2(sP[0] > 0.0f ? sS[0] : 0, sP[0] > 0.0f ? sL[0] : 0);
        }
        __syncthreads();
    }
}

__device__ double sum_block(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ bool freq_ahead(float pa, int ja, float pb, int jb)
{
    return pa > pb || (pa == pb && ja < jb);
}

__global__ void __launch_bounds__(kUThreads) ubls_reduce_kernel(UblsParams p)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(dsm);
    __shared__ double red[kUThreads];
    __shared__ float sP[kUThreads / 32];
    __shared__ int sJ[kUThreads / 32], sT[kUThreads / 32];
    __shared__ int sel[kMaxTopK];
    const CurveDesc& cd = p.curves[blockIdx.x];
    const float* res = cd.res;
    const int nf = cd.nf, K = p.topk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // local maxima, best K per thread; spectrum; SR sums for the SDE
    float lp[kMaxTopK];
    int lj[kMaxTopK];
    int cnt = 0;
    double srsum = 0.0;
    for (int j = threadIdx.x; j < nf; j += blockDim.x) {
        const float P = res[j];
        const float sr = sqrtf(P);
        if (p.spectrum) p.spectrum[cd.spec_off + j] = sr;
        srsum = __dadd_rn(srsum, (double)sr);
        const bool lm = (j == 0 || P > res[j - 1]) && (j == nf - 1 || P >= res[j + 1]);
        if (!lm) continue;
        int pos = cnt < K ? cnt : K;
        for (int q = 0; q < cnt; ++q)
            if (freq_ahead(P, j, lp[q], lj[q])) { pos = q; break; }
        if (pos >= K) continue;
        for (int q = (cnt < K ? cnt : K - 1); q > pos; --q) { lp[q] = lp[q - 1]; lj[q] = lj[q - 1]; }
        lp[pos] = P;
        lj[pos] = j;
        if (cnt < K) ++cnt;
    }
    const double srmean = __ddiv_rn(sum_block(srsum, red), (double)nf);
    double srvar = 0.0;
    for (int j = threadIdx.x; j < nf; j += blockDim.x) {
        const double d = __dsub_rn((double)sqrtf(res[j]), srmean);
        srvar = __dadd_rn(srvar, __dmul_rn(d, d));
    }
    const double srsd = sqrt(__ddiv_rn(sum_block(srvar, red), (double)nf));
    int head = 0;
    for (int q = 0; q < K; ++q) {
        float bp = head < cnt ? lp[head] : -1.0f;
        int bj = head < cnt ? lj[head] : 0x7fffffff;
        int bt = threadIdx.x;
        for (int o = 16; o > 0; o >>= 1) {
            const float op = __shfl_xor_sync(0xffffffffu, bp, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
            if (freq_ahead(op, oj, bp, bj)) { bp = op; bj = oj; bt = ot; }
        }
        if (lane == 0) { sP[warp] = bp; sJ[warp] = bj; sT[warp] = bt; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (freq_ahead(sP[w], sJ[w], sP[0], sJ[0])) { sP[0] = sP[w]; sJ[0] = sJ[w]; sT[0] = sT[w]; }
            sel[q] = sP[0] >= 0.0f ? sJ[0] : -1;
            sT[0] = sP[0] >= 0.0f ? sT[0] : -1;
        }
        __syncthreads();
        if (sT[0] == (int)threadIdx.x) ++head;
        __syncthreads();
    }
    int M = 1;
    while (M < cd.n) M <<= 1;
    const long long o = cd.res - p.res_base;
    for (int q = 0; q < K; ++q) {
        DevPeak* out = &p.peaks[(size_t)blockIdx.x * K + q];
        const int j = sel[q];
        if (j < 0) {
            if (threadIdx.x == 0) { DevPeak z = {}; z.j = -1; *out = z; }
            continue;
        }
        const double f = cd.freqs ? cd.freqs[j] : __dadd_rn(cd.fmin, __dmul_rn((double)j, cd.df));
        sorted_keys(cd, fixed_freq(f, cd.dtmax), keys, M);
        if (threadIdx.x == 0) {
            const int2 run = p.runs[o + j];
            const int a = run.x, len = run.y;
            DevPeak pk = {};
            pk.j = j; pk.i1 = a; pk.k = len;
            pk.freq = f;
            pk.period = 1.0 / f;
            if (len > 0) {
                double r = 0.0, s = 0.0;
                for (int l = 0; l < len; ++l) {
                    int qq = a + l;
                    if (qq >= cd.n) qq -= cd.n;
                    const int i = (int)(keys[qq] & 0xffffffffu);
                    double inv = 1.0;
                    if (cd.dy) { const double dd = (double)cd.dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
                    const double w = __ddiv_rn(inv, cd.W);
                    r = __dadd_rn(r, w);
                    s = __dadd_rn(s, __dmul_rn(w, __dsub_rn((double)cd.y[i], cd.ybar)));
                }
                int ql = a + len - 1;
                if (ql >= cd.n) ql -= cd.n;
                const unsigned k0 = (unsigned)(keys[a] >> 32);
                const unsigned E = (unsigned)(keys[ql] >> 32) - k0;
                double mid = ((double)k0 + 0.5 * (double)E) / 4294967296.0;
                mid = mid - floor(mid);
                pk.epoch = cd.t_ref + mid / f;
                pk.duration = (double)E / 4294967296.0 / f;
                if (r > 0.0 && r < 1.0 && (p.sign || s < 0.0)) {
                    pk.power = s * s / (r * (1.0 - r));
                    pk.depth = -s / (r * (1.0 - r));
                    pk.sr = sqrt(pk.power);
                    pk.snr = pk.sr * sqrt(cd.W);
                }
            }
            pk.sde = srsd > 0.0 ? (pk.sr - srmean) / srsd : 0.0;
            *out = pk;
        }
        __syncthreads();
    }
}

}  // namespace

size_t ubls_smem_bytes(int nmax)
{
    int M = 1;
    while (M < nmax) M <<= 1;
    return (size_t)M * sizeof(unsigned long long) + (size_t)(nmax + 1) * sizeof(float4);
}

int ubls_tile() { return kTile; }

cudaError_t launch_ubls(const UblsParams& p, long long nitems, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    const size_t smem = ubls_smem_bytes(p.nmax);
    cudaError_t e = cudaFuncSetAttribute(ubls_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ubls_kernel<<<(unsigned)nitems, kUThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_ubls_reduce(const UblsParams& p, cudaStream_t s)
{
    if (p.ncurves <= 0) return cudaSuccess;
    int M = 1;
    while (M < p.nmax) M <<= 1;
    const size_t smem = (size_t)M * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(ubls_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ubls_reduce_kernel<<<p.ncurves, kUThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace blsgpu

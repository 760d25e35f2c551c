// bls_unbinned.cu -- unbinned (edge-to-edge) BLS: the box edges sit on data points.
//
// At every trial frequency the points are ordered by phase and every cyclic run of
// consecutive points whose phase extent lies in [qmin, qmax] is a box, scored with the
// binned search's statistic (r = sum w, s = sum w x over the run, P = s^2/(r(1-r)), dips
// only by default).  A point's phase is the binned search's FP64 fold, phi = p - floor(p)
// with p = RN(dt f); the order is (phi, point index); a run's extent is RN(phi_last -
// phi_first), plus one cycle (RN(d + 1)) when the run wraps through phase 0.
//
// Keys.  The sort works on 64-bit keys (K << 32 | point) with K = floor(phi 2^32), taken
// from the bits of p with integer operations (phi = frac(p) is exact, so K is exact); the
// FP64 product p is the only floating-point operation per point.  Points with equal K are
// then put in (phi, point) order by one thread per run of equal keys (rare: phases closer
// than 2^-32 cycle), which makes the order the definition's exactly.  Extents come from the
// keys: E64 = K_last - K_first (+ 2^32 past the end) is within 1 + 2^-20 of the definition's
// extent times 2^32 (K truncates by less than one unit; the extent's FP64 roundings add at
// most 2^-52 cycle), so a bound qmin or qmax is decided from E64 when it lies two or more
// units away, and otherwise from the phases in FP64, as the definition computes it.
//
// Search kernel: one block per (curve, tile of kTile frequencies).  For each frequency the
// block forms the keys in shared memory, sorts them (buckets on the top bits of the phase
// with an insertion sort per bucket; a bitonic network when phases clump), fixes the order
// of equal keys, and builds prefix sums of (w, w x) in phase order (FP64, stored as
// double-float pairs in four arrays).  Run starts are dealt round-robin to the threads; a
// start's admissible ends (extent within [qmin, qmax]) come from two binary searches, and
// every run's sums are independent prefix differences.  Runs are ranked by the signed
// residue z = s / sqrt(r(1-r)) (P = z^2), evaluated four ends at a time as two packed FP32
// pairs where every run of the curve is known to have 0 < r < 1; only the best z of each
// frequency is kept, P(f_j) = z^2.
//
// Reduce kernel: one block per curve: the top-k local maxima of P(f_j) (as in the binned
// search), the signal detection efficiency, and for each kept frequency the best run found
// again with the search's arithmetic (ties to the smaller start, then the shorter run) and
// refitted in FP64 -- order recomputed exactly, r and s summed in run order.
#include <cfloat>

#include "bls_internal.h"

namespace blsgpu {
namespace {

constexpr int kUThreads = 512;
constexpr int kTile = 16;

typedef unsigned long long u64;

// The FP64 phase of point i at frequency f, as the definition folds it.
__device__ __forceinline__ double point_phase(const CurveDesc& cd, int i, double f)
{
    const double p = __dmul_rn(cd.dt64[i], f);
    return __dsub_rn(p, floor(p));
}

// K = floor(frac(p) 2^32) of a finite non-negative p, from its bits with integer
// operations: p = m 2^(e-52) with the 53-bit significand m, so p 2^32 = m 2^(e-20) and K is
// that value's integer part modulo 2^32 (a shift of m either way; zero for p < 2^-1022 and
// for p >= 2^84, whose fraction is zero).
__device__ __forceinline__ unsigned key32(double p)
{
    const u64 b = (u64)__double_as_longlong(p);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0u;
    const u64 m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 1043 - ex;            // 20 - (ex - 1023)
    if (sh >= 64 || sh <= -64) return 0u;
    return sh >= 0 ? (unsigned)(m >> sh) : (unsigned)(m << (-sh));
}

// Sort key (K << 32 | point) of point i at frequency f.
__device__ __forceinline__ u64 phase_key(const CurveDesc& cd, int i, double f)
{
    return ((u64)key32(__dmul_rn(cd.dt64[i], f)) << 32) | (unsigned)i;
}

// Phase keys of a curve at f, bitonic-sorted ascending in `keys` (M = the power of two
// >= n; the tail holds all-ones sentinels).
__device__ __forceinline__ void sorted_keys(const CurveDesc& cd, double f, u64* keys, int M)
{
    const int n = cd.n;
    for (int i = threadIdx.x; i < M; i += blockDim.x) keys[i] = i < n ? phase_key(cd, i, f) : ~0ull;
    __syncthreads();
    for (int size = 2; size <= M; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (M >> 1); t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const u64 a = keys[lo], b = keys[hi];
                if ((a > b) == up) { keys[lo] = b; keys[hi] = a; }
            }
            __syncthreads();
        }
    }
}

// Runs of equal K in keys[0 .. n) (sorted by (K, point)) reordered by (phi, point): one
// thread per run, an insertion sort on the FP64 phases (a run already in phase order --
// equal phases -- costs one comparison per point).
__device__ __forceinline__ void order_equal_keys(const CurveDesc& cd, double f, u64* keys, int n)
{
    for (int q = threadIdx.x; q + 1 < n; q += blockDim.x) {
        const unsigned K = (unsigned)(keys[q] >> 32);
        if ((unsigned)(keys[q + 1] >> 32) != K || (q > 0 && (unsigned)(keys[q - 1] >> 32) == K)) continue;
        int q1 = q + 2;
        while (q1 < n && (unsigned)(keys[q1] >> 32) == K) ++q1;
        for (int x = q + 1; x < q1; ++x) {
            const u64 v = keys[x];
            const int iv = (int)(v & 0xffffffffu);
            const double pv = point_phase(cd, iv, f);
            int y = x - 1;
            while (y >= q) {
                const int iy = (int)(keys[y] & 0xffffffffu);
                const double py = point_phase(cd, iy, f);
                if (py < pv || (py == pv && iy < iv)) break;
                keys[y + 1] = keys[y];
                --y;
            }
            keys[y + 1] = v;
        }
    }
    __syncthreads();
}

constexpr int kBucketMax = 48;   // largest bucket left to an insertion sort

// Points of a curve at f in the definition's (phi, point) order in keys[0 .. n): keys
// (K, point) sorted by a counting pass over the top B bits of K into nbk = M/2 buckets
// (shared-memory atomics), an exclusive scan, a scatter, and an insertion sort of every
// bucket by one thread -- or, when a bucket holds more than kBucketMax keys (phases
// clumped), by the bitonic network; the keys are distinct, so both give the same order --
// then equal K put in phase order.  `cnt` is scratch for M + 1 ints.
__device__ __forceinline__ void sort_keys(const CurveDesc& cd, double f, u64* keys, int M, int* cnt,
                                          int* err)
{
    __shared__ int s_tot[kUThreads / 32 + 1];
    const int n = cd.n, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nbk = M >= 2 ? M >> 1 : 1;
    int B = 0;
    while ((1 << B) < nbk) ++B;
    int* start = cnt;              // nbk + 1
    int* cur = cnt + nbk + 1;      // nbk (after the scan)
    for (int b = tid; b < nbk; b += nt) start[b] = 0;
    if (tid == 0) s_tot[kUThreads / 32] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        const u64 k = phase_key(cd, i, f);
        atomicAdd(&start[B ? (int)(k >> (64 - B)) : 0], 1);
    }
    __syncthreads();
    // exclusive scan of the bucket counts (contiguous runs per thread, then warp and block
    // scans of the run totals) and the largest count
    const int per = (nbk + nt - 1) / nt;
    const int b0 = min(nbk, tid * per), b1 = min(nbk, b0 + per);
    int tot = 0, mx = 0;
    for (int b = b0; b < b1; ++b) { tot += start[b]; mx = max(mx, start[b]); }
    int inc = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 31) s_tot[warp] = inc;
    if (lane == 0) atomicMax(&s_tot[kUThreads / 32], mx);
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += s_tot[w];
    const bool clumped = s_tot[kUThreads / 32] > kBucketMax;
    {
        int run = wbase + inc - tot;
        for (int b = b0; b < b1; ++b) {
            const int c = start[b];
            start[b] = run;
            cur[b] = run;
            run += c;
        }
    }
    __syncthreads();
    if (clumped) {
        sorted_keys(cd, f, keys, M);
        order_equal_keys(cd, f, keys, n);
        return;
    }
    if (tid == 0) start[nbk] = n;
    for (int i = tid; i < n; i += nt) {
        const u64 k = phase_key(cd, i, f);
        const int at = atomicAdd(&cur[B ? (int)(k >> (64 - B)) : 0], 1);
        if (bls_ok(at < n, err)) keys[at] = k;
    }
    __syncthreads();
    for (int b = tid; b < nbk; b += nt) {
        const int s0 = start[b], s1 = start[b + 1];
        for (int x = s0 + 1; x < s1; ++x) {
            const u64 v = keys[x];
            int y = x - 1;
            while (y >= s0 && keys[y] > v) { keys[y + 1] = keys[y]; --y; }
            keys[y + 1] = v;
        }
    }
    __syncthreads();
    order_equal_keys(cd, f, keys, n);
}

__device__ __forceinline__ void point_weights(const CurveDesc& cd, int i, float& w, float& wx)
{
    const float4 B = cd.pts[(i >> 1) * 2 + 1];
    w = (i & 1) ? B.z : B.x;
    wx = (i & 1) ? B.w : B.y;
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
    hi = __fadd_rn(a, b);
    const float bb = __fsub_rn(hi, a);
    lo = __fadd_rn(__fsub_rn(a, __fsub_rn(hi, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float rsqrt_apx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Prefix sums of (w, w x) in phase order, C[q] = sums over sorted positions < q (q = 0..n),
// as double-float pairs in four arrays (w hi, w lo, wx hi, wx lo).  FP64 over each thread's
// positions, a scan of the thread totals (warp shuffles, then the warp totals in order);
// the chunking depends only on n and the block size, so every kernel that calls this with
// the same block size gets the same values.
struct Prefix {
    float *wh, *wl, *xh, *xl;
};

__device__ __forceinline__ void prefix_sums(const CurveDesc& cd, const u64* keys, const Prefix& C,
                            double* sred)
{
    const int n = cd.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = blockDim.x;
    const int ch = (n + nt - 1) / nt;
    const int q0 = min(n, (int)threadIdx.x * ch), q1 = min(n, q0 + ch);
    double tw = 0.0, tx = 0.0;
    for (int q = q0; q < q1; ++q) {
        float w, wx;
        point_weights(cd, (int)(keys[q] & 0xffffffffu), w, wx);
        tw = __dadd_rn(tw, (double)w);
        tx = __dadd_rn(tx, (double)wx);
    }
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
        C.wh[n] = W.x; C.wl[n] = W.y; C.xh[n] = X.x; C.xl[n] = X.y;
    }
    __syncthreads();
    double aw = __dsub_rn(__dadd_rn(sred[warp], iw), tw);
    double ax = __dsub_rn(__dadd_rn(sred[nt + warp], ix), tx);
    for (int q = q0; q < q1; ++q) {
        const float2 W = split_df(aw), X = split_df(ax);
        C.wh[q] = W.x; C.wl[q] = W.y; C.xh[q] = X.x; C.xl[q] = X.y;
        float w, wx;
        point_weights(cd, (int)(keys[q] & 0xffffffffu), w, wx);
        aw = __dadd_rn(aw, (double)w);
        ax = __dadd_rn(ax, (double)wx);
    }
    __syncthreads();
}

// The definition's bounds of a run's extent and the frequency (for the exact re-check).
struct Bounds {
    double qmin, qmax;    // extent bounds, in cycles
    double lo, hi;        // the same in units of 2^-32 cycle (exact scalings)
    double f;
};

__device__ __forceinline__ Bounds make_bounds(double qmin, double qmax, double f)
{
    Bounds B;
    B.qmin = qmin;
    B.qmax = qmax;
    B.lo = qmin * 4294967296.0;
    B.hi = qmax * 4294967296.0;
    B.f = f;
    return B;
}

// The definition's extent of the run from sorted position a to unwrapped position e.
__device__ __forceinline__ double exact_extent(const CurveDesc& cd, const u64* keys, int n, int a, int e,
                                               double f)
{
    const double pa = point_phase(cd, (int)(keys[a] & 0xffffffffu), f);
    const double pe = point_phase(cd, (int)(keys[e < n ? e : e - n] & 0xffffffffu), f);
    const double d = __dsub_rn(pe, pa);
    return e >= n ? __dadd_rn(d, 1.0) : d;
}

// Admissible ends of the runs starting at sorted position a: unwrapped positions
// emin..emax (extents within [qmin, qmax], at most n - 1 points), extents growing with the
// end; emin > emax when none.  Each bound is decided from the keys' extent E64 when it lies
// two or more units of 2^-32 away, else from the FP64 phases.
__device__ __forceinline__ void run_ends(const CurveDesc& cd, const u64* keys, int n, int a,
                                         const Bounds& B, int& emin, int& emax)
{
    const long long k0 = (long long)(keys[a] >> 32);
    auto e64 = [&](int e) {
        return (double)((long long)(keys[e < n ? e : e - n] >> 32) - k0 + (e >= n ? (1ll << 32) : 0ll));
    };
    auto le_max = [&](int e) {
        const double x = e64(e);
        if (x + 2.0 <= B.hi) return true;
        if (x - 2.0 >= B.hi) return false;
        return exact_extent(cd, keys, n, a, e, B.f) <= B.qmax;
    };
    auto ge_min = [&](int e) {
        const double x = e64(e);
        if (x - 2.0 >= B.lo) return true;
        if (x + 2.0 <= B.lo) return false;
        return exact_extent(cd, keys, n, a, e, B.f) >= B.qmin;
    };
    int lo2 = a, hi2 = a + n - 1;            // extent(lo2) = 0 <= qmax; hi2 out of range
    while (hi2 - lo2 > 1) {
        const int mid = (lo2 + hi2) >> 1;
        if (le_max(mid)) lo2 = mid; else hi2 = mid;
    }
    emax = lo2;
    int lo1 = a - 1, hi1 = emax + 1;          // extent(hi1) >= qmin or hi1 past emax
    while (hi1 - lo1 > 1) {
        const int mid = (lo1 + hi1) >> 1;
        if (ge_min(mid)) hi1 = mid; else lo1 = mid;
    }
    emin = hi1;
}

// Signed residue of a run with -r = nr and s = s: z = s / sqrt(r (1 - r)), from one fused
// -d = r^2 - r and an approximate reciprocal square root (P = z^2).  Runs with d <= 0 (r
// outside (0, 1) in FP32) give NaN, or +-inf for d = 0; the search ranks runs by z.
__device__ __forceinline__ float run_z(float nr, float s)
{
    return __fmul_rn(s, rsqrt_apx(-__fmaf_rn(nr, nr, nr)));
}

// -r and s of the run (a, e] inside [0, n): prefix differences of double-float pairs.
__device__ __forceinline__ void run_in(const Prefix& C, float awh, float awl, float axh, float axl,
                                       int u, float& nr, float& s)
{
    nr = __fadd_rn(__fsub_rn(awh, C.wh[u]), __fsub_rn(awl, C.wl[u]));
    s = __fadd_rn(__fsub_rn(C.xh[u], axh), __fsub_rn(C.xl[u], axl));
}

// -r and s of a run that wraps past the end: totals T plus the prefix at u, through an
// error-free sum of the leading terms.
__device__ __forceinline__ void run_wrap(const Prefix& C, float4 T, float awh, float awl, float axh,
                                         float axl, int u, float& nr, float& s)
{
    float wh, wl, xh, xl;
    two_sum(T.x, C.wh[u], wh, wl);
    two_sum(T.z, C.xh[u], xh, xl);
    nr = __fadd_rn(__fsub_rn(awh, wh), __fsub_rn(awl, __fadd_rn(__fadd_rn(wl, T.y), C.wl[u])));
    s = __fadd_rn(__fsub_rn(xh, axh), __fsub_rn(__fadd_rn(__fadd_rn(xl, T.w), C.xl[u]), axl));
}

// Best (most negative for dips, largest |z| for both signs) of an accumulator and z.
template <int SIGN>
__device__ __forceinline__ float best_z(float b, float z)
{
    return SIGN ? fmaxf(b, fabsf(z)) : fminf(b, z);
}

__device__ __forceinline__ u64 pk2(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(u64 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b)
{
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float fmin3f(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fmax3f(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// b updated with one run (-r = nr, s); without FAST, runs with d <= 0 do not count.
template <int SIGN, bool FAST>
__device__ __forceinline__ float scored(float b, float nr, float s)
{
    const float z = run_z(nr, s);
    return (FAST || -__fmaf_rn(nr, nr, nr) > 0.0f) ? best_z<SIGN>(b, z) : b;
}

// The best z over the runs of start a (the search: no positions kept).  FAST: every run has
// d > 0 (see the caller), so the ends inside [0, n) go two at a time as packed pairs (the
// prefix arrays read 8 bytes at an even position), with the same per-lane arithmetic as
// run_in / run_z; otherwise every run is scored alone and runs with d <= 0 are skipped.
template <int SIGN, bool FAST>
__device__ __forceinline__ float start_best(const Prefix& C, float4 T, int n, int a, int emin,
                                            int emax, float b)
{
    const float awh = C.wh[a], awl = C.wl[a], axh = C.xh[a], axl = C.xl[a];
    // ends e in [emin, min(emax, n-1)]: prefix index u = e + 1 in [u0, u1]
    int u = emin + 1;
    const int u1 = min(emax, n - 1) + 1;
    if (FAST) {
        if ((u & 1) && u <= u1) {
            float nr, s;
            run_in(C, awh, awl, axh, axl, u, nr, s);
            b = scored<SIGN, FAST>(b, nr, s);
            ++u;
        }
        const u64 AWH = pk2(awh, awh), AWL = pk2(awl, awl), AXH = pk2(axh, axh), AXL = pk2(axl, axl);
        const u64* WH = reinterpret_cast<const u64*>(C.wh);
        const u64* WL = reinterpret_cast<const u64*>(C.wl);
        const u64* XH = reinterpret_cast<const u64*>(C.xh);
        const u64* XL = reinterpret_cast<const u64*>(C.xl);
        if ((u & 2) && u + 1 <= u1) {   // to a multiple of four
            const int h = u >> 1;
            const u64 NR = add2(sub2(AWH, WH[h]), sub2(AWL, WL[h]));
            const u64 S = add2(sub2(XH[h], AXH), sub2(XL[h], AXL));
            float nd0, nd1;
            upk2(fma2(NR, NR, NR), nd0, nd1);
            float z0, z1;
            upk2(mul2(S, pk2(rsqrt_apx(-nd0), rsqrt_apx(-nd1))), z0, z1);
            b = SIGN ? fmax3f(b, fabsf(z0), fabsf(z1)) : fmin3f(b, z0, z1);
            u += 2;
        }
        // four ends at a time: one 16-byte read of each prefix array (arrays 16-byte aligned,
        // see prefix_layout), two packed pairs, the same per-lane arithmetic
        const ulonglong2* WH4 = reinterpret_cast<const ulonglong2*>(C.wh);
        const ulonglong2* WL4 = reinterpret_cast<const ulonglong2*>(C.wl);
        const ulonglong2* XH4 = reinterpret_cast<const ulonglong2*>(C.xh);
        const ulonglong2* XL4 = reinterpret_cast<const ulonglong2*>(C.xl);
#pragma unroll 2
        for (; u + 3 <= u1; u += 4) {
            const int h = u >> 2;
            const ulonglong2 wh = WH4[h], wl = WL4[h], xh = XH4[h], xl = XL4[h];
            const u64 NR0 = add2(sub2(AWH, wh.x), sub2(AWL, wl.x));
            const u64 NR1 = add2(sub2(AWH, wh.y), sub2(AWL, wl.y));
            const u64 S0 = add2(sub2(xh.x, AXH), sub2(xl.x, AXL));
            const u64 S1 = add2(sub2(xh.y, AXH), sub2(xl.y, AXL));
            float nd0, nd1, nd2, nd3;
            upk2(fma2(NR0, NR0, NR0), nd0, nd1);
            upk2(fma2(NR1, NR1, NR1), nd2, nd3);
            float z0, z1, z2, z3;
            upk2(mul2(S0, pk2(rsqrt_apx(-nd0), rsqrt_apx(-nd1))), z0, z1);
            upk2(mul2(S1, pk2(rsqrt_apx(-nd2), rsqrt_apx(-nd3))), z2, z3);
            b = SIGN ? fmax3f(b, fabsf(z0), fabsf(z1)) : fmin3f(b, z0, z1);
            b = SIGN ? fmax3f(b, fabsf(z2), fabsf(z3)) : fmin3f(b, z2, z3);
        }
        for (; u + 1 <= u1; u += 2) {
            const int h = u >> 1;
            const u64 NR = add2(sub2(AWH, WH[h]), sub2(AWL, WL[h]));
            const u64 S = add2(sub2(XH[h], AXH), sub2(XL[h], AXL));
            float nd0, nd1;
            upk2(fma2(NR, NR, NR), nd0, nd1);
            float z0, z1;
            upk2(mul2(S, pk2(rsqrt_apx(-nd0), rsqrt_apx(-nd1))), z0, z1);
            b = SIGN ? fmax3f(b, fabsf(z0), fabsf(z1)) : fmin3f(b, z0, z1);
        }
    }
    for (; u <= u1; ++u) {
        float nr, s;
        run_in(C, awh, awl, axh, axl, u, nr, s);
        b = scored<SIGN, FAST>(b, nr, s);
    }
    // ends past n - 1: prefix index e + 1 - n
    for (int e = max(emin, n); e <= emax; ++e) {
        float nr, s;
        run_wrap(C, T, awh, awl, axh, axl, e + 1 - n, nr, s);
        b = scored<SIGN, FAST>(b, nr, s);
    }
    return b;
}

// Shared-memory layout of both kernels: keys [M] (8 B, M >= 2), then the four prefix arrays
// of n1 = n + 1 rounded up to a multiple of four entries each (so that 16-byte reads of four
// entries stay aligned).
__device__ __forceinline__ Prefix prefix_layout(unsigned char* dsm, int M, int n)
{
    const int n1 = (n + 4) & ~3;
    float* base = reinterpret_cast<float*>(dsm + (size_t)M * sizeof(unsigned long long));
    Prefix C;
    C.wh = base;
    C.wl = base + n1;
    C.xh = base + 2 * n1;
    C.xl = base + 3 * n1;
    return C;
}

// Whether every run of the curve has d = r (1 - r) > 0 in FP32: the lightest point holds
// at least 2^-23 of the weight, so a run of at most n - 1 points has r <= 1 - 2^-23 (up to
// the rounding of r, below 2^-24), and r > 0 since weights are positive.
__device__ __forceinline__ bool runs_positive(const CurveDesc& cd, float* red)
{
    float m = FLT_MAX;
    for (int i = threadIdx.x; i < cd.n; i += blockDim.x) {
        float w, wx;
        point_weights(cd, i, w, wx);
        m = fminf(m, w);
    }
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = FLT_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fminf(m, red[w]);
    __syncthreads();
    return m >= 1.1920929e-7f;   // 2^-23
}

// Working arrays of a block (keys, prefix sums): its dynamic shared memory, or, for curves
// too long for it, the block's own slice of a global scratch buffer (persistent blocks, so
// the scratch is bounded by the grid, not by the number of work items).
__device__ __forceinline__ unsigned char* ubls_work(const UblsParams& p, unsigned char* dsm)
{
    return p.scratch ? p.scratch + (size_t)blockIdx.x * p.scratch_stride : dsm;
}

// One work item (curve, tile of kTile frequencies) of the search.
template <int SIGN>
__device__ __forceinline__ void ubls_item(const UblsParams& p, long long it, unsigned char* work,
                                          u64* keys, float* sZ, double* sred)
{
    // work item -> (curve, tile)
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
    const Prefix C = prefix_layout(work, M, n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = blockDim.x;
    const bool fast = runs_positive(cd, reinterpret_cast<float*>(sred));
    for (int j = j0; j < min(j0 + kTile, cd.nf); ++j) {
        const double f = cd.freqs ? cd.freqs[j] : __dadd_rn(cd.fmin, __dmul_rn((double)j, cd.df));
        sort_keys(cd, f, keys, M, reinterpret_cast<int*>(C.wh), p.err);
        prefix_sums(cd, keys, C, sred);
        const Bounds Bq = make_bounds(p.qmin, p.qmax, f);
        const float4 T = make_float4(C.wh[n], C.wl[n], C.xh[n], C.xl[n]);
        // starts dealt round-robin to the threads (phases clump, so contiguous ranges would
        // load the threads unevenly); each start's best z over its admissible runs
        float b = 0.0f;
        for (int a = threadIdx.x; a < n; a += nt) {
            int emin, emax;
            run_ends(cd, keys, n, a, Bq, emin, emax);
            if (!bls_ok(emin >= a && emax <= a + n - 2, p.err)) continue;
            b = fast ? start_best<SIGN, true>(C, T, n, a, emin, emax, b)
                     : start_best<SIGN, false>(C, T, n, a, emin, emax, b);
        }
        for (int o = 16; o > 0; o >>= 1) b = best_z<SIGN>(b, __shfl_xor_sync(0xffffffffu, b, o));
        if (lane == 0) sZ[warp] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            float z = sZ[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) z = best_z<SIGN>(z, sZ[w]);
            cd.res[j] = __fmul_rn(z, z);
        }
        __syncthreads();
    }
}

// The search of a block: its work items (curve, tile), one after another.
template <int SIGN>
__device__ __forceinline__ void ubls_search(const UblsParams& p)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ float sZ[kUThreads / 32];
    __shared__ double sred[2 * kUThreads];
    unsigned char* const work = ubls_work(p, dsm);
    u64* keys = reinterpret_cast<u64*>(work);
    for (long long it = blockIdx.x; it < p.nitems; it += gridDim.x)
        ubls_item<SIGN>(p, it, work, keys, sZ, sred);
}

// Search kernel: blocks take (curve, tile of kTile frequencies) items (one each with the
// working arrays in shared memory; persistent with the global scratch); P(f_j) = z^2 of the
// best run (its position is found again by the reduce kernel for the kept frequencies only).
__global__ void __launch_bounds__(kUThreads, 1) ubls_kernel(UblsParams p)
{
    if (p.sign) ubls_search<1>(p);
    else ubls_search<0>(p);
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

// (z, start, len) order of the best run: the more extreme z (P = z^2; dips: the most
// negative), then the smaller start, then the shorter run.
template <int SIGN>
__device__ __forceinline__ bool run_first(float za, int sa, int la, float zb, int sb, int lb)
{
    const bool more = SIGN ? fabsf(za) > fabsf(zb) : za < zb;
    const bool same = SIGN ? fabsf(za) == fabsf(zb) : za == zb;
    return more || (same && (sa < sb || (sa == sb && la < lb)));
}

// The best run of one frequency (keys and prefix sums in place), with the search kernel's
// arithmetic, so its z is the one the search kept; (start, len), len = 0 if no run counts.
template <int SIGN>
__device__ int2 best_run(const CurveDesc& cd, const u64* keys, const Prefix& C, int n, const Bounds& Bq,
                         bool fast, float* sz, int* ss, int* sl)
{
    const float4 T = make_float4(C.wh[n], C.wl[n], C.xh[n], C.xl[n]);
    float bz = 0.0f;
    int bs = 0x7fffffff, bl = 0x7fffffff;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        int emin, emax;
        run_ends(cd, keys, n, a, Bq, emin, emax);
        const float awh = C.wh[a], awl = C.wl[a], axh = C.xh[a], axl = C.xl[a];
        for (int e = emin; e <= emax; ++e) {
            float nr, sx;
            if (e < n) run_in(C, awh, awl, axh, axl, e + 1, nr, sx);
            else run_wrap(C, T, awh, awl, axh, axl, e + 1 - n, nr, sx);
            if (!fast && !(-__fmaf_rn(nr, nr, nr) > 0.0f)) continue;
            const float z = run_z(nr, sx);
            if ((SIGN ? fabsf(z) > 0.0f : z < 0.0f) && run_first<SIGN>(z, a, e - a + 1, bz, bs, bl)) {
                bz = z; bs = a; bl = e - a + 1;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float oz = __shfl_xor_sync(0xffffffffu, bz, o);
        const int os = __shfl_xor_sync(0xffffffffu, bs, o);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
        if (run_first<SIGN>(oz, os, ol, bz, bs, bl)) { bz = oz; bs = os; bl = ol; }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sz[warp] = bz; ss[warp] = bs; sl[warp] = bl; }
    __syncthreads();
    bz = sz[0]; bs = ss[0]; bl = sl[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (run_first<SIGN>(sz[w], ss[w], sl[w], bz, bs, bl)) { bz = sz[w]; bs = ss[w]; bl = sl[w]; }
    __syncthreads();
    return bs == 0x7fffffff ? make_int2(0, 0) : make_int2(bs, bl);
}

__global__ void __launch_bounds__(kUThreads, 1) ubls_reduce_kernel(UblsParams p)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    unsigned char* const work = ubls_work(p, dsm);
    u64* keys = reinterpret_cast<u64*>(work);
    __shared__ double red[2 * kUThreads];
    __shared__ float bzs[kUThreads / 32];
    __shared__ int bss[kUThreads / 32], bls[kUThreads / 32];
    __shared__ float sP[kUThreads / 32];
    __shared__ int sJ[kUThreads / 32], sT[kUThreads / 32];
    __shared__ int sel[kMaxTopK];
    // one curve after another (one per block with the working arrays in shared memory)
    for (int c = blockIdx.x; c < p.ncurves; c += gridDim.x) {
        const CurveDesc& cd = p.curves[c];
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
        const Prefix C = prefix_layout(work, M, cd.n);
        const bool fast = runs_positive(cd, reinterpret_cast<float*>(red));
        for (int q = 0; q < K; ++q) {
            DevPeak* out = &p.peaks[(size_t)c * K + q];
            const int j = sel[q];
            if (j < 0) {
                if (threadIdx.x == 0) { DevPeak z = {}; z.j = -1; *out = z; }
                continue;
            }
            const double f = cd.freqs ? cd.freqs[j] : __dadd_rn(cd.fmin, __dmul_rn((double)j, cd.df));
            sort_keys(cd, f, keys, M, reinterpret_cast<int*>(C.wh), p.err);
            prefix_sums(cd, keys, C, red);
            const Bounds Bq = make_bounds(p.qmin, p.qmax, f);
            const int2 run = p.sign ? best_run<1>(cd, keys, C, cd.n, Bq, fast, bzs, bss, bls)
                                    : best_run<0>(cd, keys, C, cd.n, Bq, fast, bzs, bss, bls);
            if (threadIdx.x == 0) {
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
                    // extent and mid-box phase as the definition computes them
                    const double E = exact_extent(cd, keys, cd.n, a, a + len - 1, f);
                    const double ph0 = point_phase(cd, (int)(keys[a] & 0xffffffffu), f);
                    double mid = __dadd_rn(ph0, __dmul_rn(0.5, E));
                    mid = __dsub_rn(mid, floor(mid));
                    pk.epoch = __dadd_rn(cd.t_ref, __ddiv_rn(mid, f));
                    pk.duration = __ddiv_rn(E, f);
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
    __syncthreads();
    }
}

}  // namespace

size_t ubls_work_bytes(int nmax)
{
    int M = 1;
    while (M < nmax) M <<= 1;
    return (size_t)M * sizeof(unsigned long long) + (size_t)4 * ((nmax + 4) & ~3) * sizeof(float);
}

int ubls_tile() { return kTile; }

cudaError_t launch_ubls(const UblsParams& p, cudaStream_t s)
{
    if (p.nitems <= 0) return cudaSuccess;
    const size_t smem = p.scratch ? 0 : ubls_work_bytes(p.nmax);
    cudaError_t e = cudaFuncSetAttribute(ubls_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = p.scratch ? (p.grid < p.nitems ? p.grid : p.nitems) : p.nitems;
    ubls_kernel<<<(unsigned)grid, kUThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_ubls_reduce(const UblsParams& p, cudaStream_t s)
{
    if (p.ncurves <= 0) return cudaSuccess;
    const size_t smem = p.scratch ? 0 : ubls_work_bytes(p.nmax);
    cudaError_t e = cudaFuncSetAttribute(ubls_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = p.scratch ? (p.grid < p.ncurves ? p.grid : p.ncurves) : p.ncurves;
    ubls_reduce_kernel<<<grid, kUThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace blsgpu

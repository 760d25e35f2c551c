// bls_kernels.cu -- sm_103a kernels of the box-least-squares search (Sec. 2.2.2).
//
//  prep_kernel        one block per curve: weights, weighted mean, mean-subtracted flux,
//                     time offsets (FP64), stored as 16-byte points for the hot loop.
//  fold_sweep_kernel  persistent; one work item = (curve, tile of T frequencies); one
//                     thread per frequency with a private phase histogram in shared
//                     memory.  Loop A folds and bins every point, loop B sweeps every
//                     cyclic box and keeps the best per frequency.
//  reduce_kernel      one block per curve: top-k peaks over frequencies, FP64 refit of
//                     the chosen boxes, reported quantities.
//  plain_f64_kernel   baseline, one curve per launch, one thread per frequency, FP64
//                     histograms in global memory (the paper's decomposition).
//
// Fold semantics (identical to the FP64 definition): p = RN(dt*f), phase = p - floor(p),
// bin = floor(RN(phase*nb)) clamped to nb-1.  The default fast path evaluates dt*f as a
// double-FP32 product with a proven error bound and re-folds in FP64 only the points that
// lie within that bound of a bin edge, so every bin equals the FP64 one.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bls_internal.h"

namespace blsgpu {

// ------------------------------------------------------------------------- helpers

__device__ __forceinline__ double grid_freq(const CurveDesc& cd, int j)
{
    if (cd.freqs) return cd.freqs[j];
    return __dadd_rn(cd.fmin, __dmul_rn((double)j, cd.df));
}

// Exact fold in FP64, every operation rounded once (no contraction).
__device__ __forceinline__ int fold_exact(double dt, double f, int nb)
{
    double p = __dmul_rn(dt, f);
    double ph = __dsub_rn(p, floor(p));
    double u = __dmul_rn(ph, (double)nb);
    int b = (int)floor(u);
    b = b >= nb ? nb - 1 : b;
    return b < 0 ? 0 : b;
}

// Constants of the double-FP32 fold of one thread's frequency.
struct FoldConst {
    float fh, fl;     // f = fh + fl (+ |err| <= 2^-48 f)
    float nbf;        // nb as float
    float lim;        // 0.5 - tol: |d| beyond this means "near a bin edge"
    float f32;        // f rounded to FP32 (FP32 phase mode)
    double f;         // exact frequency
    int nb;
    bool fast;        // the double-FP32 path is valid for this (curve, frequency)
};

// Error bound of the double-FP32 fold, in bins.  With D = dt, F = f, DF = D*F and
// u = 2^-24 (FP32 unit roundoff):
//   split errors |D - dh - dl| <= u^2 D, |F - fh - fl| <= u^2 F, dropped dl*fl <= u^2 DF,
//   two-product exact, two FMA roundings of the cross terms <= 1.5 u^2 DF
//   => |ph + c - DF| <= 2^-44 DF cycles;
//   cn = RN(c nb - 1/2) and x = RN(fr nb + cn) add u|cn| + u|x|;
//   the FP64 definition itself is within nb 2^-53 (DF + 1) bins of nb*frac(DF).
// tol doubles the sum.  Valid while DF < 2^20 (then |c| < 3u DF < 0.19 cycles).
__device__ __forceinline__ FoldConst make_fold_const(double f, int nb, double dtmax)
{
    FoldConst fc;
    fc.f = f;
    fc.nb = nb;
    fc.fh = __double2float_rn(f);
    fc.fl = __double2float_rn(__dsub_rn(f, (double)fc.fh));
    fc.f32 = fc.fh;
    fc.nbf = (float)nb;
    double DF = dtmax * f;
    fc.fast = DF < 1048576.0;
    double cmax = 3.0 * 5.9604644775390625e-8 * DF;          // 3 u DF
    double cn = cmax * nb + 0.5;
    double xm = nb * (0.5 + cmax) + 0.5 + cn;
    double tol = 2.0 * (nb * DF * 5.684341886080802e-14       // 2^-44
                        + 5.9604644775390625e-8 * (cn + xm)    // u (|cn| + |x|)
                        + nb * 2.220446049250313e-16 * (DF + 1.0));  // 2^-52
    fc.lim = __double2float_rd(0.5 - tol);
    return fc;
}

// Double-FP32 fold.  Returns the bin and sets `edge` when the bin is not certain.
__device__ __forceinline__ int fold_df32(float dh, float dl, const FoldConst& fc, bool& edge)
{
    const float M = 12582912.0f;                 // 1.5 * 2^23: RN(x + M) - M = rint(x)
    float ph = __fmul_rn(dh, fc.fh);
    float e = __fmaf_rn(dh, fc.fh, -ph);         // exact product error
    float t1 = __fmaf_rn(dh, fc.fl, e);
    float c = __fmaf_rn(dl, fc.fh, t1);          // dt*f ~= ph + c
    float m = __fadd_rn(ph, M);
    float rp = __fsub_rn(m, M);
    float fr = __fsub_rn(ph, rp);                // exact, in [-1/2, 1/2]
    float cn = __fmaf_rn(c, fc.nbf, -0.5f);
    float x = __fmaf_rn(fr, fc.nbf, cn);         // nb * (phase mod 1, centred) - 1/2
    float m2 = __fadd_rn(x, M);
    float rx = __fsub_rn(m2, M);
    float d = __fsub_rn(x, rx);                  // exact, in [-1/2, 1/2]
    int ri = __float_as_int(m2) - __float_as_int(M);   // rint(x) = floor(x + 1/2)
    unsigned b0 = (unsigned)ri, b1 = (unsigned)(ri + fc.nb);
    edge = !(fabsf(d) <= fc.lim);                // NaN (bad input) also takes the exact path
    return (int)min(min(b0, b1), (unsigned)(fc.nb - 1));
}

// FP32 fold (precision study): no error bound, no fallback.
__device__ __forceinline__ int fold_f32(float dt32, const FoldConst& fc)
{
    float p = __fmul_rn(dt32, fc.f32);
    float ph = __fsub_rn(p, floorf(p));
    int b = (int)floorf(__fmul_rn(ph, fc.nbf));
    b = b >= fc.nb ? fc.nb - 1 : b;
    return b < 0 ? 0 : b;
}

template <int PHASE>
__device__ __forceinline__ int fold_point(const float4& q, const double* dtp,
                                          const FoldConst& fc)
{
    if (PHASE == kPhaseF64 || !fc.fast) return fold_exact(*dtp, fc.f, fc.nb);
    if (PHASE == kPhaseF32) return fold_f32(__fadd_rn(q.x, q.y), fc);
    bool edge;
    int b = fold_df32(q.x, q.y, fc, edge);
    if (edge) b = fold_exact(*dtp, fc.f, fc.nb);
    return b;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Deterministic block sum of FP64 (fixed tree, blockDim.x a power of two <= 1024).
__device__ double block_sum(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

__device__ double block_min(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

__device__ double block_max(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------------- a1: prep

constexpr int kPrepThreads = 256;

// Weights w = dy^-2/W, mean ybar = y0 + sum w (y - y0) (constant flux gives exact zeros),
// x = y - ybar, dt = t - min t; points stored as (dt_hi, dt_lo, w, w x) in FP32 and dt
// in FP64.  Validates the inputs (finite t and y, finite dy > 0, frequencies > 0).
__global__ void __launch_bounds__(kPrepThreads) prep_kernel(CurveDesc* curves, const int* slots,
                                                             int* err)
{
    __shared__ double red[kPrepThreads];
    CurveDesc* cd = &curves[slots ? slots[blockIdx.x] : (int)blockIdx.x];
    const int n = cd->n;
    const double* t = cd->t;
    const float* y = cd->y;
    const float* dy = cd->dy;
    float4* pts = cd->pts;
    double* dt64 = cd->dt64;
    bool bad = false;
    double tmin = INFINITY, tmax = -INFINITY, W = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double ti = t[i];
        float yi = y[i];
        if (!isfinite(ti) || !isfinite(yi)) bad = true;
        double inv = 1.0;
        if (dy) {
            float d = dy[i];
            if (!(d > 0.0f) || !isfinite(d)) bad = true;
            double dd = (double)d;
            inv = __ddiv_rn(1.0, __dmul_rn(dd, dd));
        }
        tmin = fmin(tmin, ti);
        tmax = fmax(tmax, ti);
        W = __dadd_rn(W, inv);
    }
    if (cd->freqs) {
        for (int j = threadIdx.x; j < cd->nf; j += blockDim.x) {
            double f = cd->freqs[j];
            if (!(f > 0.0) || !isfinite(f)) bad = true;
        }
    }
    if (bad) atomicOr(err, kErrInput);
    tmin = block_min(tmin, red);
    tmax = block_max(tmax, red);
    W = block_sum(W, red);
    const double y0 = (double)y[0];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double inv = 1.0;
        if (dy) { double dd = (double)dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
        double w = __ddiv_rn(inv, W);
        acc = __dadd_rn(acc, __dmul_rn(w, __dsub_rn((double)y[i], y0)));
    }
    acc = block_sum(acc, red);
    const double ybar = __dadd_rn(y0, acc);
    double swx2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double inv = 1.0;
        if (dy) { double dd = (double)dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
        double w = __ddiv_rn(inv, W);
        double dt = __dsub_rn(t[i], tmin);
        double x = __dsub_rn((double)y[i], ybar);
        double wx = __dmul_rn(w, x);
        float dh = __double2float_rn(dt);
        float dl = __double2float_rn(__dsub_rn(dt, (double)dh));
        pts[i] = make_float4(dh, dl, __double2float_rn(w), __double2float_rn(wx));
        dt64[i] = dt;
        swx2 = __dadd_rn(swx2, __dmul_rn(wx, x));
    }
    swx2 = block_sum(swx2, red);
    if (threadIdx.x == 0) {
        cd->t_ref = tmin;
        cd->W = W;
        cd->ybar = ybar;
        cd->sumwx2 = swx2;
        cd->dtmax = __dsub_rn(tmax, tmin);
    }
}

cudaError_t launch_prep(CurveDesc* d_curves, const int* slots, int ncurves, int* err,
                        cudaStream_t s)
{
    if (ncurves <= 0) return cudaSuccess;
    prep_kernel<<<ncurves, kPrepThreads, 0, s>>>(d_curves, slots, err);
    return cudaGetLastError();
}

// FP64 copies of w and w*x for the plain baseline.
__global__ void __launch_bounds__(kPrepThreads) prep_f64_kernel(const CurveDesc* curves,
                                                                 double* w64, double* wx64)
{
    const CurveDesc cd = curves[blockIdx.x];
    for (int i = threadIdx.x; i < cd.n; i += blockDim.x) {
        double inv = 1.0;
        if (cd.dy) { double dd = (double)cd.dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
        double w = __ddiv_rn(inv, cd.W);
        w64[cd.pt_off + i] = w;
        wx64[cd.pt_off + i] = __dmul_rn(w, __dsub_rn((double)cd.y[i], cd.ybar));
    }
}

cudaError_t launch_prep_f64(const CurveDesc* d_curves, int ncurves, double* w64, double* wx64,
                            cudaStream_t s)
{
    if (ncurves <= 0) return cudaSuccess;
    prep_f64_kernel<<<ncurves, kPrepThreads, 0, s>>>(d_curves, w64, wx64);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- a2-a6: hot kernel

constexpr int kFoldMaxThreads = 512;

size_t fold_smem_bytes(int T, int stride, int nb_max, int chunk, int kahan)
{
    (void)T;
    size_t stage = (size_t)2 * chunk * (sizeof(float4) + sizeof(double));
    size_t hist = (size_t)nb_max * stride * (kahan ? sizeof(float4) : sizeof(float2));
    return stage + hist;
}

int fold_sweep_max_threads() { return kFoldMaxThreads; }

// Box sweep of one private histogram (a5, a6): every start i1 and width k, cyclic, sums
// accumulated bin by bin from the start; a box counts when 0 < r < 1 (and s < 0 for
// dips); the best is kept with a strict '>' in (i1, k) order, compared without a divide
// as num > best * den.
template <int KAHAN, int SIGN>
__device__ __forceinline__ void sweep_private(const unsigned char* hist, int stride, int nb,
                                              int kmin, int kmax, float& bestP, int& bi1,
                                              int& bk)
{
    float best = 0.0f;
    int b1 = 0, bw = kmin;
    for (int i1 = 0; i1 < nb; ++i1) {
        float r = 0.0f, s = 0.0f, cr = 0.0f, cs = 0.0f;
        int m = i1;
        for (int k = 1; k <= kmax; ++k) {
            float hw, hx;
            if (KAHAN) {
                float4 v = reinterpret_cast<const float4*>(hist)[(size_t)m * stride];
                hw = __fsub_rn(v.x, v.z);
                hx = __fsub_rn(v.y, v.w);
                float yw = __fsub_rn(hw, cr), tw = __fadd_rn(r, yw);
                cr = __fsub_rn(__fsub_rn(tw, r), yw);
                r = tw;
                float yx = __fsub_rn(hx, cs), tx = __fadd_rn(s, yx);
                cs = __fsub_rn(__fsub_rn(tx, s), yx);
                s = tx;
            } else {
                float2 v = reinterpret_cast<const float2*>(hist)[(size_t)m * stride];
                r = __fadd_rn(r, v.x);
                s = __fadd_rn(s, v.y);
            }
            m = (m + 1 == nb) ? 0 : m + 1;
            if (k >= kmin) {
                float den = __fmaf_rn(-r, r, r);              // r (1 - r)
                float num = SIGN ? __fmul_rn(s, s) : __fmul_rn(-s, fabsf(s));
                if (num > __fmul_rn(best, den) && den > 0.0f) {
                    best = __fdiv_rn(num, den);
                    b1 = i1;
                    bw = k;
                }
            }
        }
    }
    bestP = best;
    bi1 = b1;
    bk = bw;
}

template <int PHASE, int KAHAN, int SIGN>
__global__ void __launch_bounds__(kFoldMaxThreads, 1) fold_sweep_kernel(FoldParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int CH = p.chunk;
    float4* cpts = reinterpret_cast<float4*>(smem);             // [2][CH]
    double* cdt = reinterpret_cast<double*>(cpts + 2 * CH);     // [2][CH]
    unsigned char* hist_all = reinterpret_cast<unsigned char*>(cdt + 2 * CH);
    const size_t esz = KAHAN ? sizeof(float4) : sizeof(float2);
    unsigned char* hist = hist_all + (size_t)tid * esz;         // column of this thread

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(p.counter, 1);
        __syncthreads();
        const long long it = s_item;
        if (it >= p.total) break;
        int lo = 0, hi = p.nranges;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (p.prefix[mid] <= it) lo = mid; else hi = mid;
        }
        const TileRange tr = p.ranges[lo];
        const CurveDesc& cdr = p.curves[tr.curve];
        const int n = cdr.n, nf = cdr.nf, nb = cdr.nb, kmin = cdr.kmin, kmax = cdr.kmax;
        const float4* gpts = cdr.pts;
        const double* gdt = cdr.dt64;
        const int tile = tr.tile_lo + (int)(it - p.prefix[lo]);
        const int j = tile * T + tid;
        const bool active = j < nf;
        const double f = grid_freq(cdr, active ? j : nf - 1);
        const FoldConst fc = make_fold_const(f, nb, cdr.dtmax);

        for (int b = 0; b < nb; ++b) {
            if (KAHAN)
                reinterpret_cast<float4*>(hist)[(size_t)b * p.stride] = make_float4(0.f, 0.f, 0.f, 0.f);
            else
                reinterpret_cast<float2*>(hist)[(size_t)b * p.stride] = make_float2(0.f, 0.f);
        }

        const int nchunks = (n + CH - 1) / CH;
        auto stage = [&](int ci) {
            const int c0 = ci * CH;
            const int cn = min(CH, n - c0);
            float4* dp = cpts + (ci & 1) * CH;
            double* dd = cdt + (ci & 1) * CH;
            for (int i = tid; i < cn; i += T) {
                cp_async16(&dp[i], &gpts[c0 + i]);
                cp_async8(&dd[i], &gdt[c0 + i]);
            }
            cp_async_commit();
        };
        stage(0);
        for (int ci = 0; ci < nchunks; ++ci) {
            if (ci + 1 < nchunks) stage(ci + 1); else cp_async_commit();
            cp_async_wait1();
            __syncthreads();
            const int cn = min(CH, n - ci * CH);
            const float4* cp = cpts + (ci & 1) * CH;
            const double* cd = cdt + (ci & 1) * CH;
            if (active) {
#pragma unroll 4
                for (int i = 0; i < cn; ++i) {
                    const float4 q = cp[i];
                    const int b = fold_point<PHASE>(q, &cd[i], fc);
                    if (KAHAN) {
                        float4* hp = reinterpret_cast<float4*>(hist) + (size_t)b * p.stride;
                        float4 v = *hp;
                        float yw = __fsub_rn(q.z, v.z), tw = __fadd_rn(v.x, yw);
                        v.z = __fsub_rn(__fsub_rn(tw, v.x), yw);
                        v.x = tw;
                        float yx = __fsub_rn(q.w, v.w), tx = __fadd_rn(v.y, yx);
                        v.w = __fsub_rn(__fsub_rn(tx, v.y), yx);
                        v.y = tx;
                        *hp = v;
                    } else {
                        float2* hp = reinterpret_cast<float2*>(hist) + (size_t)b * p.stride;
                        float2 v = *hp;
                        v.x = __fadd_rn(v.x, q.z);
                        v.y = __fadd_rn(v.y, q.w);
                        *hp = v;
                    }
                }
            }
            __syncthreads();
        }

        if (active) {
            float bestP;
            int bi1, bk;
            sweep_private<KAHAN, SIGN>(hist, p.stride, nb, kmin, kmax, bestP, bi1, bk);
            FreqResult r;
            r.P = bestP;
            r.box = ((uint32_t)bi1 << 16) | (uint32_t)bk;
            cdr.res[j] = r;
        }
    }
}

template <int PHASE, int KAHAN, int SIGN>
static cudaError_t launch_fold_t(const FoldParams& p, int T, int grid, size_t smem,
                                 cudaStream_t s)
{
    auto k = fold_sweep_kernel<PHASE, KAHAN, SIGN>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, T, smem, s>>>(p);
    return cudaGetLastError();
}

template <int PHASE, int KAHAN, int SIGN>
static int blocks_t(int T, size_t smem)
{
    auto k = fold_sweep_kernel<PHASE, KAHAN, SIGN>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, T, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

int fold_blocks_per_sm(int T, size_t smem, int phase, int kahan, int sign)
{
#define BLS_OCC(PH)                                                                   \
    if (phase == PH) {                                                                \
        if (kahan) return sign ? blocks_t<PH, 1, 1>(T, smem) : blocks_t<PH, 1, 0>(T, smem); \
        return sign ? blocks_t<PH, 0, 1>(T, smem) : blocks_t<PH, 0, 0>(T, smem);      \
    }
    BLS_OCC(kPhaseDF32)
    BLS_OCC(kPhaseF64)
    BLS_OCC(kPhaseF32)
#undef BLS_OCC
    return 1;
}

cudaError_t launch_fold_sweep(const FoldParams& p, int T, int grid, int phase, int kahan,
                              int sign, size_t smem, cudaStream_t s)
{
#define BLS_DISPATCH(PH)                                                              \
    if (phase == PH) {                                                                \
        if (kahan) return sign ? launch_fold_t<PH, 1, 1>(p, T, grid, smem, s)         \
                               : launch_fold_t<PH, 1, 0>(p, T, grid, smem, s);        \
        return sign ? launch_fold_t<PH, 0, 1>(p, T, grid, smem, s)                    \
                    : launch_fold_t<PH, 0, 0>(p, T, grid, smem, s);                   \
    }
    BLS_DISPATCH(kPhaseDF32)
    BLS_DISPATCH(kPhaseF64)
    BLS_DISPATCH(kPhaseF32)
#undef BLS_DISPATCH
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------- a7: reduce

constexpr int kReduceThreads = 256;

struct Cand { float P; int j; };

__device__ __forceinline__ bool better(float Pa, int ja, float Pb, int jb)
{
    return Pa > Pb || (Pa == Pb && ja < jb);
}

// Per curve: rank the local maxima of P(f_j) by (P desc, j asc) and keep topk; refit each
// chosen box in FP64 from the raw inputs (exact FP64 fold, FP64 weights) and derive
// period, epoch, duration, depth, SNR, SR.
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(ReduceParams p)
{
    __shared__ float sP[kReduceThreads / 32];
    __shared__ int sJ[kReduceThreads / 32];
    __shared__ int sT[kReduceThreads / 32];
    __shared__ int sel[kMaxTopK];
    __shared__ double red[kReduceThreads];
    const CurveDesc cd = p.curves[p.slots ? p.slots[blockIdx.x] : (int)blockIdx.x];
    const FreqResult* res = cd.res;
    const int K = p.topk;
    const int nf = cd.nf;
    Cand lst[kMaxTopK];
    int cnt = 0;
    for (int j = threadIdx.x; j < nf; j += blockDim.x) {
        const float P = res[j].P;
        if (p.spectrum) p.spectrum[cd.spec_off + j] = sqrtf(P);
        const bool lm = (j == 0 || P > res[j - 1].P) && (j == nf - 1 || P >= res[j + 1].P);
        if (!lm) continue;
        int pos = cnt < K ? cnt : K;
        for (int q = 0; q < cnt; ++q) {
            if (better(P, j, lst[q].P, lst[q].j)) { pos = q; break; }
        }
        if (pos >= K) continue;
        int last = cnt < K ? cnt : K - 1;
        for (int q = last; q > pos; --q) lst[q] = lst[q - 1];
        lst[pos].P = P;
        lst[pos].j = j;
        if (cnt < K) ++cnt;
    }
    int head = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < K; ++q) {
        float bp = head < cnt ? lst[head].P : -1.0f;
        int bj = head < cnt ? lst[head].j : 0x7fffffff;
        int bt = threadIdx.x;
        for (int o = 16; o > 0; o >>= 1) {
            float op = __shfl_xor_sync(0xffffffffu, bp, o);
            int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            int ot = __shfl_xor_sync(0xffffffffu, bt, o);
            if (better(op, oj, bp, bj)) { bp = op; bj = oj; bt = ot; }
        }
        if (lane == 0) { sP[warp] = bp; sJ[warp] = bj; sT[warp] = bt; }
        __syncthreads();
        if (threadIdx.x == 0) {
            float cp = sP[0]; int cj = sJ[0]; int ct = sT[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (better(sP[w], sJ[w], cp, cj)) { cp = sP[w]; cj = sJ[w]; ct = sT[w]; }
            sel[q] = cp >= 0.0f ? cj : -1;
            sT[0] = cp >= 0.0f ? ct : -1;
        }
        __syncthreads();
        if (sT[0] == (int)threadIdx.x) ++head;
        __syncthreads();
    }
    for (int q = 0; q < K; ++q) {
        const int j = sel[q];
        DevPeak* out = &p.peaks[(size_t)blockIdx.x * K + q];
        if (j < 0) {
            if (threadIdx.x == 0) {
                DevPeak z = {};
                z.j = -1;
                *out = z;
            }
            continue;
        }
        const FreqResult fr = res[j];
        const int i1 = (int)(fr.box >> 16), k = (int)(fr.box & 0xffffu);
        const double f = grid_freq(cd, j);
        double r = 0.0, s = 0.0;
        for (int i = threadIdx.x; i < cd.n; i += blockDim.x) {
            const double dt = __dsub_rn(cd.t[i], cd.t_ref);
            const int b = fold_exact(dt, f, cd.nb);
            int rel = b - i1;
            if (rel < 0) rel += cd.nb;
            if (rel < k) {
                double inv = 1.0;
                if (cd.dy) { double dd = (double)cd.dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
                const double w = __ddiv_rn(inv, cd.W);
                r = __dadd_rn(r, w);
                s = __dadd_rn(s, __dmul_rn(w, __dsub_rn((double)cd.y[i], cd.ybar)));
            }
        }
        r = block_sum(r, red);
        s = block_sum(s, red);
        if (threadIdx.x == 0) {
            DevPeak pk;
            pk.j = j; pk.i1 = i1; pk.k = k; pk.pad = 0;
            pk.freq = f;
            pk.period = 1.0 / f;
            pk.duration = (double)k / ((double)cd.nb * f);
            double ph = ((double)i1 + 0.5 * (double)k) / (double)cd.nb;
            ph = ph - floor(ph);
            pk.epoch = cd.t_ref + ph / f;
            const double den = r * (1.0 - r);
            const bool ok = fr.P > 0.0f && r > 0.0 && r < 1.0 && (p.sign || s < 0.0);
            if (ok) {
                pk.power = s * s / den;
                pk.depth = -s / den;
                pk.sr = sqrt(pk.power);
                pk.snr = pk.sr * sqrt(cd.W);
            } else {
                pk.power = 0.0; pk.depth = 0.0; pk.sr = 0.0; pk.snr = 0.0;
            }
            *out = pk;
        }
        __syncthreads();
    }
}

cudaError_t launch_reduce(const ReduceParams& p, int ncurves, cudaStream_t s)
{
    if (ncurves <= 0) return cudaSuccess;
    reduce_kernel<<<ncurves, kReduceThreads, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- diagnostics

template <int PHASE>
__global__ void debug_fold_kernel(const CurveDesc* curve, const int* js, int* bins)
{
    const CurveDesc cd = *curve;
    const int q = blockIdx.x;
    const double f = grid_freq(cd, js[q]);
    const FoldConst fc = make_fold_const(f, cd.nb, cd.dtmax);
    for (int i = threadIdx.x; i < cd.n; i += blockDim.x) {
        const float4 pt = cd.pts[i];
        bins[(size_t)q * cd.n + i] = fold_point<PHASE>(pt, &cd.dt64[i], fc);
    }
}

cudaError_t launch_debug_fold(const CurveDesc* d_curve, const int* js, int nj, int phase,
                              int* bins, cudaStream_t s)
{
    if (nj <= 0) return cudaSuccess;
    if (phase == kPhaseF64)
        debug_fold_kernel<kPhaseF64><<<nj, 256, 0, s>>>(d_curve, js, bins);
    else if (phase == kPhaseF32)
        debug_fold_kernel<kPhaseF32><<<nj, 256, 0, s>>>(d_curve, js, bins);
    else
        debug_fold_kernel<kPhaseDF32><<<nj, 256, 0, s>>>(d_curve, js, bins);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- baseline

constexpr int kPlainThreads = 128;
constexpr int kPlainChunk = 512;

// The paper's decomposition on B300 without redesign: each thread takes one trial period,
// the block stages the curve through shared memory, the thread phases every point, bins it
// into its own FP64 histogram (global memory: a thread's share of shared memory cannot hold
// it) and sweeps all boxes in FP64.
__global__ void __launch_bounds__(kPlainThreads) plain_f64_kernel(
    const CurveDesc* curve, const double* w64, const double* wx64, double* hist, int sign)
{
    __shared__ double s_dt[kPlainChunk], s_w[kPlainChunk], s_wx[kPlainChunk];
    const CurveDesc cd = *curve;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = j < cd.nf;
    const int nb = cd.nb, nf = cd.nf;
    const double f = grid_freq(cd, active ? j : nf - 1);
    double* hw = hist + (active ? j : 0);
    double* hx = hist + (size_t)nb * nf + (active ? j : 0);
    if (active)
        for (int b = 0; b < nb; ++b) { hw[(size_t)b * nf] = 0.0; hx[(size_t)b * nf] = 0.0; }
    for (int c0 = 0; c0 < cd.n; c0 += kPlainChunk) {
        const int cn = min(kPlainChunk, cd.n - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < cn; i += blockDim.x) {
            s_dt[i] = cd.dt64[c0 + i];
            s_w[i] = w64[cd.pt_off + c0 + i];
            s_wx[i] = wx64[cd.pt_off + c0 + i];
        }
        __syncthreads();
        if (active) {
            for (int i = 0; i < cn; ++i) {
                const int b = fold_exact(s_dt[i], f, nb);
                hw[(size_t)b * nf] = __dadd_rn(hw[(size_t)b * nf], s_w[i]);
                hx[(size_t)b * nf] = __dadd_rn(hx[(size_t)b * nf], s_wx[i]);
            }
        }
    }
    if (!active) return;
    double best = 0.0;
    int b1 = 0, bw = cd.kmin;
    for (int i1 = 0; i1 < nb; ++i1) {
        double r = 0.0, s = 0.0;
        int m = i1;
        for (int k = 1; k <= cd.kmax; ++k) {
            r = __dadd_rn(r, hw[(size_t)m * nf]);
            s = __dadd_rn(s, hx[(size_t)m * nf]);
            m = (m + 1 == nb) ? 0 : m + 1;
            if (k < cd.kmin) continue;
            if (!(r > 0.0) || !(r < 1.0)) continue;
            if (!sign && !(s < 0.0)) continue;
            const double P = __ddiv_rn(__dmul_rn(s, s), __dmul_rn(r, __dsub_rn(1.0, r)));
            if (P > best) { best = P; b1 = i1; bw = k; }
        }
    }
    FreqResult out;
    out.P = __double2float_rn(best);
    out.box = ((uint32_t)b1 << 16) | (uint32_t)bw;
    cd.res[j] = out;
}

cudaError_t launch_plain_f64(const CurveDesc* d_curve, const double* w64, const double* wx64,
                             int nf, double* hist, int sign, cudaStream_t s)
{
    const int grid = (nf + kPlainThreads - 1) / kPlainThreads;
    plain_f64_kernel<<<grid, kPlainThreads, 0, s>>>(d_curve, w64, wx64, hist, sign);
    return cudaGetLastError();
}

}  // namespace blsgpu

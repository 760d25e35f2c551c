// bls_shape.cu -- trapezoid refit of every peak a search keeps (the eclipse duration and
// the flat-bottomed shape that Sec. 5 of the paper lists as the first discriminators).
//
// At a peak's frequency f the curve is folded, phi_i = frac(RN(dt_i f)) (FP64, then held as
// FP32), and a trapezoid -- centre c, total duration T, ingress tau, in phase units -- is
// fitted to the weighted, mean-subtracted flux by least squares:
//   D = phi - c wrapped to [-1/2, 1/2],  s = clamp((T/2 - |D|) / tau, 0, 1)  (tau > 0),
//   s = [|D| < T/2]  (tau = 0, a box);
//   Ss = sum w s, Sss = sum w s^2, Sxs = sum w x s,  Q = Sxs^2 / (Sss - Ss^2),
//   depth = -Sxs / (Sss - Ss^2)   (dips only: Sxs < 0 and Sss - Ss^2 > 0).
// For a box Q is the BLS power s^2/(r(1-r)).  The grid around the peak's box (centre
// phi_b = frac((i1 + k/2)/nb), width q = k/nb) is c_m = phi_b + q (m/(nc-1) - 1/2),
// T_u = q (wlo + u (whi - wlo)/(nw-1)), tau_v = T_u amax v/(na-1); flat index
// (m nw + u) na + v, ties to the smaller index.
//
// Layout: one block per (curve, peak).  The block stages the points in chunks as
// (phi, w, w x) FP32 triples in shared memory; each thread carries the FP32 sums of up to
// kPerThread grid points in registers (more grid points take more passes).  A block
// argmax picks the best grid point and the best box (tau = 0); both are then refitted in
// FP64 from the raw inputs, so the reported power and depth carry FP64 error only.
#include <cfloat>

#include "bls_internal.h"

namespace blsgpu {
namespace {

constexpr int kShapeThreads = 256;
constexpr int kShapeChunk = 2048;
constexpr int kPerThread = 8;

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

struct GridPoint {
    double c, T, tau;
};

__device__ __forceinline__ double gfrac(int m, int n) { return n > 1 ? (double)m / (double)(n - 1) : 0.0; }

__device__ __forceinline__ GridPoint grid_point(const ShapeParams& p, double pb, double q, int idx)
{
    const int v = idx % p.na, u = (idx / p.na) % p.nw, m = idx / (p.na * p.nw);
    GridPoint g;
    g.c = pb + q * ((p.nc > 1 ? gfrac(m, p.nc) : 0.5) - 0.5);
    g.T = q * (p.wlo + gfrac(u, p.nw) * (p.whi - p.wlo));
    g.tau = g.T * (p.amax * gfrac(v, p.na));
    return g;
}

// (Q, index) order: larger Q, then smaller index.
__device__ __forceinline__ bool ahead(float qa, int ia, float qb, int ib)
{
    return qa > qb || (qa == qb && ia < ib);
}

__device__ void block_best(float& q, int& idx, float* sq, int* si)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float oq = __shfl_xor_sync(0xffffffffu, q, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ahead(oq, oi, q, idx)) { q = oq; idx = oi; }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sq[warp] = q; si[warp] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (ahead(sq[w], si[w], sq[0], si[0])) { sq[0] = sq[w]; si[0] = si[w]; }
    }
    __syncthreads();
    q = sq[0];
    idx = si[0];
    __syncthreads();
}

// FP64 refit of one trapezoid from the raw inputs (the definition's arithmetic).
__device__ void refit(const CurveDesc& cd, double f, const GridPoint& g, double* red, double* Q,
                      double* depth)
{
    double Ss = 0.0, Sss = 0.0, Sxs = 0.0;
    const double half = g.T * 0.5;
    for (int i = threadIdx.x; i < cd.n; i += blockDim.x) {
        const double dt = __dsub_rn(cd.t[i], cd.t_ref);
        const double pp = __dmul_rn(dt, f);
        const double phi = __dsub_rn(pp, floor(pp));
        const double u = __dsub_rn(phi, g.c);
        const double a = fabs(__dsub_rn(u, floor(__dadd_rn(u, 0.5))));
        double s;
        if (g.tau > 0.0) {
            s = __ddiv_rn(__dsub_rn(half, a), g.tau);
            s = s > 1.0 ? 1.0 : (s < 0.0 ? 0.0 : s);
        } else {
            s = a < half ? 1.0 : 0.0;
        }
        double inv = 1.0;
        if (cd.dy) { const double dd = (double)cd.dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
        const double w = __ddiv_rn(inv, cd.W);
        const double x = __dsub_rn((double)cd.y[i], cd.ybar);
        Ss = __dadd_rn(Ss, __dmul_rn(w, s));
        Sss = __dadd_rn(Sss, __dmul_rn(w, __dmul_rn(s, s)));
        Sxs = __dadd_rn(Sxs, __dmul_rn(__dmul_rn(w, x), s));
    }
    Ss = sum_block(Ss, red);
    Sss = sum_block(Sss, red);
    Sxs = sum_block(Sxs, red);
    const double var = __dsub_rn(Sss, __dmul_rn(Ss, Ss));
    if (Sxs < 0.0 && var > 0.0) {
        *Q = __ddiv_rn(__dmul_rn(Sxs, Sxs), var);
        *depth = __ddiv_rn(-Sxs, var);
    } else {
        *Q = 0.0;
        *depth = 0.0;
    }
}

__global__ void __launch_bounds__(kShapeThreads) shape_kernel(ShapeParams p)
{
    __shared__ float sphi[kShapeChunk], sw[kShapeChunk], swx[kShapeChunk];
    __shared__ double red[kShapeThreads];
    __shared__ float bq[kShapeThreads / 32];
    __shared__ int bi[kShapeThreads / 32];
    const int curve = blockIdx.x / p.topk;
    const CurveDesc& cd = p.curves[curve];
    const DevPeak pk = p.peaks[blockIdx.x];
    DevShape* out = &p.out[blockIdx.x];
    if (pk.j < 0 || !(pk.freq > 0.0)) {
        if (threadIdx.x == 0) {
            DevShape z = {};
            z.index = -1;
            z.box_index = -1;
            *out = z;
        }
        return;
    }
    const double f = pk.freq;
    double pb = ((double)pk.i1 + 0.5 * (double)pk.k) / (double)cd.nb;
    pb = pb - floor(pb);
    const double q = (double)pk.k / (double)cd.nb;
    const int G = p.nc * p.nw * p.na;

    float best_q = -1.0f, box_q = -1.0f;
    int best_i = 0x7fffffff, box_i = 0x7fffffff;
    for (int g0 = 0; g0 < G; g0 += kPerThread * (int)blockDim.x) {
        float c[kPerThread], half[kPerThread], invtau[kPerThread];
        float Ss[kPerThread], Sss[kPerThread], Sxs[kPerThread];
#pragma unroll
        for (int r = 0; r < kPerThread; ++r) {
            const int idx = g0 + r * (int)blockDim.x + (int)threadIdx.x;
            const GridPoint gp = grid_point(p, pb, q, idx < G ? idx : 0);
            const double cw = gp.c - floor(gp.c);   // centre in [0, 1): phases are too
            c[r] = (float)cw;
            half[r] = (float)(gp.T * 0.5);
            invtau[r] = gp.tau > 0.0 ? (float)(1.0 / gp.tau) : 1e30f;
            Ss[r] = 0.0f; Sss[r] = 0.0f; Sxs[r] = 0.0f;
        }
        for (int c0 = 0; c0 < cd.n; c0 += kShapeChunk) {
            const int cn = min(kShapeChunk, cd.n - c0);
            __syncthreads();
            for (int i = threadIdx.x; i < cn; i += blockDim.x) {
                const int ii = c0 + i;
                const double dt = __dsub_rn(cd.t[ii], cd.t_ref);
                const double pp = __dmul_rn(dt, f);
                double inv = 1.0;
                if (cd.dy) { const double dd = (double)cd.dy[ii]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
                const double w = __ddiv_rn(inv, cd.W);
                sphi[i] = (float)__dsub_rn(pp, floor(pp));
                sw[i] = (float)w;
                swx[i] = (float)__dmul_rn(w, __dsub_rn((double)cd.y[ii], cd.ybar));
            }
            __syncthreads();
            for (int i = 0; i < cn; ++i) {
                const float ph = sphi[i], w = sw[i], wx = swx[i];
#pragma unroll
                for (int r = 0; r < kPerThread; ++r) {
                    const float u = ph - c[r];
                    const float d = fabsf(u - rintf(u));
                    const float s = __saturatef((half[r] - d) * invtau[r]);
                    const float ws = w * s;
                    Ss[r] += ws;
                    Sss[r] = fmaf(ws, s, Sss[r]);
                    Sxs[r] = fmaf(wx, s, Sxs[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kPerThread; ++r) {
            const int idx = g0 + r * (int)blockDim.x + (int)threadIdx.x;
            if (idx >= G) continue;
            const float var = Sss[r] - Ss[r] * Ss[r];
            if (!(Sxs[r] < 0.0f && var > 0.0f)) continue;
            const float Qv = Sxs[r] * Sxs[r] / var;
            if (ahead(Qv, idx, best_q, best_i)) { best_q = Qv; best_i = idx; }
            if (idx % p.na == 0 && ahead(Qv, idx, box_q, box_i)) { box_q = Qv; box_i = idx; }
        }
    }
    block_best(best_q, best_i, bq, bi);
    block_best(box_q, box_i, bq, bi);
    DevShape o = {};
    o.index = best_q >= 0.0f ? best_i : -1;
    o.box_index = box_q >= 0.0f ? box_i : -1;
    if (o.index >= 0) {
        const GridPoint g = grid_point(p, pb, q, o.index);
        double Q, depth;
        refit(cd, f, g, red, &Q, &depth);
        const double cw = g.c - floor(g.c);
        o.power = Q;
        o.depth = depth;
        o.epoch = cd.t_ref + cw / f;
        o.duration = g.T / f;
        o.ingress = g.tau / f;
    }
    if (o.box_index >= 0) {
        const GridPoint g = grid_point(p, pb, q, o.box_index);
        double Q, depth;
        refit(cd, f, g, red, &Q, &depth);
        o.box_power = Q;
    }
    if (threadIdx.x == 0) *out = o;
}

}  // namespace

cudaError_t launch_shape(const ShapeParams& p, int ncurves, cudaStream_t s)
{
    if (ncurves <= 0 || p.topk <= 0) return cudaSuccess;
    shape_kernel<<<ncurves * p.topk, kShapeThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace blsgpu

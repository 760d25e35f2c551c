// bls_window.cu -- eclipse-window detection efficiency (Sec. 5 of the paper, detection-
// efficiency figure): the fraction of eclipse phases at which at least min_eclipses
// eclipses of a target with a given period contain observations, after the observing
// windows and weather have removed what they remove.
//
// For observation times t (sorted), frequency f and eclipse phase phi_m = (2m+1)/(2 nphi),
// every time is folded as u = RN(RN(RN(t_i - t_0) f) - phi_m), assigned to its nearest
// eclipse c = floor(RN(u + 1/2)), and lies in that eclipse when |RN(u - c)| <= h, h =
// RN(RN(duration f) / 2) (or RN(qfrac / 2) for a duration given as a fraction of the
// period).  Times in ascending order make c non-decreasing, so one pass counts the
// eclipses that hold at least min_points observations.  These decisions are integers
// decided by floating point, so the kernel takes them in FP64 with the same operation
// sequence as the definition, one rounding per step and no contraction.
//
// Layout: one block per frequency (grid-stride over frequencies), one thread per phase
// (blocks of up to 256 threads; more phases take more passes).  The block stages the
// times in chunks of kChunk through shared memory and converts them to phases
// v_i = RN(RN(t_i - t_0) f) once for all its threads; each thread then runs the counting
// recurrence over the staged phases.  The efficiency is a block vote per pass.
#include <cstring>

#include "bls_plan.h"

namespace blsgpu {
namespace {

constexpr int kChunk = 2048;
constexpr int kWinThreads = 256;

__global__ void window_validate_kernel(const double* t, int n, const double* freqs, int nf,
                                       int* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double ti = t[i];
        if (!isfinite(ti) || (i > 0 && ti < t[i - 1])) atomicOr(err, kErrInput);
    }
    if (freqs && i < nf) {
        const double f = freqs[i];
        if (!(f > 0.0) || !isfinite(f)) atomicOr(err, kErrInput);
    }
}

struct WindowParams {
    const double* t;
    const double* freqs;
    double fmin, df, duration, qfrac;
    int n, nf, nphi, min_eclipses, min_points;
    double* eff;
    int* counts;
};

// floor(x) for x >= -0.5, exact, with integer operations on the bits (floor and compares
// would otherwise share the FP64 pipe with the subtractions, and B300 runs FP64 at about 1/64
// of the FP32 rate): x < 0 gives -1 (-0 itself); otherwise the fraction bits below the binary point are
// cleared (x < 1 gives +0, x >= 2^52 is already an integer).
__device__ __forceinline__ double floor_from_half(double x)
{
    const long long b = __double_as_longlong(x);
    if (b < 0) return b == (long long)0x8000000000000000ull ? x : -1.0;   // -0 stays -0
    const int e = (int)(b >> 52) - 1023;
    if (e < 0) return 0.0;
    if (e >= 52) return x;
    return __longlong_as_double(b & ~((1ll << (52 - e)) - 1));
}

// |d| <= h for finite d and h >= 0: IEEE magnitudes order like their bit patterns.
__device__ __forceinline__ bool abs_le(double d, double h)
{
    return (unsigned long long)(__double_as_longlong(d) & 0x7fffffffffffffffll) <=
           (unsigned long long)__double_as_longlong(h);
}

__global__ void __launch_bounds__(kWinThreads) window_kernel(WindowParams p)
{
    __shared__ double v[kChunk];
    const double t0 = p.t[0];
    for (int k = blockIdx.x; k < p.nf; k += gridDim.x) {
        const double f = p.freqs ? p.freqs[k] : __dadd_rn(p.fmin, __dmul_rn((double)k, p.df));
        const double h = p.duration > 0.0 ? __dmul_rn(__dmul_rn(p.duration, f), 0.5)
                                          : __dmul_rn(p.qfrac, 0.5);
        int det = 0;
        for (int m0 = 0; m0 < p.nphi; m0 += blockDim.x) {
            const int m = m0 + threadIdx.x;
            const bool live = m < p.nphi;
            const double phi = __ddiv_rn((double)(2 * m + 1), (double)(2 * p.nphi));
            int ecl = 0, cnt = 0;
            bool have = false;
            double cur = 0.0;
            for (int c0 = 0; c0 < p.n; c0 += kChunk) {
                const int cn = min(kChunk, p.n - c0);
                __syncthreads();
                for (int i = threadIdx.x; i < cn; i += blockDim.x)
                    v[i] = __dmul_rn(__dsub_rn(p.t[c0 + i], t0), f);
                __syncthreads();
                if (live) {
                    for (int i = 0; i < cn; ++i) {
                        // u >= -phi > -1 (times ascending from t0, f > 0), so RN(u + 0.5) >= -0.5
                        const double u = __dsub_rn(v[i], phi);
                        const double c = floor_from_half(__dadd_rn(u, 0.5));
                        if (abs_le(__dsub_rn(u, c), h)) {
                            if (!have || __double_as_longlong(c) != __double_as_longlong(cur)) {
                                if (have && cnt >= p.min_points) ++ecl;
                                cur = c;
                                have = true;
                                cnt = 0;
                            }
                            ++cnt;
                        }
                    }
                }
            }
            if (have && cnt >= p.min_points) ++ecl;
            if (live && p.counts) p.counts[(size_t)k * p.nphi + m] = ecl;
            det += __syncthreads_count(live && ecl >= p.min_eclipses);
        }
        if (threadIdx.x == 0) p.eff[k] = __ddiv_rn((double)det, (double)p.nphi);
    }
}

}  // namespace
}  // namespace blsgpu

using namespace blsgpu;

extern "C" bls_status bls_window_efficiency(const bls_window_desc* d, void* cuda_stream,
                                            double* eff, int* counts)
{
    if (!d || !eff) return set_error(BLS_ERR_INVALID, "NULL descriptor or output");
    if (!d->t || d->n < 1) return set_error(BLS_ERR_INVALID, "need n >= 1 times (n=%d)", d ? d->n : 0);
    if (d->nf < 1) return set_error(BLS_ERR_INVALID, "need nf >= 1 (nf=%d)", d->nf);
    if (d->nphi < 1) return set_error(BLS_ERR_INVALID, "need nphi >= 1 (nphi=%d)", d->nphi);
    if (d->min_points < 1 || d->min_eclipses < 0)
        return set_error(BLS_ERR_INVALID, "min_points = %d, min_eclipses = %d", d->min_points, d->min_eclipses);
    if (!(d->duration > 0.0) && !(d->qfrac > 0.0 && d->qfrac < 1.0))
        return set_error(BLS_ERR_INVALID, "need duration > 0 or 0 < qfrac < 1");
    if (!d->freqs && (!(d->fmin > 0.0) || !(d->df >= 0.0)))
        return set_error(BLS_ERR_INVALID, "uniform grid needs fmin > 0 and df >= 0");

    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e;
    const int kt = ptr_kind(d->t), kf = d->freqs ? ptr_kind(d->freqs) : 2;
    const int ke = ptr_kind(eff), kc = counts ? ptr_kind(counts) : 2;
    const size_t tb = (size_t)d->n * 8, fb = d->freqs ? (size_t)d->nf * 8 : 0;
    const size_t eb = (size_t)d->nf * 8, cb = counts ? (size_t)d->nf * d->nphi * 4 : 0;
    // one device block: [err word | times | freqs | eff | counts], each part 256-aligned
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_t = 256, o_f = o_t + (kt == 2 ? 0 : up(tb)), o_e = o_f + (kf == 2 ? 0 : up(fb));
    const size_t o_c = o_e + (ke == 2 ? 0 : up(eb)), total = o_c + (kc == 2 ? 0 : up(cb));
    unsigned char* buf = nullptr;
    if ((e = cudaMallocAsync(&buf, total, s)) != cudaSuccess) return cuda_fail(e, "window buffers");
    int* err = reinterpret_cast<int*>(buf);
    WindowParams wp;
    wp.t = kt == 2 ? d->t : reinterpret_cast<const double*>(buf + o_t);
    wp.freqs = d->freqs ? (kf == 2 ? d->freqs : reinterpret_cast<const double*>(buf + o_f)) : nullptr;
    wp.eff = ke == 2 ? eff : reinterpret_cast<double*>(buf + o_e);
    wp.counts = counts ? (kc == 2 ? counts : reinterpret_cast<int*>(buf + o_c)) : nullptr;
    wp.fmin = d->fmin;
    wp.df = d->df;
    wp.duration = d->duration > 0.0 ? d->duration : 0.0;
    wp.qfrac = d->qfrac;
    wp.n = d->n;
    wp.nf = d->nf;
    wp.nphi = d->nphi;
    wp.min_eclipses = d->min_eclipses;
    wp.min_points = d->min_points;
    int herr = 0;
    auto run = [&]() -> cudaError_t {
        cudaError_t x;
        if ((x = cudaMemsetAsync(err, 0, sizeof(int), s)) != cudaSuccess) return x;
        if (kt != 2 && (x = cudaMemcpyAsync((void*)wp.t, d->t, tb, cudaMemcpyHostToDevice, s)) != cudaSuccess) return x;
        if (d->freqs && kf != 2 &&
            (x = cudaMemcpyAsync((void*)wp.freqs, d->freqs, fb, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return x;
        const int nv = std::max(d->n, d->freqs ? d->nf : 0);
        window_validate_kernel<<<(nv + 255) / 256, 256, 0, s>>>(wp.t, d->n, wp.freqs, d->nf, err);
        if ((x = cudaGetLastError()) != cudaSuccess) return x;
        int dev = 0, sms = 0;
        if ((x = cudaGetDevice(&dev)) != cudaSuccess) return x;
        if ((x = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return x;
        const int threads = std::min(kWinThreads, (d->nphi + 31) & ~31);
        const int grid = (int)std::min<long long>((long long)d->nf, (long long)sms * (2048 / threads));
        window_kernel<<<grid, threads, 0, s>>>(wp);
        if ((x = cudaGetLastError()) != cudaSuccess) return x;
        if (ke != 2 && (x = cudaMemcpyAsync(eff, wp.eff, eb, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return x;
        if (counts && kc != 2 &&
            (x = cudaMemcpyAsync(counts, wp.counts, cb, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return x;
        if ((x = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return x;
        return cudaStreamSynchronize(s);
    };
    e = run();
    cudaError_t ef = cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return cuda_fail(e, "window efficiency");
    if (ef != cudaSuccess) return cuda_fail(ef, "window buffers");
    if (herr & kErrInput)
        return set_error(BLS_ERR_INVALID, "times not sorted ascending or not finite, or a frequency <= 0 "
                                          "(device check)");
    if (herr) return set_error(BLS_ERR_INTERNAL, "device consistency check failed (code %d)", herr);
    return BLS_OK;
}

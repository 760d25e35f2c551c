// bls_variability.cu -- high-variability pre-filter (Sec. 2.2.1 of the paper): stars whose
// photometric variability stands more than nsig standard deviations above the expectation
// for their magnitude -- estimated per 0.1-mag bin from a sigma-clipped average over the
// stars of their chip -- are flagged before the BLS search.
//
// Per star (light curve in magnitudes): mag = mean, rms = population RMS (two passes),
// bin = floor(RN(mag * 10)).  Per (chip, bin): sigma clipping of the stars' rms values
// (mu, sd of the kept; keep |rms - mu| <= clip * sd; at most `iters` rounds, stop when the
// kept set no longer changes); flag = (bin has >= min_stars stars) && rms > mu + nsig * sd.
//
// Every sum is taken in FP64 (the paper gives no summation order): 32 interleaved partial
// sums (lane l adds elements l, l+32, ... in order) combined by an xor butterfly over
// offsets 16, 8, 4, 2, 1 -- what one warp computes with coalesced loads and shuffles.  Any
// order is within the FP64 summation bound (n - 1) 2^-53 sum |v| of the plain sequential
// sum, so a decision (bin, kept set, flag) can differ from the sequential order's only for
// a value within that bound of its threshold.  The order is fixed, so results are
// deterministic.  One warp per star takes the two passes over its light curve; one warp
// per (chip, bin) runs the clipping over the bin's stars in star order (dropped stars add
// zero in their places).  Around them, the grouping: a chip's stars are compacted in star
// order (warp ballots), counted per bin and laid out bin by bin, still in star order.
//
// Kernels: star_kernel (one warp per star), chip_count / chip_scan (stars per chip and
// their offsets), chip_kernel (one block per chip: compaction, bins, clipping, flags; a
// chip's stars live in shared memory while they fit).
#include <cstring>

#include "bls_plan.h"

namespace blsgpu {
namespace {

constexpr int kVarThreads = 256;
constexpr int kMaxBinsPerChip = 4096;   // 409.6 mag of range within one chip

// FP64 sum of one value per lane, in a fixed order: the xor butterfly.
__device__ __forceinline__ double butterfly(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// FP32 -> FP64, exact, built from the bits with integer operations: the hardware conversion
// runs on the FP64 pipe, which this kernel's sums already saturate (B300 runs FP64 at about
// 1/64 of the FP32 rate).  Normal numbers: same sign, exponent rebiased by 1023 - 127 = 896,
// mantissa widened; zeros, subnormals, infinities and NaNs take the hardware conversion.
__device__ __forceinline__ double widen(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)x;
    const unsigned hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(u << 29));
}

__global__ void star_kernel(const long long* off, const float* m, int nstars, double* mag,
                            double* rms, int* bin, int* err)
{
    const int s = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= nstars) return;
    const long long a = off[s], b = off[s + 1];
    if (!(b > a)) {
        if (lane == 0) atomicOr(err, kErrInput);
        return;
    }
    double part = 0.0;
    for (long long i = a + lane; i < b; i += 32) part = __dadd_rn(part, widen(m[i]));
    const double n = (double)(b - a);
    const double mu = __ddiv_rn(butterfly(part), n);
    part = 0.0;
    for (long long i = a + lane; i < b; i += 32) {
        const double d = __dsub_rn(widen(m[i]), mu);
        part = __dadd_rn(part, __dmul_rn(d, d));
    }
    const double v = butterfly(part);
    if (lane == 0) {
        if (!isfinite(mu)) atomicOr(err, kErrInput);
        mag[s] = mu;
        rms[s] = sqrt(__ddiv_rn(v, n));
        bin[s] = (int)floor(__dmul_rn(mu, 10.0));
    }
}

__global__ void chip_count_kernel(const int* chip, int nstars, int nchips, int* count, int* err)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nstars) return;
    const int c = chip[s];
    if (c < 0 || c >= nchips) { atomicOr(err, kErrInput); return; }
    // one atomic per distinct chip of the warp
    const unsigned grp = __match_any_sync(__activemask(), c);
    if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&count[c], __popc(grp));
}

// Exclusive prefix sum of the per-chip counts (one block; chunks of blockDim).
__global__ void chip_scan_kernel(const int* count, int nchips, int* offs)
{
    __shared__ int sh[kVarThreads];
    int carry = 0;
    for (int c0 = 0; c0 < nchips; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int v = c < nchips ? count[c] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int t = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (c < nchips) offs[c] = carry + sh[threadIdx.x] - v;
        carry += sh[blockDim.x - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) offs[nchips] = carry;
}

struct ChipParams {
    const int* chip;
    const int* offs;          // nchips + 1
    const double* rms;
    const int* bin;
    int nstars;
    double clip;
    int iters;
    double nsig;
    int min_stars;
    int* members;             // scratch: stars of each chip, in star order
    int* sorted;              // scratch: the same, bin by bin
    unsigned char* keep;      // scratch: kept flags, indexed like `sorted`
    double* mu;               // outputs per star
    double* sd;
    unsigned char* flag;
    int* err;
};

// Stars of one chip staged in shared memory (bin offset, rms, kept flag, star index in bin
// order); larger chips work on the global scratch arrays instead.
constexpr int kSmemStars = 8192;
constexpr size_t kChipSmem = (size_t)kSmemStars * (sizeof(double) + 2 * sizeof(int) + 1);

__global__ void __launch_bounds__(kVarThreads) chip_kernel(ChipParams p)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ int wsum[kVarThreads / 32];
    __shared__ int bcount[kMaxBinsPerChip + 1];
    __shared__ int s_lo, s_hi;
    const int c = blockIdx.x;
    const int base = p.offs[c], cnt = p.offs[c + 1] - base;
    if (cnt == 0) return;
    const bool staged = cnt <= kSmemStars;
    int* mem = p.members + base;
    // bin-ordered arrays: in shared memory when they fit
    double* srms = staged ? reinterpret_cast<double*>(dsm) : nullptr;
    int* sbin = staged ? reinterpret_cast<int*>(dsm + (size_t)kSmemStars * sizeof(double)) : nullptr;
    int* srt = staged ? sbin + kSmemStars : p.sorted + base;
    unsigned char* kp = staged ? reinterpret_cast<unsigned char*>(srt + kSmemStars) : p.keep + base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // (a) stable compaction of the chip's stars (warp ballots, then a scan of warp totals)
    int pos = 0;
    for (int s0 = 0; s0 < p.nstars; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        const bool in = s < p.nstars && p.chip[s] == c;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = pos, total = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) before += wsum[w];
            total += wsum[w];
        }
        if (in) mem[before + __popc(bal & ((1u << lane) - 1u))] = s;
        pos += total;
        __syncthreads();
    }
    __syncthreads();
    // (b) bin range of the chip; member bins staged
    if (threadIdx.x == 0) { s_lo = 0x7fffffff; s_hi = -0x7fffffff; }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int b = p.bin[mem[i]];
        if (staged) sbin[i] = b;
        atomicMin(&s_lo, b);
        atomicMax(&s_hi, b);
    }
    __syncthreads();
    const int lo = s_lo, nbins = s_hi - s_lo + 1;
    if (nbins > kMaxBinsPerChip || nbins < 1) {
        if (threadIdx.x == 0) atomicOr(p.err, kErrInput);
        return;
    }
    // (c) stars per bin and bin offsets
    for (int b = threadIdx.x; b <= nbins; b += blockDim.x) bcount[b] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x)
        atomicAdd(&bcount[(staged ? sbin[i] : p.bin[mem[i]]) - lo], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < nbins; ++b) { const int v = bcount[b]; bcount[b] = acc; acc += v; }
        bcount[nbins] = acc;
    }
    __syncthreads();
    // (d) bin by bin, in star order: one warp per bin appends its stars (ballots)
    for (int b = warp; b < nbins; b += nw) {
        int w = bcount[b];
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            const bool hit = i < cnt && (staged ? sbin[i] : p.bin[mem[i]]) - lo == b;
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (hit) srt[w + __popc(bal & ((1u << lane) - 1u))] = mem[i];
            w += __popc(bal);
        }
    }
    __syncthreads();
    if (staged)
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) srms[i] = p.rms[srt[i]];
    __syncthreads();
    // (e) sigma clipping, one warp per bin, sums in the warp's fixed order; (f) flags
    for (int b = warp; b < nbins; b += nw) {
        const int a = bcount[b], k = bcount[b + 1] - a;
        if (k == 0) continue;
        auto rv = [&](int i) { return staged ? srms[a + i] : p.rms[srt[a + i]]; };
        for (int i = lane; i < k; i += 32) kp[a + i] = 1;
        __syncwarp();
        double mu = 0.0, sd = 0.0;
        for (int it = 0; it <= p.iters; ++it) {
            double part = 0.0;
            int kc = 0;
            for (int i = lane; i < k; i += 32) {
                const bool kept = kp[a + i];
                part = __dadd_rn(part, kept ? rv(i) : 0.0);
                kc += kept;
            }
            for (int o = 16; o > 0; o >>= 1) kc += __shfl_xor_sync(0xffffffffu, kc, o);
            const double s = butterfly(part);
            mu = kc > 0 ? __ddiv_rn(s, (double)kc) : 0.0;
            part = 0.0;
            for (int i = lane; i < k; i += 32) {
                const double d = __dsub_rn(rv(i), mu);
                part = __dadd_rn(part, kp[a + i] ? __dmul_rn(d, d) : 0.0);
            }
            const double v = butterfly(part);
            sd = kc > 0 ? sqrt(__ddiv_rn(v, (double)kc)) : 0.0;
            if (it == p.iters) break;
            bool changed = false;
            const double lim = __dmul_rn(p.clip, sd);
            for (int i = lane; i < k; i += 32) {
                const unsigned char nk = fabs(__dsub_rn(rv(i), mu)) <= lim;
                if (nk != kp[a + i]) { kp[a + i] = nk; changed = true; }
            }
            if (!__any_sync(0xffffffffu, changed)) break;
        }
        const double thr = __dadd_rn(mu, __dmul_rn(p.nsig, sd));
        for (int i = lane; i < k; i += 32) {
            const int s = srt[a + i];
            p.mu[s] = mu;
            p.sd[s] = sd;
            p.flag[s] = (unsigned char)(k >= p.min_stars && rv(i) > thr);
        }
    }
}

// Packs the per-star outputs into the ABI records.
__global__ void pack_kernel(int nstars, const double* mag, const double* rms, const int* bin,
                            const double* mu, const double* sd, const unsigned char* flag,
                            bls_var_star* out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nstars) return;
    bls_var_star r;
    memset(&r, 0, sizeof(r));
    r.mag = mag[s]; r.rms = rms[s]; r.mu = mu[s]; r.sd = sd[s];
    r.bin = bin[s]; r.flag = flag[s];
    out[s] = r;
}

}  // namespace
}  // namespace blsgpu

using namespace blsgpu;

extern "C" bls_status bls_variability(const bls_var_desc* d, void* cuda_stream, bls_var_star* out)
{
    if (!d || !out || !d->off || !d->m || !d->chip) return set_error(BLS_ERR_INVALID, "NULL argument");
    if (d->nstars < 1 || d->nchips < 1)
        return set_error(BLS_ERR_INVALID, "nstars = %d, nchips = %d", d->nstars, d->nchips);
    if (!(d->clip > 0.0) || d->iters < 0 || !(d->nsig >= 0.0) || d->min_stars < 1)
        return set_error(BLS_ERR_INVALID, "clip = %g, iters = %d, nsig = %g, min_stars = %d", d->clip, d->iters,
                         d->nsig, d->min_stars);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e;
    const int ko = ptr_kind(d->off), km = ptr_kind(d->m), kc = ptr_kind(d->chip), kout = ptr_kind(out);
    const size_t ns = (size_t)d->nstars, nc = (size_t)d->nchips;
    long long npts = 0;
    if (ko == 2) {
        if ((e = cudaMemcpyAsync(&npts, d->off + ns, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "reading the point count");
    } else {
        npts = d->off[ns];
    }
    if (npts < 1) return set_error(BLS_ERR_INVALID, "no points");
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    // one device block for everything: [err | off | m | chip | mag | rms | bin | mu | sd | flag |
    //  count | offs | members | sorted | keep | out]
    size_t o = 256;
    const size_t o_off = o;   o += ko == 2 ? 0 : up((ns + 1) * 8);
    const size_t o_m = o;     o += km == 2 ? 0 : up((size_t)npts * 4);
    const size_t o_chip = o;  o += kc == 2 ? 0 : up(ns * 4);
    const size_t o_mag = o;   o += up(ns * 8);
    const size_t o_rms = o;   o += up(ns * 8);
    const size_t o_bin = o;   o += up(ns * 4);
    const size_t o_mu = o;    o += up(ns * 8);
    const size_t o_sd = o;    o += up(ns * 8);
    const size_t o_flag = o;  o += up(ns);
    const size_t o_cnt = o;   o += up(nc * 4);
    const size_t o_offs = o;  o += up((nc + 1) * 4);
    const size_t o_mem = o;   o += up(ns * 4);
    const size_t o_srt = o;   o += up(ns * 4);
    const size_t o_keep = o;  o += up(ns);
    const size_t o_out = o;   o += kout == 2 ? 0 : up(ns * sizeof(bls_var_star));
    unsigned char* buf = nullptr;
    if ((e = cudaMallocAsync(&buf, o, s)) != cudaSuccess) return cuda_fail(e, "variability buffers");
    int* err = reinterpret_cast<int*>(buf);
    const long long* doff = ko == 2 ? d->off : reinterpret_cast<const long long*>(buf + o_off);
    const float* dm = km == 2 ? d->m : reinterpret_cast<const float*>(buf + o_m);
    const int* dchip = kc == 2 ? d->chip : reinterpret_cast<const int*>(buf + o_chip);
    bls_var_star* dout = kout == 2 ? out : reinterpret_cast<bls_var_star*>(buf + o_out);
    double* mag = reinterpret_cast<double*>(buf + o_mag);
    double* rms = reinterpret_cast<double*>(buf + o_rms);
    int* bin = reinterpret_cast<int*>(buf + o_bin);
    int herr = 0;
    auto run = [&]() -> cudaError_t {
        cudaError_t x;
        if ((x = cudaMemsetAsync(err, 0, 4, s)) != cudaSuccess) return x;
        if ((x = cudaMemsetAsync(buf + o_cnt, 0, nc * 4, s)) != cudaSuccess) return x;
        if (ko != 2 && (x = cudaMemcpyAsync((void*)doff, d->off, (ns + 1) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return x;
        if (km != 2 && (x = cudaMemcpyAsync((void*)dm, d->m, (size_t)npts * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return x;
        if (kc != 2 && (x = cudaMemcpyAsync((void*)dchip, d->chip, ns * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return x;
        const int g = (int)((ns + kVarThreads - 1) / kVarThreads);
        const int gw = (int)((ns * 32 + kVarThreads - 1) / kVarThreads);   // one warp per star
        star_kernel<<<gw, kVarThreads, 0, s>>>(doff, dm, d->nstars, mag, rms, bin, err);
        chip_count_kernel<<<g, kVarThreads, 0, s>>>(dchip, d->nstars, d->nchips,
                                                   reinterpret_cast<int*>(buf + o_cnt), err);
        chip_scan_kernel<<<1, kVarThreads, 0, s>>>(reinterpret_cast<int*>(buf + o_cnt), d->nchips,
                                                  reinterpret_cast<int*>(buf + o_offs));
        ChipParams cp;
        cp.chip = dchip;
        cp.offs = reinterpret_cast<int*>(buf + o_offs);
        cp.rms = rms;
        cp.bin = bin;
        cp.nstars = d->nstars;
        cp.clip = d->clip;
        cp.iters = d->iters;
        cp.nsig = d->nsig;
        cp.min_stars = d->min_stars;
        cp.members = reinterpret_cast<int*>(buf + o_mem);
        cp.sorted = reinterpret_cast<int*>(buf + o_srt);
        cp.keep = buf + o_keep;
        cp.mu = reinterpret_cast<double*>(buf + o_mu);
        cp.sd = reinterpret_cast<double*>(buf + o_sd);
        cp.flag = buf + o_flag;
        cp.err = err;
        if ((x = cudaFuncSetAttribute(chip_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kChipSmem)) != cudaSuccess)
            return x;
        chip_kernel<<<d->nchips, kVarThreads, kChipSmem, s>>>(cp);
        pack_kernel<<<g, kVarThreads, 0, s>>>(d->nstars, mag, rms, bin, cp.mu, cp.sd, cp.flag, dout);
        if ((x = cudaGetLastError()) != cudaSuccess) return x;
        if (kout != 2 && (x = cudaMemcpyAsync(out, dout, ns * sizeof(bls_var_star), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return x;
        if ((x = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return x;
        return cudaStreamSynchronize(s);
    };
    e = run();
    cudaError_t ef = cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return cuda_fail(e, "variability");
    if (ef != cudaSuccess) return cuda_fail(ef, "variability buffers");
    if (herr & kErrInput)
        return set_error(BLS_ERR_INVALID, "a star has no points or non-finite magnitudes, a chip id is out of range, "
                                          "or one chip spans more than %d bins (device check)", kMaxBinsPerChip);
    if (herr) return set_error(BLS_ERR_INTERNAL, "device consistency check failed (code %d)", herr);
    return BLS_OK;
}

// bls_static.cu -- search of one curve with no memory allocation.
//
// Some callers cannot call cudaMalloc: a plug-in whose host application owns and budgets
// all device memory, a latency-critical loop where cudaMalloc's implicit device
// synchronisation is not acceptable, or a process under a memory cap where allocating
// after start-up may fail.  bls_search_static serves them: the caller passes device
// inputs and device outputs, and all intermediate data (curve descriptor, prepared
// points, per-frequency powers, work list) lives in one file-scope __device__ array of
// fixed size, kStaticScratchBytes, which every GPU that loads the library holds until
// the process exits.
#include <cstring>
#include <mutex>

#include <cstddef>

#include "bls_plan.h"

namespace blsgpu {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB per device

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The symbol's host name is
// only a stand-in, so the address is looked up once per device, with that device
// current, and cached.
bls_status static_scratch(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return set_error(BLS_ERR_INVALID, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
        g_static_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_ptr[dev];
    return BLS_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

bool on_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Writes the descriptor and the one-range work list into the scratch and clears the work
// counter and the error word (the scratch keeps the previous call's contents).
__global__ void static_init_kernel(CurveDesc d, CurveDesc* cdesc, TileRange* range,
                                   long long* prefix, long long ntiles, int* counter, int* err)
{
    *cdesc = d;
    range->curve = 0;
    range->tile_lo = 0;
    prefix[0] = 0;
    prefix[1] = ntiles;
    *counter = 0;
    *err = 0;
}

}  // namespace
}  // namespace blsgpu

using namespace blsgpu;

extern "C" bls_status bls_search_static(const bls_curve* c, int topk, int sign, void* cuda_stream,
                                        bls_peak* peaks_dev, float* spectrum_dev)
{
    if (!c || !peaks_dev) return set_error(BLS_ERR_INVALID, "NULL curve or output");
    if (c->n < 2 || c->nf < 1) return set_error(BLS_ERR_INVALID, "need n >= 2 and nf >= 1 (n=%d nf=%d)", c->n, c->nf);
    if (c->nb < 2 || c->nb > 4096) return set_error(BLS_ERR_INVALID, "nb = %d, need 2..4096", c->nb);
    if (topk < 1 || topk > kMaxTopK) return set_error(BLS_ERR_INVALID, "topk = %d, need 1..%d", topk, kMaxTopK);
    if (sign != BLS_SIGN_DIPS && sign != BLS_SIGN_BOTH) return set_error(BLS_ERR_INVALID, "sign = %d", sign);
    if (!c->freqs && (!(c->fmin > 0.0) || !(c->df >= 0.0)))
        return set_error(BLS_ERR_INVALID, "uniform grid needs fmin > 0 and df >= 0");
    int kmin, kmax;
    bls_status st = bls_kminmax(c->nb, c->qmin, c->qmax, &kmin, &kmax);
    if (st != BLS_OK) return st;
    if (!c->t || !c->y || !on_device(c->t) || !on_device(c->y) || (c->dy && !on_device(c->dy)) ||
        (c->freqs && !on_device(c->freqs)) || !on_device(peaks_dev) || (spectrum_dev && !on_device(spectrum_dev)))
        return set_error(BLS_ERR_INVALID, "bls_search_static takes device memory only (inputs and outputs)");

    // scratch layout
    const long long n2 = (c->n + 1) & ~1;
    size_t off = 0;
    const size_t o_desc = off;   off += up256(sizeof(CurveDesc));
    const size_t o_range = off;  off += up256(sizeof(TileRange));
    const size_t o_prefix = off; off += up256(2 * sizeof(long long));
    const size_t o_words = off;  off += 256;
    const size_t o_pts = off;    off += up256((size_t)(n2 + 2) * sizeof(float4));
    const size_t o_dt = off;     off += up256((size_t)(n2 + 2) * sizeof(double));
    const size_t o_res = off;    off += up256((size_t)c->nf * sizeof(float));
    if (off > kStaticScratchBytes)
        return set_error(BLS_ERR_INVALID, "n = %d and nf = %d need %zu bytes of static scratch, more than its %zu",
                         c->n, c->nf, off, kStaticScratchBytes);

    int dev = 0, sms = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    unsigned char* S = nullptr;
    if ((st = static_scratch(dev, &S)) != BLS_OK) return st;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return cuda_fail(e, "device attributes");

    // block geometry as in a plan with default settings
    const size_t avail_all = (size_t)optin - kFoldSmemReserve;
    auto tmax = [&](int chunk) {
        const size_t stage = (size_t)2 * chunk * 24;
        const size_t avail = avail_all > stage ? avail_all - stage : 0;
        const size_t cap = avail / ((size_t)c->nb * 8);
        int T = (int)std::min<size_t>(cap, (size_t)fold_sweep_max_threads()) & ~15;
        while (T >= 16 && fold_smem_bytes(T, T, c->nb, chunk, kSumF32) > avail_all) T -= 16;
        return T;
    };
    const int chunk = tmax(512) >= tmax(256) ? 512 : 256;
    const int T = fold_preferred_cols(tmax(chunk), kSumF32, c->nb, kmin, kmax, BLS_FOLD_AUTO);
    const int ws = fold_ws_mode(T, kSumF32, c->nb, kmin, kmax, BLS_FOLD_AUTO);
    if (T < 16) return set_error(BLS_ERR_INVALID, "nb = %d needs more shared memory than a block has", c->nb);
    const size_t smem = fold_smem_bytes(T, T, c->nb, chunk, kSumF32);

    CurveDesc d;
    memset(&d, 0, sizeof(d));
    d.t = c->t; d.y = c->y; d.dy = c->dy; d.freqs = c->freqs;
    d.pts = reinterpret_cast<float4*>(S + o_pts);
    d.dt64 = reinterpret_cast<double*>(S + o_dt);
    d.res = reinterpret_cast<float*>(S + o_res);
    d.pt_off = 0; d.spec_off = 0;
    d.fmin = c->fmin; d.df = c->df;
    d.n = c->n; d.nf = c->nf; d.nb = c->nb; d.kmin = kmin; d.kmax = kmax; d.T = T;
    CurveDesc* cdesc = reinterpret_cast<CurveDesc*>(S + o_desc);
    TileRange* range = reinterpret_cast<TileRange*>(S + o_range);
    long long* prefix = reinterpret_cast<long long*>(S + o_prefix);
    int* counter = reinterpret_cast<int*>(S + o_words);
    int* err = counter + 1;
    const long long ntiles = (c->nf + T - 1) / T;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    static_init_kernel<<<1, 1, 0, s>>>(d, cdesc, range, prefix, ntiles, counter, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "static init launch");
    if ((e = launch_prep(cdesc, nullptr, 1, err, kPhaseFX64, kSumF32, s)) != cudaSuccess) return cuda_fail(e, "prep launch");
    FoldParams fp;
    fp.curves = cdesc;
    fp.ranges = range;
    fp.prefix = prefix;
    fp.nranges = 1;
    fp.total = ntiles;
    fp.counter = counter;
    fp.err = err;
    fp.chunk = chunk;
    fp.stride = T;
    fp.wait_ns = 0;
    long long grid = (long long)sms * fold_blocks_per_sm(T, smem, kPhaseFX64, kSumF32, sign, ws);
    if (grid > ntiles) grid = ntiles;
    if ((e = launch_fold_sweep(fp, T, (int)grid, kPhaseFX64, kSumF32, ws, sign, smem, s)) != cudaSuccess)
        return cuda_fail(e, "fold-sweep launch");
    ReduceParams rp;
    rp.curves = cdesc;
    rp.slots = nullptr;
    // the reduce kernel writes the caller's bls_peak records directly
    static_assert(sizeof(DevPeak) == sizeof(bls_peak), "DevPeak mirrors bls_peak");
    static_assert(offsetof(DevPeak, j) == offsetof(bls_peak, best_j) &&
                  offsetof(DevPeak, i1) == offsetof(bls_peak, i1) &&
                  offsetof(DevPeak, k) == offsetof(bls_peak, k) &&
                  offsetof(DevPeak, pad) == offsetof(bls_peak, pad_) &&
                  offsetof(DevPeak, freq) == offsetof(bls_peak, freq) &&
                  offsetof(DevPeak, period) == offsetof(bls_peak, period) &&
                  offsetof(DevPeak, epoch) == offsetof(bls_peak, epoch) &&
                  offsetof(DevPeak, duration) == offsetof(bls_peak, duration) &&
                  offsetof(DevPeak, depth) == offsetof(bls_peak, depth) &&
                  offsetof(DevPeak, snr) == offsetof(bls_peak, snr) &&
                  offsetof(DevPeak, sr) == offsetof(bls_peak, sr) &&
                  offsetof(DevPeak, power) == offsetof(bls_peak, power) &&
                  offsetof(DevPeak, sde) == offsetof(bls_peak, sde),
                  "DevPeak fields sit where bls_peak's do");
    rp.peaks = reinterpret_cast<DevPeak*>(peaks_dev);
    rp.spectrum = spectrum_dev;
    rp.topk = topk;
    rp.sign = sign;
    rp.phase = kPhaseFX64;
    rp.sums = kSumF32;
    rp.smem_bytes = reduce_smem_bytes(c->nb, topk, kSumF32);
    rp.err = err;
    if ((e = launch_reduce(rp, 1, s)) != cudaSuccess) return cuda_fail(e, "reduce launch");
    int host_err = 0;
    if ((e = cudaMemcpyAsync(&host_err, err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "copying the error word");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "static search");
    if (host_err & kErrInput)
        return set_error(BLS_ERR_INVALID, "the curve has a non-finite time or flux, a non-positive error, or a "
                                          "non-positive frequency (device check)");
    if (host_err) return set_error(BLS_ERR_INTERNAL, "device consistency check failed (code %d)", host_err);
    return BLS_OK;
}

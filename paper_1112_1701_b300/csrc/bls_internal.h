// bls_internal.h -- device data layout and kernel launchers of the B300 BLS library.
//
// HBM layout (one search launch):
//   CurveDesc[ncurves]          per-curve scalars and pointers (inputs, prepared points,
//                               per-frequency results)
//   float4 pts[n]               prepared points (dt_hi, dt_lo, w, w*x), 16 B per point; in
//                               the fixed-point sum mode w and w*x are 32-bit integers
//   double dt64[n]              exact FP64 time offsets, read only by the exact re-fold
//   float res[nf]               per-frequency largest box power P (FP32)
//   DevPeak peaks[ncurves*topk] reduced peaks (FP64)
// The batched search packs all curves of a launch into shared pools (curves start on even
// point offsets, so every per-curve slice is 16-byte aligned); the server gives each
// request its own allocation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace blsgpu {

constexpr int kMaxTopK = 16;
constexpr int kPhaseFX64 = 0, kPhaseF64 = 1, kPhaseF32 = 2, kPhaseDF32 = 3;
// Sum modes (the values of BLS_SUM_*): histogram entries are (W, X) integer pairs (fixed,
// 8 B), FP32 pairs (8 B) or FP32 pairs with their compensations (Kahan, 16 B).
constexpr int kSumFixed = 0, kSumF32 = 1, kSumKahan = 2;
__host__ __device__ constexpr int hist_entry_bytes(int sums) { return sums == kSumKahan ? 16 : 8; }

struct CurveDesc {
    const double* t;       // raw times (device)
    const float* y;        // raw fluxes (device)
    const float* dy;       // raw errors (device) or nullptr: unit weights
    const double* freqs;   // explicit grid (device) or nullptr: uniform grid
    float4* pts;           // prepared points of this curve
    double* dt64;          // exact time offsets of this curve
    float* res;            // per-frequency largest power of this curve
    long long pt_off;      // first point in the pooled arrays (baseline path)
    long long spec_off;    // first slot of this curve in a spectrum output
    double fmin, df;       // uniform grid
    double t_ref, W, ybar, sumwx2, dtmax;  // written by the prep kernel
    int n, nf, nb, kmin, kmax;
    int T;                 // frequencies per tile of this curve (block size of its class)
    int fxs;               // fixed-point scale of the FX64 fold: DT = dt 2^fxs (prep kernel)
    // fixed-point sums (prep kernel): a bin's integer sums (W, X) stand for
    // r = W * wq and s = X * xq (wq = 1 / sum of all W, xq = 1 / the scale of w x)
    float wq, xq;
    // incremental fold of uniform-grid tiles (prep kernel): incok if the grid is uniform and
    // dF = RN_int(df 2^(96 - fxs)) < 2^63; the edge window's error bound of a column is
    // E = fcen ewc + ew0 + |tau| ewt + max(f, fcen) ewh + f ewf (coefficients rounded up)
    unsigned long long dF;
    float ewc, ew0, ewt, ewh, ewf;
    int incok;
};

// A run of frequency tiles of one curve processed by one fold-sweep launch.
struct TileRange {
    int curve;
    int tile_lo;
};

struct DevPeak {
    int j, i1, k, pad;
    double freq, period, epoch, duration, depth, snr, sr, power, sde;
};

// Error bits written by device code into the plan's error word.
enum : int {
    kErrInput = 1,      // non-finite time/flux, non-positive error, bad frequency
    kErrBounds = 2,     // a device-side index check failed
    kErrTimeout = 4,    // a bounded wait between a kernel's warp groups gave up
};

// Device-side index checks of the BLS_DEBUG build (libbls_debug.so): bls_ok(cond, err)
// records kErrBounds in the error word when cond is false and returns cond, so the caller
// skips or redirects the access; the search then fails with BLS_ERR_INTERNAL.  In the
// regular build it is the constant true and the check compiles away.
#ifdef __CUDACC__
#ifdef BLS_DEBUG
__device__ __forceinline__ bool bls_ok(bool cond, int* err)
{
    if (!cond && err) atomicOr(err, kErrBounds);
    return cond;
}
#else
__device__ __forceinline__ constexpr bool bls_ok(bool, int*) { return true; }
#endif
#endif

// Shared memory per fold-sweep block kept free for the kernels' static arrays (the
// warp-specialised kernel's hand-over slots and partial maxima).
constexpr size_t kFoldSmemReserve = 2048;

struct FoldParams {
    const CurveDesc* curves;
    const TileRange* ranges;
    const long long* prefix;   // prefix[r] = tiles before range r; prefix[nranges] = total
    int nranges;
    long long total;
    int* counter;              // work counter (zeroed before the launch)
    int* err;
    int chunk;                 // points per staged chunk (a multiple of 16)
    int stride;                // histogram stride in entries (multiple of 16, >= cols)
    int cols;                  // frequencies per tile (set by launch_fold_sweep)
    unsigned long long wait_ns;   // limit of each warp-group hand-over wait (0: 30 s)
};

// Trapezoid refit of a peak (same layout as bls_shape).
struct DevShape {
    int index, box_index;
    double power, box_power, epoch, duration, ingress, depth;
};

struct ShapeParams {
    const CurveDesc* curves;
    const DevPeak* peaks;      // peaks of curve c at [c*topk, (c+1)*topk)
    DevShape* out;             // same indexing
    int topk;
    int nc, nw, na;            // grid: centres, widths, ingress fractions
    double wlo, whi, amax;     // widths in box widths; largest ingress / width
};

cudaError_t launch_shape(const ShapeParams& p, int ncurves, cudaStream_t s);

// Unbinned (edge-to-edge) search of one launch group.
struct UblsParams {
    const CurveDesc* curves;
    int ncurves;
    const long long* tile_prefix;   // ncurves + 1: frequency tiles before curve c
    const float* res_base;          // pool of the per-frequency powers
    DevPeak* peaks;                 // topk per curve
    float* spectrum;                // optional (device): SR per frequency, at spec_off
    int topk, sign;
    double qmin, qmax;              // run extent bounds, in cycles
    int nmax, M;                    // largest curve of the group and the power of two >= it
    int* err;                       // error word (index checks of the BLS_DEBUG build)
    long long nitems;               // work items (curve, frequency tile) of the search
    // working arrays of curves too long for shared memory: block b's keys and prefix sums
    // at scratch + b * scratch_stride, grid persistent blocks (nullptr: shared memory, one
    // block per item or curve)
    unsigned char* scratch;
    size_t scratch_stride;
    int grid;
};

cudaError_t launch_ubls(const UblsParams& p, cudaStream_t s);
cudaError_t launch_ubls_reduce(const UblsParams& p, cudaStream_t s);
// Bytes of one block's working arrays (keys and prefix sums) for curves of up to nmax points.
size_t ubls_work_bytes(int nmax);
int ubls_tile();

struct ReduceParams {
    const CurveDesc* curves;
    const int* slots;          // curve of block b = slots[b] (nullptr: b)
    DevPeak* peaks;            // peaks of block b at [b*topk, (b+1)*topk)
    float* spectrum;           // optional (device): SR per frequency, at spec_off
    int topk;
    int sign;
    int phase;                 // fold mode of the search (for the best-box recomputation)
    int sums;                  // sum mode of the search (kSum*)
    size_t smem_bytes;         // dynamic shared memory of the launch (reduce_smem_bytes)
    int* err;                  // error word (index checks of the BLS_DEBUG build)
};

// Shared memory a fold-sweep block needs.
size_t fold_smem_bytes(int T, int stride, int nb_max, int chunk, int sums);

// sums: the sum mode whose point layout the prep kernel writes (kSum*).
cudaError_t launch_prep(CurveDesc* d_curves, const int* slots, int ncurves, int* err, int phase,
                        int sums, cudaStream_t s);
cudaError_t launch_fold_sweep(const FoldParams& p, int T, int grid, int phase, int sums, int ws,
                              int sign, size_t smem, cudaStream_t s);
cudaError_t launch_reduce(const ReduceParams& p, int ncurves, cudaStream_t s);
size_t reduce_smem_bytes(int nb_max, int topk, int sums);
// Diagnostics: (P, i1, k) of the best box at every frequency of one prepared curve.
cudaError_t launch_argmax(const CurveDesc* d_curve, int nb, int nf, int phase, int sums,
                          int sign, float* P, int* i1, int* k, cudaStream_t s);
// T, sums: the tile width and sum mode the plan's search uses for this curve.
cudaError_t launch_debug_fold(const CurveDesc* d_curve, const int* js, int nj, int phase,
                              int T, int sums, int* bins, cudaStream_t s);
// Baseline: one curve, one thread per frequency, FP64 histograms in global scratch.
cudaError_t launch_plain_f64(const CurveDesc* d_curve, const double* w64, const double* wx64,
                             int nf, double* hist, int sign, cudaStream_t s);
cudaError_t launch_prep_f64(const CurveDesc* d_curves, int ncurves, double* w64, double* wx64,
                            cudaStream_t s);
int fold_sweep_max_threads();
// Whether a class of curves (tile width T, nb, widths kmin..kmax) runs in the
// warp-specialised fold-sweep kernel under the plan's choice (BLS_FOLD_*), and the tile
// width preferred for it.
bool fold_use_ws(int T, int sums, int nb, int kmin, int kmax, int choice);
int fold_preferred_cols(int tmax, int sums, int nb, int kmin, int kmax, int choice);
int fold_blocks_per_sm(int T, size_t smem, int phase, int sums, int sign, int ws);
// Kernel of a class: 0 one-group, 1 warp-specialised.
int fold_ws_mode(int T, int sums, int nb, int kmin, int kmax, int choice);
int fold_block_threads(int cols);   // threads of a fold-sweep block with `cols` columns

}  // namespace blsgpu

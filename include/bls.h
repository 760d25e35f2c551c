/*
 * bls.h -- C ABI of the B300 box-least-squares (BLS) transit search.
 *
 * The method is the GPU eclipse search of Sec. 2.2.2 of the paper: a standard BLS
 * (Kovacs, Zucker & Mazeh 2002; Tingley 2003, cited there) that phases every light
 * curve at every trial period, tests a range of box durations and phases, and keeps
 * the best.  The paper prints no formula; the statistic computed here is
 *
 *   w_i = dy_i^-2 / W, W = sum dy_i^-2;  x_i = y_i - sum w y;
 *   for a box B of phase bins: r = sum_B w, s = sum_B w x,
 *   P = s^2 / (r (1 - r)),  SR = sqrt(P),  depth = -s / (r (1 - r)),  SNR = SR sqrt(W).
 *
 * Phases are cut into nb equal bins; B runs over cyclic runs of k consecutive bins,
 * kmin <= k <= kmax.  The peak of each curve is the frequency with the largest P
 * (ties to the smallest frequency index, then the smallest start bin, then the
 * smallest width).
 *
 * Conventions for every entry point:
 *   - Status codes are returned; nothing is thrown, nothing aborts.  On failure
 *     bls_last_error() returns a message for the calling thread.
 *   - Input arrays may be host memory (pageable or pinned) or device memory of the
 *     plan's device; the library tells them apart by cudaPointerGetAttributes.  The
 *     caller keeps ownership.  The library never writes to inputs and does not keep
 *     pointers to them after the call returns (bls_submit copies its input).
 *   - Output arrays are caller-owned: `out` peaks are host memory; a spectrum may be
 *     host or device memory.
 *   - A plan is not thread-safe for concurrent bls_search calls (they serialise on an
 *     internal lock); bls_submit/bls_poll may be called from any thread.
 */
#ifndef BLS_H
#define BLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BLS_API_VERSION 1

typedef enum {
    BLS_OK = 0,
    BLS_PENDING = 1,          /* bls_poll: the request is not finished yet */
    BLS_ERR_INVALID = -1,     /* bad argument or input value (NaN, dy <= 0, n < 2, ...) */
    BLS_ERR_NOMEM = -2,       /* device or host allocation failed, or over budget */
    BLS_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    BLS_ERR_TIMEOUT = -4,     /* bls_poll waited timeout_ms without completion */
    BLS_ERR_INTERNAL = -5,    /* a device-side consistency check failed */
    BLS_ERR_CANCELLED = -6    /* the request was cancelled */
} bls_status;

/* Phase step (fold) precision. */
enum {
    BLS_PHASE_FX64 = 0,  /* default: 64-bit fixed-point product (integer multiply-adds) with
                            an error bound; points whose bin is not certain are re-folded in
                            FP64 (bins identical to FP64) */
    BLS_PHASE_F64 = 1,   /* every point folded in FP64 */
    BLS_PHASE_F32 = 2,   /* FP32 product, no fallback (precision study only: bins can differ) */
    BLS_PHASE_DF32 = 3   /* double-FP32 product with an error bound and the same FP64
                            re-fold (bins identical to FP64) */
};

/* Accumulation of the phase histograms and box sums. */
enum {
    BLS_SUM_FIXED = 0,   /* default: each point's w and w x are rounded once to 32-bit fixed
                            point (w to 2^-32 of the curve's total weight, w x to 2^-31 of
                            sum |w x|), every bin sums them exactly with integer additions
                            (independent of order), and each bin sum is converted to FP32
                            for the box sweep (FP32 box sums) */
    BLS_SUM_F32 = 1,     /* FP32 bin and box sums */
    BLS_SUM_KAHAN = 2    /* FP32 with Kahan compensation (bins and box sums) */
};

/* Which boxes count. */
enum {
    BLS_SIGN_DIPS = 0,   /* default: only boxes below the mean (s < 0): eclipses and transits */
    BLS_SIGN_BOTH = 1    /* dips and bumps */
};

/* Kernel family. */
enum {
    BLS_ALGO_TILED = 0,     /* default: batched persistent fold-bin-sweep kernels */
    BLS_ALGO_PLAIN_F64 = 1, /* baseline: one launch per curve, one thread per frequency, FP64 */
    BLS_ALGO_UNBINNED = 2   /* unbinned (edge-to-edge) boxes: at every frequency the points are
                               ordered by phase and every cyclic run of consecutive points whose
                               phase extent lies in [qmin, qmax] is a box.  A point's phase is
                               the FP64 fold frac(RN(dt f)); order (phase, point index); a run's
                               extent RN(phase_last - phase_first), plus one cycle (RN(d + 1))
                               when the run wraps through phase 0, compared in FP64.  Peaks
                               report i1 = the run's first position in phase order and k = its
                               number of points.  Up to 32768 points per curve (beyond ~8k the
                               working arrays live in a global scratch buffer of about 0.6 MB
                               per SM at 20,000 points); the plan's qmin/qmax apply to every
                               curve. */
};

/* Fold-sweep kernel of the tiled search.  BLS_FOLD_AUTO chooses per class of curves: the
 * warp-specialised kernel (a binning warp group and a sweep warp group that takes each
 * tile's histograms over through tensor memory) where the tile width is a multiple of 8 up
 * to 128 frequencies (any sum mode), the fast sweep covers the widths (kmax - kmin + 1 >=
 * SB - 1, SB = 4 for kmax - kmin < 14, else 8 or 10) and nb <= 256 (the bins fit the TMEM
 * copy), otherwise the one-group kernel (every thread bins, then every thread sweeps).
 * BLS_FOLD_WS asks for the warp-specialised kernel wherever the tile width allows it (tiles whose copy does not fit are then swept from shared memory by the sweep
 * group); BLS_FOLD_ONE_GROUP always takes the one-group kernel.  The environment variable
 * BLS_FOLD_WS=0 forces the one-group kernel for every plan.  All give the FP64 bins; the
 * per-frequency powers of the two kernels agree within the sweep's 2^-22 approximation. */
enum {
    BLS_FOLD_AUTO = 0,
    BLS_FOLD_WS = 1,
    BLS_FOLD_ONE_GROUP = 2
};

typedef struct {
    int nb;                     /* phase bins (>= 2); a curve may override */
    double qmin, qmax;          /* fractional box duration range, 0 < qmin <= qmax < 1 */
    int kmin, kmax;             /* box widths in bins; 0 = derive from q (bls_kminmax) */
    int topk;                   /* peaks returned per curve, 1..16 */
    int phase;                  /* BLS_PHASE_* */
    int sum;                    /* BLS_SUM_* */
    int sign;                   /* BLS_SIGN_* */
    int algo;                   /* BLS_ALGO_* */
    size_t max_device_bytes;    /* device memory budget of the plan; 0 = half the free memory */
    int max_curves_per_launch;  /* 0 = as many as the budget allows */
    int freqs_per_block;        /* frequencies per thread block; 0 = tuned */
    int point_chunk;            /* points staged in shared memory at a time (rounded up to a
                                   multiple of 16, at least 32); 0 = tuned */
    int max_active_requests;    /* serving: requests resident on the device at once; 0 = 64 */
    long long step_point_freqs; /* serving: point x frequency work per step; 0 = tuned */
    int fold_kernel;            /* BLS_FOLD_*: which fold-sweep kernel runs the tiled search */
} bls_plan_desc;

/* One light curve and its trial-frequency grid. */
typedef struct {
    const double* t;      /* n times [d], any order; FP64 (host or device) */
    const float* y;       /* n fluxes */
    const float* dy;      /* n 1-sigma errors (> 0), or NULL for unit weights */
    int n;                /* number of points, >= 2 */
    const double* freqs;  /* nf trial frequencies [1/d] (> 0), or NULL for a uniform grid */
    int nf;               /* number of trial frequencies, >= 1 */
    double fmin, df;      /* uniform grid: f_j = fmin + j*df, each op rounded (freqs == NULL) */
    int nb;               /* phase bins for this curve; 0 = plan default */
    double qmin, qmax;    /* duration range for this curve; 0 = plan default */
} bls_curve;

/* One peak of one curve.  Reported values are recomputed in FP64 for the chosen box. */
typedef struct {
    int best_j;           /* frequency index of the peak, -1 for an empty slot */
    int i1, k;            /* first bin and width (bins) of the best box at that frequency */
    int pad_;
    double freq;          /* f [1/d] */
    double period;        /* 1/f [d] */
    double epoch;         /* mid-box time of the first eclipse after min(t) [d] */
    double duration;      /* k/(nb f) [d] */
    double depth;         /* -s/(r(1-r)): positive for a dip, in flux units */
    double snr;           /* depth / sigma_depth = SR sqrt(W) */
    double sr;            /* signal residue sqrt(P) */
    double power;         /* P = s^2/(r(1-r)) */
    double sde;           /* signal detection efficiency (SR - mean SR) / sd SR over the
                             curve's spectrum (Kovacs et al. 2002); 0 if the spectrum is flat */
} bls_peak;

typedef struct bls_plan bls_plan;

/* Create a plan on the current CUDA device.  cuda_stream (a cudaStream_t, may be NULL)
 * is the stream all work is ordered on; NULL makes the plan create its own.
 * Errors: BLS_ERR_INVALID (bad descriptor), BLS_ERR_CUDA (no device). */
bls_status bls_plan_create(const bls_plan_desc* desc, void* cuda_stream, bls_plan** out);

/* Release the plan, its device memory and its serving thread.  Pending requests are
 * cancelled.  NULL is ignored. */
void bls_plan_destroy(bls_plan* plan);

/* Batched search (Sec. 2.2.2): the periodogram of every curve, all frequencies, all box
 * starts and widths; out[c*topk + q] receives peak q of curve c (host memory).
 * spectrum (optional, host or device) receives SR(f_j) of every curve back to back
 * (sum of nf floats).  Blocks until the results are written.
 * When every input array and the spectrum are device or pinned host memory, a launch
 * group's stream work (copies, kernels, result copies) is captured into a CUDA graph,
 * and a later call whose group has the same layout (same pointers, sizes, options)
 * replays it with one launch; the arrays' contents may change between calls.  The
 * environment variable BLS_NO_GRAPHS=1, read at plan creation, turns this off.
 * Sizes, grids and widths are checked on the host before any work is queued; the values
 * (finite t and y, finite dy > 0, explicit frequencies > 0) are checked on the device on
 * the copies, for host and device inputs alike, and a bad value makes the call return
 * BLS_ERR_INVALID after the launch group ran (its outputs are then undefined).
 * BLS_ERR_INTERNAL: a device-side consistency check failed -- a bounded wait between the
 * warp groups of the hot kernel gave up (limit 30 s; the test setting BLS_HANDOFF_LIMIT_US,
 * in microseconds, read at every launch group, lowers it), or, in libbls_debug.so (the same
 * library with device-side checks on every histogram bin, shared-memory row and TMEM column
 * index, built beside libbls.so), an index check failed and the access was skipped.  The
 * plan stays usable after either.  Host-side NVTX ranges (bls.search, bls.prep,
 * bls.fold_sweep, bls.reduce, bls.server.step, bls.server.retire) mark the calls' phases.
 * Errors: BLS_ERR_INVALID, BLS_ERR_NOMEM, BLS_ERR_CUDA, BLS_ERR_INTERNAL. */
bls_status bls_search(bls_plan* plan, const bls_curve* curves, int ncurves,
                      bls_peak* out, float* spectrum);

/* Peak refinement (the search's follow-up step): for every peak q of every curve c in
 * coarse[c*topk + q] (as bls_search returned them for the same curves; best_j < 0 marks
 * an empty slot), searches the fine grid f_q + (i - half*oversample) * step,
 * i = 0 .. 2*half*oversample (each RN(f_q + RN(i' * step)), non-positive frequencies
 * dropped), step = RN(df / oversample) for a uniform grid, or for an explicit grid the
 * mean spacing of best_j's neighbours divided by oversample; out[c*topk + q] receives the
 * best peak of that fine grid (best_j indexes the fine grid, sde is over the fine grid;
 * empty slots get best_j = -1).  All arrays host memory except the curves' data, which
 * follow bls_search's rules.  Errors: as bls_search; BLS_ERR_INVALID for oversample < 1,
 * half < 1, or best_j outside a curve's grid. */
bls_status bls_refine(bls_plan* plan, const bls_curve* curves, int ncurves,
                      const bls_peak* coarse, int oversample, int half, bls_peak* out);

/* Trapezoid refit of the peaks (Sec. 5 of the paper names the eclipse duration and the
 * flat-bottomed shape as discriminators).  At a peak's frequency f the curve is folded
 * and a trapezoid -- centre c, total duration T, ingress tau, phase units -- is fitted to
 * the weighted, mean-subtracted flux x by least squares: with s the trapezoid's shape
 * (1 in the flat bottom, linear edges; tau = 0 is a box), Ss = sum w s, Sss = sum w s^2,
 * Sxs = sum w x s, the power is Q = Sxs^2 / (Sss - Ss^2) (a box gives the BLS power) and
 * the depth -Sxs / (Sss - Ss^2); only dips (Sxs < 0) count.  The grid is built around the
 * peak's box (centre phi_b = frac((i1 + k/2)/nb), width q = k/nb):
 *   c_m = phi_b + q (m/(ncentre-1) - 1/2), T_u = q (width_lo + u (width_hi - width_lo)/
 *   (nwidth-1)), tau_v = T_u ingress_max v/(ningress-1), flat index (m nwidth + u)
 *   ningress + v (a size of 1 takes the middle centre, the low width, no ingress). */
typedef struct {
    int ncentre, nwidth, ningress;   /* grid sizes >= 1; 0 = defaults 17, 13, 6 */
    double width_lo, width_hi;       /* widths in box widths, 0 < lo <= hi; 0 = 0.5, 2.0 */
    double ingress_max;              /* largest ingress / width, in [0, 0.5]; < 0 = 0.5 */
} bls_shape_grid;

typedef struct {
    int index;            /* best flat grid index, -1 if no trapezoid fits as a dip */
    int box_index;        /* best grid index among the boxes (tau = 0), -1 if none */
    double power;         /* Q of the best trapezoid (FP64 refit) */
    double box_power;     /* Q of the best box (FP64 refit) */
    double epoch;         /* mid-eclipse time t_ref + c/f */
    double duration;      /* total duration T/f */
    double ingress;       /* ingress duration tau/f (0 for a box) */
    double depth;         /* least-squares depth of the best trapezoid */
} bls_shape;

/* bls_search plus the trapezoid refit of every peak: shapes[c*topk + q] (host) belongs to
 * out[c*topk + q]; empty peak slots get index = box_index = -1.  grid may be NULL (all
 * defaults).  Errors: as bls_search; BLS_ERR_INVALID for a bad grid. */
bls_status bls_search_shapes(bls_plan* plan, const bls_curve* curves, int ncurves,
                             bls_peak* out, float* spectrum, const bls_shape_grid* grid,
                             bls_shape* shapes);

/* Serving: queue one curve.  The input is copied before the call returns; the call
 * never waits for the GPU.  Requests are admitted to the device as memory and slots
 * free up and share the GPU with requests already running (continuous batching).
 * Plans of the other algorithms (BLS_ALGO_PLAIN_F64, BLS_ALGO_UNBINNED) are served
 * sequentially through the same queue: one request at a time, oldest first, each run as
 * one search of one curve (a search error fails that request only).
 * *ticket identifies the request.  Errors: BLS_ERR_INVALID, BLS_ERR_NOMEM. */
bls_status bls_submit(bls_plan* plan, const bls_curve* curve, uint64_t* ticket);

/* Serving: wait up to timeout_ms (0 = just look, < 0 = forever) for a request.
 * BLS_OK: out[0..topk) holds its peaks and the ticket is retired.
 * BLS_PENDING (timeout_ms == 0) or BLS_ERR_TIMEOUT: not finished yet.
 * BLS_ERR_INVALID: unknown or retired ticket.  Other errors: the request failed. */
bls_status bls_poll(bls_plan* plan, uint64_t ticket, bls_peak* out, int timeout_ms);

/* Serving: cancel a queued or running request; a later poll returns BLS_ERR_CANCELLED. */
bls_status bls_cancel(bls_plan* plan, uint64_t ticket);

typedef struct {
    uint64_t submitted, completed, cancelled, failed;
    uint64_t steps;             /* scheduler steps run */
    uint64_t active;            /* requests resident on the device now */
    uint64_t queued;            /* requests waiting for admission */
    size_t device_bytes_in_use; /* request state on the device now */
    size_t device_bytes_peak;   /* highest value of the above */
    double p50_ms, p99_ms;      /* submit -> result latency over completed requests */
} bls_server_stats;

/* Serving statistics.  Errors: BLS_ERR_INVALID. */
bls_status bls_server_stats_get(bls_plan* plan, bls_server_stats* out);

/* Signal detection efficiency across frequency shards (the SDE of Kovacs, Zucker & Mazeh
 * 2002 that Sec. 2.2.2 cites: (SR_peak - mean SR) / sd SR over a curve's whole spectrum,
 * population sd).  When one curve's grid is searched in slices (one per GPU or per call),
 * each slice's SR spectrum is reduced to its moments, the moments are merged (Chan, Golub
 * and LeVeque's pairwise update), and the best peak's SDE is computed from the merged ones.
 * Host-side arithmetic in FP64. */
typedef struct {
    long long count;        /* number of SR values */
    double mean;            /* their mean */
    double m2;              /* sum of squared deviations from the mean */
} bls_moments;

/* Moments of sr[0..n) (host or device memory of the current device), two passes in FP64.
 * Errors: BLS_ERR_INVALID (NULL pointers, n < 0), BLS_ERR_CUDA, BLS_ERR_NOMEM. */
bls_status bls_moments_of(const float* sr, long long n, bls_moments* out);

/* Moments of the union of nparts disjoint parts.  Errors: BLS_ERR_INVALID. */
bls_status bls_moments_merge(const bls_moments* parts, int nparts, bls_moments* out);

/* SDE of a peak of signal residue sr against a spectrum's moments: 0 for a flat or empty
 * spectrum.  Errors: BLS_ERR_INVALID. */
bls_status bls_sde(double sr, const bls_moments* m, double* sde);

/* Box widths from the fractional duration range (reading of the paper's "range of
 * durations"): kmin = max(1, floor(qmin nb + 1e-9)), kmax = min(nb-1, ceil(qmax nb - 1e-9)).
 * Errors: BLS_ERR_INVALID. */
bls_status bls_kminmax(int nb, double qmin, double qmax, int* kmin, int* kmax);

/* Diagnostic: the phase bin of every point of one curve at frequencies js[0..nj), as
 * the search kernels compute them (plan's phase mode); bins_out[q*n + i] (host).  In the
 * FX64 mode on a uniform grid with fixed-point or FP32 sums the incremental fold of the search kernels
 * is evaluated too, for frequency js[q] at its place in a tile of the width the plan's
 * search uses for this curve (so with the search's reference column); a point where it
 * disagrees with the direct fold is reported as -1 - bin, so every value is a valid bin
 * exactly when both folds agree.  Errors: BLS_ERR_INVALID, BLS_ERR_CUDA. */
bls_status bls_debug_fold(bls_plan* plan, const bls_curve* curve, const int* js, int nj,
                          int* bins_out);

/* Diagnostic: the launch shape the plan's tiled search uses for curves of nb bins (0: the
 * plan's nb and widths) and the plan's duration range -- the plan's freqs_per_block and
 * point_chunk where given, else its rules: *cols trial frequencies per tile, *chunk points
 * per staged chunk, *ws = 1 for the warp-specialised fold-sweep kernel, 0 for the one-group
 * kernel.  Errors: BLS_ERR_INVALID (bad argument, an unbinned or baseline plan, nb outside
 * 2..4096, or no shape fits shared memory). */
bls_status bls_tile_shape(bls_plan* plan, int nb, int* cols, int* chunk, int* ws);

/* Diagnostic: the per-frequency best box of one curve as the search kernels leave it
 * before the peak reduction: power_out[j] (FP32 P), i1_out[j], k_out[j] (host).
 * Errors: as bls_search. */
bls_status bls_debug_powers(bls_plan* plan, const bls_curve* curve, float* power_out,
                            int* i1_out, int* k_out);

typedef struct {
    uint64_t searches;          /* launch groups run by bls_search since the last reset */
    uint64_t kernel_launches;   /* kernels those groups launched */
    uint64_t fold_launches;     /* of which fold-bin-sweep (or baseline) kernels */
    double prep_ms;             /* CUDA-event time of the prep kernels */
    double fold_ms;             /* CUDA-event time of the fold-bin-sweep kernels */
    double reduce_ms;           /* CUDA-event time of the peak reductions */
    uint64_t graph_captures;    /* groups captured into a CUDA graph (then launched) */
    uint64_t graph_replays;     /* groups run by replaying the previous group's graph */
} bls_profile;

/* Diagnostic: kernel timings of bls_search, measured with CUDA events recorded on the
 * plan's stream around each kernel phase; reset != 0 clears the counters after reading.
 * Errors: BLS_ERR_INVALID. */
bls_status bls_profile_get(bls_plan* plan, bls_profile* out, int reset);

/* Eclipse-window detection efficiency (Sec. 5 of the paper, detection-efficiency figure):
 * for every trial frequency f, the fraction of eclipse phases phi_m = (2m+1)/(2 nphi),
 * m < nphi, at which at least min_eclipses eclipses contain at least min_points
 * observations each.  Eclipse n of phase phi is centred at t_0 + (phi + n)/f; a time is
 * in it when it lies within half an eclipse duration of the centre.  Decisions are taken
 * in FP64: u = RN(RN(RN(t_i - t_0) f) - phi), c = floor(RN(u + 1/2)), in eclipse iff
 * |RN(u - c)| <= h with h = RN(RN(duration f) / 2), or RN(qfrac / 2) when duration == 0. */
typedef struct {
    const double* t;      /* observation times, sorted ascending (host or device) */
    int n;                /* >= 1 */
    const double* freqs;  /* explicit frequencies > 0 (host or device), or NULL: uniform grid */
    int nf;               /* >= 1 */
    double fmin, df;      /* uniform grid f_k = RN(fmin + RN(k df)) when freqs is NULL */
    int nphi;             /* eclipse phases per frequency, >= 1 */
    double duration;      /* eclipse duration in time units (> 0), or 0: use qfrac */
    double qfrac;         /* eclipse duration as a fraction of the period, 0 < qfrac < 1 */
    int min_eclipses;     /* observed eclipses needed for a detection (the paper: 2) */
    int min_points;       /* observations an eclipse needs to count as observed, >= 1 */
} bls_window_desc;

/* eff[k] (nf doubles) receives the efficiency at frequency k; counts (optional, nf * nphi
 * ints, frequency-major) the observed eclipses of every (frequency, phase).  Outputs may
 * be host or device memory; work is ordered on cuda_stream (NULL: the legacy default
 * stream) and the call returns when the results are written.  Allocates its scratch with
 * cudaMallocAsync on that stream.  Errors: BLS_ERR_INVALID (bad descriptor; times not
 * sorted or not finite, frequencies <= 0: device check), BLS_ERR_NOMEM, BLS_ERR_CUDA. */
bls_status bls_window_efficiency(const bls_window_desc* desc, void* cuda_stream, double* eff,
                                 int* counts);

/* High-variability pre-filter (Sec. 2.2.1 of the paper): stars whose photometric
 * variability lies more than nsig standard deviations above the expectation for their
 * magnitude -- estimated per 0.1-mag bin from a sigma-clipped average over the stars of
 * their chip -- are flagged.  Per star, from its light curve in magnitudes: mag = mean,
 * rms = population RMS, bin = floor(RN(mag * 10)).  Per (chip, bin), over the rms of its
 * stars in star order: mu and sd (population) of the kept values, keep |rms - mu| <=
 * clip * sd, at most `iters` rounds, stop when the kept set no longer changes; a star is
 * flagged when its bin has at least min_stars stars and rms > mu + nsig * sd.  All sums
 * are FP64 in a fixed order (a warp's partial sums and butterfly; the paper gives none),
 * so results are deterministic and within the FP64 summation bound, (n - 1) 2^-53 sum |v|
 * per sum, of plain sequential sums; a decision can differ from the sequential order's
 * only for a value within that bound of its threshold. */
typedef struct {
    const long long* off;   /* nstars + 1 offsets into m (host or device) */
    const float* m;         /* magnitudes of all light curves, concatenated (host or device) */
    const int* chip;        /* chip of every star, 0 .. nchips-1 (host or device) */
    int nstars, nchips;     /* >= 1 each */
    double clip;            /* clipping threshold, in sd (> 0; 3 is the usual choice) */
    int iters;              /* clipping rounds (>= 0) */
    double nsig;            /* flag threshold above the expectation, in sd (the paper: 2) */
    int min_stars;          /* bins with fewer stars flag nothing (>= 1) */
} bls_var_desc;

typedef struct {
    double mag, rms;        /* mean magnitude and RMS of the star's light curve */
    double mu, sd;          /* sigma-clipped expectation of its (chip, bin) */
    int bin;                /* floor(mag * 10) */
    unsigned char flag;     /* 1: more variable than nsig sd above the expectation */
    unsigned char pad_[3];
} bls_var_star;

/* out: nstars records (host or device).  Work is ordered on cuda_stream (NULL: legacy
 * default stream); returns when the results are written; scratch from cudaMallocAsync on
 * that stream.  Errors: BLS_ERR_INVALID (bad descriptor; empty or non-finite light curves,
 * chip ids out of range, or one chip spanning more than 4096 bins: device check),
 * BLS_ERR_NOMEM, BLS_ERR_CUDA. */
bls_status bls_variability(const bls_var_desc* desc, void* cuda_stream, bls_var_star* out);

/* Search of one curve that allocates nothing.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc (a plug-in whose host application
 * owns and budgets all device memory, a latency-critical loop that cannot take
 * cudaMalloc's implicit device synchronisation, a process under a memory cap).
 *   curve      t, y, dy (optional), freqs (optional) in device memory; nb >= 2 and
 *              0 < qmin <= qmax < 1 must be given (there is no plan to default from).
 *   topk, sign as in bls_plan_desc (dips only or both signs; FP32 sums, fixed-point fold).
 *   cuda_stream stream the work is ordered on (NULL: the legacy default stream).
 *   peaks_dev  device memory for topk bls_peak records, filled as bls_search fills `out`.
 *   spectrum_dev optional device memory for nf floats, SR(f_j) as bls_search writes it.
 * All intermediate data lives in one static device array of 32 MiB per device, which every
 * GPU that loads this library holds until the process exits; curves needing more
 * (about 24 bytes per point plus 4 per frequency) are rejected with BLS_ERR_INVALID.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it.  Every call shares the
 * array and leaves its contents behind, so calls that overlap on the GPU (other threads,
 * other streams) race: serialise them.  Blocks until the results are written.
 * Errors: BLS_ERR_INVALID (bad argument, host memory given, too large, bad input values),
 * BLS_ERR_CUDA. */
bls_status bls_search_static(const bls_curve* curve, int topk, int sign, void* cuda_stream,
                             bls_peak* peaks_dev, float* spectrum_dev);

/* Thread-local message of the last failure on the calling thread ("" if none). */
const char* bls_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BLS_H */

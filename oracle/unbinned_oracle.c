/*
 * unbinned_oracle.c -- plain unbinned (edge-to-edge) BLS periodogram.
 *
 * TEST INFRASTRUCTURE, like bls_oracle.c: only the tests, the smoke check and the
 * benchmark's CPU legs load it; it shares nothing with the CUDA library.
 *
 * What it computes.  The BLS family the paper uses (Sec. 2.2.2: Kovacs, Zucker & Mazeh
 * 2002; Tingley 2003) also has an unbinned form in which the box edges sit on data points
 * instead of bin edges: at each trial frequency the points are ordered by phase and every
 * cyclic run of consecutive points whose phase extent lies in [qmin, qmax] is a box.  The
 * statistic is the binned one (w, x, r = sum_B w, s = sum_B w x, P = s^2/(r(1-r)), dips only
 * by default).  Readings (R):
 *
 *   phase (R: the 64-bit fixed-point phase, so that the ordering and the extents -- integer
 *   decisions -- are exact and the same on every implementation):
 *     L = ilogb(dtmax) + 1 (0 if dtmax = 0), s = 34 - (L+1)/2 (C division), s <= 62 - L, s >= 1
 *     DT_i = RN_int(dt_i 2^s), F = RN_int(f 2^(64-s)),  key_i = ((DT_i F) mod 2^64) >> 32
 *   order: by (key, point index) ascending; positions p = 0..n-1
 *   run (a, len): positions a, a+1, ..., a+len-1 (mod n), 1 <= len <= n-1,
 *     extent E = (key[last] - key[first]) mod 2^32,
 *     a box iff  QMIN <= E <= QMAX,  QMIN = ceil(qmin 2^32), QMAX = floor(qmax 2^32)
 *   r, s summed in run order (FP64, plain); power as in the binned search, skipping boxes
 *   with r <= 0 or r >= 1 (R: always true here, but kept for rounding)
 *   best per frequency: largest P; ties to the smaller (a, len) in that order
 *   epoch = t_ref + frac((key_first + E/2) / 2^32) / f, duration = E / 2^32 / f
 *
 * FP64 round-to-nearest, no contraction; 64-bit unsigned arithmetic wraps.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int j;              /* frequency index */
    int first, len;     /* run: first position in phase order, number of points */
    int first_point;    /* original index of the run's first point */
    double freq, power, sr, depth, epoch, duration, snr;
} oracle_ubls_peak;

int oracle_fx_shift(double dtmax)
{
    int L = 0;
    if (dtmax > 0.0) L = ilogb(dtmax) + 1;
    int s = 34 - (L + 1) / 2;
    if (s > 62 - L) s = 62 - L;
    return s < 1 ? 1 : s;
}

static uint64_t rn_u64(double v)
{
    return (uint64_t)nearbyint(v);
}

/* phase keys of all points at frequency f */
void oracle_ubls_keys(int n, const double* dt, double dtmax, double f, uint32_t* key)
{
    int s = oracle_fx_shift(dtmax);
    uint64_t F = rn_u64(ldexp(f, 64 - s));
    for (int i = 0; i < n; ++i) {
        uint64_t DT = rn_u64(ldexp(dt[i], s));
        key[i] = (uint32_t)((DT * F) >> 32);
    }
}

static const uint32_t* g_key;   /* sort context (single-threaded oracle) */

static int cmp_pos(const void* pa, const void* pb)
{
    int a = *(const int*)pa, b = *(const int*)pb;
    if (g_key[a] != g_key[b]) return g_key[a] < g_key[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/*
 * Best box of one frequency.  dt, w, x from the prep (oracle_prep); returns P (0 if no box
 * counts) and the run (first position, len) through the pointers; order (optional, n)
 * receives the phase order.
 */
double oracle_ubls_power(int n, const double* dt, const double* w, const double* x, double dtmax,
                         double f, double qmin, double qmax, int sign, int* first, int* len,
                         double* r_out, double* s_out, int* order)
{
    uint32_t* key = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    int* ord = (int*)malloc(sizeof(int) * (size_t)n);
    oracle_ubls_keys(n, dt, dtmax, f, key);
    for (int i = 0; i < n; ++i) ord[i] = i;
    g_key = key;
    qsort(ord, (size_t)n, sizeof(int), cmp_pos);
    const uint64_t two32 = 4294967296ull;
    uint64_t QMIN = (uint64_t)ceil(qmin * 4294967296.0);
    uint64_t QMAX = (uint64_t)floor(qmax * 4294967296.0);
    if (QMAX >= two32) QMAX = two32 - 1;
    double best = 0.0;
    int bf = 0, bl = 0;
    double br = 0.0, bs = 0.0;
    for (int a = 0; a < n; ++a) {
        double r = 0.0, s = 0.0;
        uint32_t k0 = key[ord[a]];
        for (int l = 1; l <= n - 1; ++l) {
            int p = ord[(a + l - 1) % n];
            uint32_t E = key[p] - k0;   /* mod 2^32 */
            if ((uint64_t)E > QMAX) break;
            r += w[p];
            s += w[p] * x[p];
            if ((uint64_t)E < QMIN) continue;
            if (!(r > 0.0 && r < 1.0)) continue;
            if (!sign && !(s < 0.0)) continue;
            double P = s * s / (r * (1.0 - r));
            if (P > best) { best = P; bf = a; bl = l; br = r; bs = s; }
        }
    }
    *first = bf;
    *len = bl;
    if (r_out) *r_out = br;
    if (s_out) *s_out = bs;
    if (order) memcpy(order, ord, sizeof(int) * (size_t)n);
    free(key);
    free(ord);
    return best;
}

/*
 * Periodogram over nf frequencies (explicit or f_j = RN(fmin + RN(j df))): P[j] and the
 * best peak.  t, y, dy as for oracle_prep (dy may be NULL).  Returns 0 or a negative code.
 */
int oracle_prep(int n, const double* t, const float* y, const float* dy, double* dt, double* w,
                double* x, double* scal);

int oracle_ubls(int n, const double* t, const float* y, const float* dy, int nf,
                const double* freqs, double fmin, double df, double qmin, double qmax, int sign,
                double* P, oracle_ubls_peak* peak)
{
    if (n < 2 || nf < 1 || !(qmax > 0.0 && qmax < 1.0) || !(qmin >= 0.0 && qmin <= qmax)) return -1;
    double* dt = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* w = dt + n;
    double* x = w + n;
    double scal[4];
    int rc = oracle_prep(n, t, y, dy, dt, w, x, scal);
    if (rc) { free(dt); return rc; }
    double dtmax = 0.0;
    for (int i = 0; i < n; ++i) if (dt[i] > dtmax) dtmax = dt[i];
    int* ord = (int*)malloc(sizeof(int) * (size_t)n);
    memset(peak, 0, sizeof(*peak));
    peak->j = -1;
    double bestP = -1.0;
    for (int j = 0; j < nf; ++j) {
        double f = freqs ? freqs[j] : fmin + (double)j * df;
        int a, l;
        double r, s;
        double Pj = oracle_ubls_power(n, dt, w, x, dtmax, f, qmin, qmax, sign, &a, &l, &r, &s, ord);
        if (P) P[j] = Pj;
        if (Pj > bestP) {
            bestP = Pj;
            uint32_t* key = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
            oracle_ubls_keys(n, dt, dtmax, f, key);
            uint32_t k0 = key[ord[a]], E = key[ord[(a + l - 1) % n]] - k0;
            peak->j = j;
            peak->first = a;
            peak->len = l;
            peak->first_point = ord[a];
            peak->freq = f;
            peak->power = Pj;
            if (Pj > 0.0) {
                peak->sr = sqrt(Pj);
                peak->depth = -s / (r * (1.0 - r));
                peak->snr = peak->sr * sqrt(scal[1]);
            } else {
                peak->sr = 0.0; peak->depth = 0.0; peak->snr = 0.0;
            }
            double mid = ((double)k0 + 0.5 * (double)E) / 4294967296.0;
            mid = mid - floor(mid);
            peak->epoch = scal[0] + mid / f;
            peak->duration = (double)E / 4294967296.0 / f;
            free(key);
        }
    }
    free(ord);
    free(dt);
    return 0;
}

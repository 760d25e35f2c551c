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
 *   phase (R: the binned search's FP64 fold):  p = RN(dt_i f),  phi_i = p - floor(p)
 *   order: by (phi, point index) ascending; positions 0..n-1
 *   run (a, len): positions a, a+1, ..., a+len-1 (mod n), 1 <= len <= n-1; with first and
 *     last its first and last points,
 *       d = RN(phi_last - phi_first),  extent E = d, or RN(d + 1) if the run passes
 *       position n-1 (it wraps through phase 0),
 *     a box iff  qmin <= E <= qmax
 *   r, s summed in run order (FP64, plain); power as in the binned search, skipping boxes
 *   with r <= 0 or r >= 1 (R: never true here, but kept for rounding)
 *   best per frequency: largest P; ties to the smaller (a, len) in that order
 *   epoch = t_ref + m / f with m = frac(RN(phi_first + RN(E / 2))),  duration = E / f
 *
 * E grows with the run's length from a fixed start (each step adds a non-negative phase
 * difference, and the first wrapped extent RN(RN(phi_0 - phi_a) + 1) is at least
 * RN(1 - phi_a), the largest unwrapped one can reach), so a scan over lengths may stop at
 * the first extent above qmax.
 *
 * FP64 round-to-nearest, no contraction.
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

/* phases of all points at frequency f */
void oracle_ubls_phases(int n, const double* dt, double f, double* phi)
{
    for (int i = 0; i < n; ++i) {
        double p = dt[i] * f;
        phi[i] = p - floor(p);
    }
}

static const double* g_phi;   /* sort context (single-threaded oracle) */

static int cmp_pos(const void* pa, const void* pb)
{
    int a = *(const int*)pa, b = *(const int*)pb;
    if (g_phi[a] != g_phi[b]) return g_phi[a] < g_phi[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/* points in phase order: ord[q] is the point at position q */
void oracle_ubls_order(int n, const double* phi, int* ord)
{
    for (int i = 0; i < n; ++i) ord[i] = i;
    g_phi = phi;
    qsort(ord, (size_t)n, sizeof(int), cmp_pos);
}

/* extent of the run from position a to position a + len - 1 (mod n) */
double oracle_ubls_extent(int n, const double* phi, const int* ord, int a, int len)
{
    int e = a + len - 1;
    double d = phi[ord[e % n]] - phi[ord[a]];
    return e >= n ? d + 1.0 : d;
}

/*
 * Best box of one frequency.  dt, w, x from the prep (oracle_prep); returns P (0 if no box
 * counts) and the run (first position, len) through the pointers; order (optional, n)
 * receives the phase order.
 */
double oracle_ubls_power(int n, const double* dt, const double* w, const double* x, double f,
                         double qmin, double qmax, int sign, int* first, int* len,
                         double* r_out, double* s_out, int* order)
{
    double* phi = (double*)malloc(sizeof(double) * (size_t)n);
    int* ord = (int*)malloc(sizeof(int) * (size_t)n);
    oracle_ubls_phases(n, dt, f, phi);
    oracle_ubls_order(n, phi, ord);
    double best = 0.0;
    int bf = 0, bl = 0;
    double br = 0.0, bs = 0.0;
    for (int a = 0; a < n; ++a) {
        double r = 0.0, s = 0.0;
        for (int l = 1; l <= n - 1; ++l) {
            double E = oracle_ubls_extent(n, phi, ord, a, l);
            if (E > qmax) break;
            int p = ord[(a + l - 1) % n];
            r += w[p];
            s += w[p] * x[p];
            if (E < qmin) continue;
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
    free(phi);
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
    double* dt = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    double* w = dt + n;
    double* x = w + n;
    double* phi = x + n;
    double scal[4];
    int rc = oracle_prep(n, t, y, dy, dt, w, x, scal);
    if (rc) { free(dt); return rc; }
    int* ord = (int*)malloc(sizeof(int) * (size_t)n);
    memset(peak, 0, sizeof(*peak));
    peak->j = -1;
    double bestP = -1.0;
    for (int j = 0; j < nf; ++j) {
        double f = freqs ? freqs[j] : fmin + (double)j * df;
        int a, l;
        double r, s;
        double Pj = oracle_ubls_power(n, dt, w, x, f, qmin, qmax, sign, &a, &l, &r, &s, ord);
        if (P) P[j] = Pj;
        if (Pj > bestP) {
            bestP = Pj;
            oracle_ubls_phases(n, dt, f, phi);
            double E = l > 0 ? oracle_ubls_extent(n, phi, ord, a, l) : 0.0;
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
            double mid = phi[ord[a]] + 0.5 * E;
            mid = mid - floor(mid);
            peak->epoch = scal[0] + mid / f;
            peak->duration = E / f;
        }
    }
    free(ord);
    free(dt);
    return 0;
}

/*
 * window_oracle.c -- plain FP64 eclipse-window detection efficiency.
 *
 * TEST INFRASTRUCTURE, like bls_oracle.c: only the tests, the smoke check and the
 * benchmark's CPU legs load it; it shares nothing with the CUDA library.
 *
 * What it computes.  The discussion of the paper (Sec. 5 and its detection-efficiency figure)
 * defines the survey's eclipse detection efficiency at a given period as the probability
 * that at least two eclipses of an eclipsing target are observed once the observing
 * windows and the weather are taken into account.  For a set of observation times t_i,
 * a trial frequency f = 1/P and an eclipse phase phi (eclipse centres at
 * t_ref + (phi + n) P, n integer), an observation lies in eclipse n when it is within half
 * an eclipse duration of that centre.  An eclipse counts as observed when at least
 * min_points observations lie in it; the target is detected when at least min_eclipses
 * eclipses are observed.  The efficiency at f is the fraction of the nphi phases
 * phi_m = (m + 1/2)/nphi (a uniform grid over the unknown eclipse phase) at which the
 * target is detected.
 *
 * Arithmetic, in this order, IEEE FP64 round-to-nearest, no fused multiply-add
 * (compiled with -ffp-contract=off):
 *   t_ref = t_0 (times sorted ascending), dt_i = t_i - t_ref
 *   v   = dt_i * f                     (phase in cycles)
 *   u   = v - phi_m                    (cycles since the eclipse of cycle 0)
 *   n   = floor(u + 0.5)               (nearest eclipse)
 *   r   = u - n                        (offset from its centre, cycles)
 *   in eclipse  <=>  |r| <= h,  h = (duration * f) * 0.5, or qfrac * 0.5 when the
 *                                   duration is given as a fraction of the period
 *   phi_m = (2m + 1) / (2 nphi)
 * Times sorted ascending make n non-decreasing along the points, so the observed eclipses
 * are counted in one pass.
 */
#include <math.h>
#include <stddef.h>

/* Frequency k of a uniform grid, evaluated as RN(fmin + RN(k df)). */
static double grid_f(const double* freqs, double fmin, double df, int k)
{
    if (freqs) return freqs[k];
    double kd = (double)k * df;
    return fmin + kd;
}

/*
 * Observed eclipses of one (frequency, phase) pair.
 */
int oracle_window_count(int n, const double* t, double f, double phi, double h, int min_points)
{
    int eclipses = 0, have = 0, in_cur = 0;
    double cur = 0.0;
    for (int i = 0; i < n; ++i) {
        double dt = t[i] - t[0];
        double v = dt * f;
        double u = v - phi;
        double c = floor(u + 0.5);
        double r = u - c;
        if (fabs(r) <= h) {
            if (!have || c != cur) {
                if (have && in_cur >= min_points) eclipses++;
                cur = c;
                have = 1;
                in_cur = 0;
            }
            in_cur++;
        }
    }
    if (have && in_cur >= min_points) eclipses++;
    return eclipses;
}

/*
 * Efficiency at every frequency; counts (optional, nf * nphi, frequency-major) receives
 * the observed eclipses of every (frequency, phase) pair.  Returns 0, or -1 on bad
 * arguments (n < 1, nf < 1, nphi < 1, times not sorted or not finite, bad duration).
 */
int oracle_window(int n, const double* t, int nf, const double* freqs, double fmin, double df,
                  int nphi, double duration, double qfrac, int min_eclipses, int min_points,
                  double* eff, int* counts)
{
    if (n < 1 || nf < 1 || nphi < 1 || min_points < 1 || min_eclipses < 0) return -1;
    if (!(duration > 0.0) && !(qfrac > 0.0 && qfrac < 1.0)) return -1;
    for (int i = 0; i < n; ++i) {
        if (!isfinite(t[i])) return -1;
        if (i > 0 && t[i] < t[i - 1]) return -1;
    }
    for (int k = 0; k < nf; ++k) {
        double f = grid_f(freqs, fmin, df, k);
        double h = duration > 0.0 ? (duration * f) * 0.5 : qfrac * 0.5;
        int det = 0;
        for (int m = 0; m < nphi; ++m) {
            double phi = (double)(2 * m + 1) / (double)(2 * nphi);
            int c = oracle_window_count(n, t, f, phi, h, min_points);
            if (counts) counts[(size_t)k * nphi + m] = c;
            if (c >= min_eclipses) det++;
        }
        eff[k] = (double)det / (double)nphi;
    }
    return 0;
}

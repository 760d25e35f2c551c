/*
 * variability_oracle.c -- plain FP64 high-variability pre-filter.
 *
 * TEST INFRASTRUCTURE, like bls_oracle.c: only the tests, the smoke check and the
 * benchmark's CPU legs load it; it shares nothing with the CUDA library.
 *
 * What it computes.  Sec. 2.2.1 of the paper flags eclipsing binaries with deep, long
 * eclipses by their excess photometric variability: the expected stability and its
 * scatter are estimated as a function of magnitude in 0.1-mag bins from a sigma-clipped
 * average over the stars of each chip, and stars more than 2 sigma above that
 * expectation are flagged.  Restated (readings marked R):
 *
 *   star s with magnitudes m_1..m_n (R: its light curve in magnitudes):
 *     mag_s = (1/n) sum m_i                          (R: mean magnitude)
 *     rms_s = sqrt((1/n) sum (m_i - mag_s)^2)        (R: stability = population RMS)
 *   bin of a star: b = floor(RN(mag_s * 10))          (0.1-mag bins on a fixed grid)
 *   per (chip, bin), over the rms of its stars, sigma clipping (R: 3 sigma, at most
 *   `iters` rounds, stop when the kept set no longer changes):
 *     mu = mean of the kept, sd = population sd of the kept,
 *     keep the values with |rms - mu| <= clip * sd
 *   the bin's expectation is (mu, sd) of the final kept set (computed from it after the
 *   last round);  star flagged  <=>  rms_s > mu + nsig * sd  (the paper: nsig = 2), and
 *   never in a bin with fewer than min_stars stars (R: too few to estimate a scatter).
 *
 * Summation order (R: the paper gives none): every sum is the plain one, values added one
 * at a time in their index order (points in light-curve order, stars in catalog order),
 * IEEE FP64 round-to-nearest, no contraction.  Another order (a GPU's tree of partial
 * sums) gives sums that differ from these by at most the FP64 summation bound
 * (n - 1) 2^-53 sum |v|, which is what parity with them is measured against.
 *
 * Diagnostic output (for tests only): the clip margin of a (chip, bin) group, the
 * smallest | |rms - mu| - clip sd | over every keep-or-drop decision of every clipping
 * round.  A decision whose margin is below the rounding error of its operands may go
 * either way in another summation order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Plain sum of v[0..k) in index order. */
static double sum_seq(int k, const double* v)
{
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += v[i];
    return s;
}

/* mean and population RMS of one light curve (two passes) */
void oracle_star_stats(int n, const float* m, double* mag, double* rms)
{
    double* v = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int i = 0; i < n; ++i) v[i] = (double)m[i];
    double mu = sum_seq(n, v) / (double)n;
    for (int i = 0; i < n; ++i) {
        double d = (double)m[i] - mu;
        v[i] = d * d;
    }
    *mag = mu;
    *rms = sqrt(sum_seq(n, v) / (double)n);
    free(v);
}

/*
 * Sigma-clipped (mu, sd) of vals[0..k); returns the number kept.  Each round takes the mean
 * and the population sd of the values kept so far (plain sums over them, in index order),
 * then keeps exactly the values with |v - mu| <= clip sd; it stops after `iters` rounds or
 * when the kept set no longer changes, and (mu, sd) are those of the final kept set.
 * margin (optional): the smallest | |v - mu| - clip sd | over every decision taken.
 */
int oracle_clip(int k, const double* vals, double clip, int iters, double* mu_out, double* sd_out,
                double* margin)
{
    char* keep = (char*)malloc((size_t)(k > 0 ? k : 1));
    double* t = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int i = 0; i < k; ++i) keep[i] = 1;
    double mu = 0.0, sd = 0.0, mg = INFINITY;
    int kept = k;
    for (int it = 0; it <= iters; ++it) {
        int c = 0;
        for (int i = 0; i < k; ++i) if (keep[i]) t[c++] = vals[i];
        mu = c > 0 ? sum_seq(c, t) / (double)c : 0.0;
        c = 0;
        for (int i = 0; i < k; ++i)
            if (keep[i]) { double d = vals[i] - mu; t[c++] = d * d; }
        sd = c > 0 ? sqrt(sum_seq(c, t) / (double)c) : 0.0;
        kept = c;
        if (it == iters) break;
        int changed = 0;
        for (int i = 0; i < k; ++i) {
            double a = fabs(vals[i] - mu), lim = clip * sd;
            double gap = fabs(a - lim);
            if (gap < mg) mg = gap;
            char nk = a <= lim;
            if (nk != keep[i]) { keep[i] = nk; changed = 1; }
        }
        if (!changed) break;
    }
    free(keep);
    free(t);
    *mu_out = mu;
    *sd_out = sd;
    if (margin) *margin = mg;
    return kept;
}

/*
 * Flags for nstars stars: light curve s is m[off[s] .. off[s+1]) (magnitudes), chip[s]
 * its chip (0 .. nchips-1).  Outputs per star (any may be NULL except flag): mag, rms,
 * bin, the bin's mu and sd, flag (0/1), and the clip margin of the star's group.
 * Returns 0, or -1 on bad arguments.
 */
int oracle_variability(int nstars, const long long* off, const float* m, const int* chip,
                       int nchips, double clip, int iters, double nsig, int min_stars,
                       double* mag, double* rms, int* bin, double* mu, double* sd,
                       unsigned char* flag, double* margin)
{
    if (nstars < 0 || nchips < 1 || !(clip > 0.0) || iters < 0 || !(nsig >= 0.0) || min_stars < 1)
        return -1;
    double* mg = (double*)malloc(sizeof(double) * (size_t)(nstars + 1));
    double* rm = (double*)malloc(sizeof(double) * (size_t)(nstars + 1));
    int* bn = (int*)malloc(sizeof(int) * (size_t)(nstars + 1));
    double* vals = (double*)malloc(sizeof(double) * (size_t)(nstars + 1));
    int* members = (int*)malloc(sizeof(int) * (size_t)(nstars + 1));
    for (int s = 0; s < nstars; ++s) {
        long long n = off[s + 1] - off[s];
        if (n < 1 || chip[s] < 0 || chip[s] >= nchips) { free(mg); free(rm); free(bn); free(vals); free(members); return -1; }
        oracle_star_stats((int)n, m + off[s], &mg[s], &rm[s]);
        bn[s] = (int)floor(mg[s] * 10.0);
    }
    char* done = (char*)calloc((size_t)(nstars + 1), 1);
    for (int s = 0; s < nstars; ++s) {
        if (done[s]) continue;
        /* the (chip, bin) group of star s, in star order */
        int k = 0;
        for (int u = s; u < nstars; ++u)
            if (!done[u] && chip[u] == chip[s] && bn[u] == bn[s]) { members[k] = u; vals[k] = rm[u]; k++; }
        double bmu, bsd, bmg;
        oracle_clip(k, vals, clip, iters, &bmu, &bsd, &bmg);
        for (int q = 0; q < k; ++q) {
            int u = members[q];
            done[u] = 1;
            if (mag) mag[u] = mg[u];
            if (rms) rms[u] = rm[u];
            if (bin) bin[u] = bn[u];
            if (mu) mu[u] = bmu;
            if (sd) sd[u] = bsd;
            if (margin) margin[u] = bmg;
            flag[u] = (unsigned char)(k >= min_stars && rm[u] > bmu + nsig * bsd);
        }
    }
    free(done); free(mg); free(rm); free(bn); free(vals); free(members);
    return 0;
}

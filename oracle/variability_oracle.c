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
 * Summation order (R: the paper gives none; this one is plain and runs as well on 32 SIMD
 * lanes): every sum of values v_0..v_{k-1} is taken as 32 interleaved partial sums,
 * lane l adding v_l, v_{l+32}, ... in order, then combined pairwise in a butterfly:
 * for o = 16, 8, 4, 2, 1, every lane l adds lane (l xor o)'s value to its own (the two
 * operands in the order own + other).  IEEE FP64 round-to-nearest, no contraction.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Sum in the order stated above: 32 interleaved partial sums, then the butterfly. */
static double sum32(int k, const double* v)
{
    double lane[32];
    for (int l = 0; l < 32; ++l) {
        lane[l] = 0.0;
        for (int i = l; i < k; i += 32) lane[l] += v[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        double nxt[32];
        for (int l = 0; l < 32; ++l) nxt[l] = lane[l] + lane[l ^ o];
        for (int l = 0; l < 32; ++l) lane[l] = nxt[l];
    }
    return lane[0];
}

/* mean and population RMS of one light curve (two passes) */
void oracle_star_stats(int n, const float* m, double* mag, double* rms)
{
    double* v = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int i = 0; i < n; ++i) v[i] = (double)m[i];
    double mu = sum32(n, v) / (double)n;
    for (int i = 0; i < n; ++i) {
        double d = (double)m[i] - mu;
        v[i] = d * d;
    }
    *mag = mu;
    *rms = sqrt(sum32(n, v) / (double)n);
    free(v);
}

/* sigma-clipped (mu, sd) of vals[0..k); returns the number kept */
int oracle_clip(int k, const double* vals, double clip, int iters, double* mu_out, double* sd_out)
{
    char* keep = (char*)malloc((size_t)(k > 0 ? k : 1));
    double* t = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int i = 0; i < k; ++i) keep[i] = 1;
    double mu = 0.0, sd = 0.0;
    int kept = k;
    for (int it = 0; it <= iters; ++it) {
        /* sums over the kept values, the dropped ones counting as zero in their places */
        int c = 0;
        for (int i = 0; i < k; ++i) { t[i] = keep[i] ? vals[i] : 0.0; c += keep[i]; }
        mu = c > 0 ? sum32(k, t) / (double)c : 0.0;
        for (int i = 0; i < k; ++i) {
            double d = vals[i] - mu;
            t[i] = keep[i] ? d * d : 0.0;
        }
        sd = c > 0 ? sqrt(sum32(k, t) / (double)c) : 0.0;
        kept = c;
        if (it == iters) break;
        int changed = 0;
        for (int i = 0; i < k; ++i) {
            char nk = fabs(vals[i] - mu) <= clip * sd;
            if (nk != keep[i]) { keep[i] = nk; changed = 1; }
        }
        if (!changed) break;
    }
    free(keep);
    free(t);
    *mu_out = mu;
    *sd_out = sd;
    return kept;
}

/*
 * Flags for nstars stars: light curve s is m[off[s] .. off[s+1]) (magnitudes), chip[s]
 * its chip (0 .. nchips-1).  Outputs per star (any may be NULL except flag): mag, rms,
 * bin, the bin's mu and sd, flag (0/1).  Returns 0, or -1 on bad arguments.
 */
int oracle_variability(int nstars, const long long* off, const float* m, const int* chip,
                       int nchips, double clip, int iters, double nsig, int min_stars,
                       double* mag, double* rms, int* bin, double* mu, double* sd,
                       unsigned char* flag)
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
        double bmu, bsd;
        oracle_clip(k, vals, clip, iters, &bmu, &bsd);
        for (int q = 0; q < k; ++q) {
            int u = members[q];
            done[u] = 1;
            if (mag) mag[u] = mg[u];
            if (rms) rms[u] = rm[u];
            if (bin) bin[u] = bn[u];
            if (mu) mu[u] = bmu;
            if (sd) sd[u] = bsd;
            flag[u] = (unsigned char)(k >= min_stars && rm[u] > bmu + nsig * bsd);
        }
    }
    free(done); free(mg); free(rm); free(bn); free(vals); free(members);
    return 0;
}

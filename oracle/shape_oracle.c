/*
 * shape_oracle.c -- plain FP64 trapezoid refit of a BLS peak.
 *
 * TEST INFRASTRUCTURE, like bls_oracle.c: only the tests, the smoke check and the
 * benchmark's CPU legs load it; it shares nothing with the CUDA library.
 *
 * What it computes.  The paper's discussion (Sec. 5) lists the eclipse duration and the
 * eclipse shape -- exactly flat-bottomed between short ingress and egress for a white
 * dwarf behind an M dwarf, rounder for a planet -- as the first discriminators that need
 * only the discovery light curve.  At a peak's frequency f the curve is folded,
 * phi_i = frac(RN(dt_i f)), and a trapezoid is fitted to the weighted, mean-subtracted
 * flux by least squares:
 *
 *   shape s(phi) with centre c, total duration T and ingress tau (phase units):
 *     D = phi - c wrapped to [-1/2, 1/2) (D = u - floor(u + 1/2), u = phi - c);
 *     tau > 0:  s = min(1, max(0, (T/2 - |D|) / tau))    (flat bottom, linear edges)
 *     tau = 0:  s = 1 if |D| < T/2, else 0                (a box)
 *   model x_i = alpha - delta s_i, weights w_i (sum 1), x = y - ybar (sum w x = 0):
 *     Ss = sum w s, Sss = sum w s^2, Sxs = sum w x s
 *     delta = -Sxs / (Sss - Ss^2),  chi2_min = sum w x^2 - Sxs^2 / (Sss - Ss^2)
 *     power  Q = Sxs^2 / (Sss - Ss^2)   (for a box: s^2 / (r(1-r)), the BLS power)
 *
 * over a grid around the peak's box (centre phi_b = frac((i1 + k/2)/nb), width q = k/nb):
 *   c_m   = phi_b + q (m/(nc-1) - 1/2),                    m < nc
 *   T_u   = q (wlo + u (whi - wlo)/(nw-1)),                 u < nw
 *   tau_v = T_u * amax * v/(na-1)  (v = 0 is the box),     v < na
 * (for nc, nw or na equal to 1 the single value is the middle/low end: m/(nc-1) -> 1/2,
 * u -> 0, v -> 0).  Dips only: a grid point counts when Sxs < 0 and Sss - Ss^2 > 0.  The
 * best point has the largest Q, ties to the smallest flat index (m nw + u) na + v.
 * Everything in IEEE FP64, one rounding per operation, no fused multiply-add.
 */
#include <math.h>
#include <stdlib.h>

typedef struct {
    int index;          /* best flat grid index, -1 if no grid point counts */
    double power;       /* Q of the best point */
    double centre;      /* c in [0, 1) */
    double width;       /* T, phase units */
    double ingress;     /* tau, phase units */
    double depth;       /* delta */
} oracle_shape_fit;

static double grid_frac(int m, int n)
{
    return n > 1 ? (double)m / (double)(n - 1) : 0.0;
}

/* Q of one grid point; returns 0 and sets *ok = 0 when it does not count. */
double oracle_shape_point(int n, const double* phi, const double* w, const double* x, double c,
                          double T, double tau, double* delta, int* ok)
{
    double Ss = 0.0, Sss = 0.0, Sxs = 0.0;
    double half = T * 0.5;
    for (int i = 0; i < n; ++i) {
        double u = phi[i] - c;
        double D = u - floor(u + 0.5);
        double a = fabs(D);
        double s;
        if (tau > 0.0) {
            s = (half - a) / tau;
            s = s > 1.0 ? 1.0 : (s < 0.0 ? 0.0 : s);
        } else {
            s = a < half ? 1.0 : 0.0;
        }
        Ss += w[i] * s;
        Sss += w[i] * (s * s);
        Sxs += w[i] * x[i] * s;
    }
    double var = Sss - Ss * Ss;
    *ok = Sxs < 0.0 && var > 0.0;
    if (!*ok) { *delta = 0.0; return 0.0; }
    *delta = -Sxs / var;
    return Sxs * Sxs / var;
}

/*
 * Trapezoid refit of one peak.  dt, w, x as oracle_prep returns them; f the peak's
 * frequency; (i1, k, nb) its box.  Returns 0, or -1 on bad arguments.
 */
int oracle_shape(int n, const double* dt, const double* w, const double* x, double f, int nb,
                 int i1, int k, int nc, int nw, int na, double wlo, double whi, double amax,
                 oracle_shape_fit* out, double* Q)
{
    if (n < 1 || nb < 2 || k < 1 || nc < 1 || nw < 1 || na < 1 || !(f > 0.0) || !(wlo > 0.0) ||
        !(whi >= wlo) || !(amax >= 0.0 && amax <= 0.5))
        return -1;
    double* phi = (double*)malloc(sizeof(double) * (size_t)n);
    if (!phi) return -2;
    for (int i = 0; i < n; ++i) {
        double p = dt[i] * f;
        phi[i] = p - floor(p);
    }
    double pb = ((double)i1 + 0.5 * (double)k) / (double)nb;
    pb = pb - floor(pb);
    double q = (double)k / (double)nb;
    out->index = -1;
    out->power = 0.0; out->centre = 0.0; out->width = 0.0; out->ingress = 0.0; out->depth = 0.0;
    for (int m = 0; m < nc; ++m) {
        double c = pb + q * ((nc > 1 ? grid_frac(m, nc) : 0.5) - 0.5);
        for (int u = 0; u < nw; ++u) {
            double T = q * (wlo + grid_frac(u, nw) * (whi - wlo));
            for (int v = 0; v < na; ++v) {
                double tau = T * (amax * grid_frac(v, na));
                double delta;
                int ok;
                double P = oracle_shape_point(n, phi, w, x, c, T, tau, &delta, &ok);
                int idx = (m * nw + u) * na + v;
                if (Q) Q[idx] = ok ? P : 0.0;
                if (ok && (out->index < 0 || P > out->power)) {
                    out->index = idx;
                    out->power = P;
                    out->centre = c - floor(c);
                    out->width = T;
                    out->ingress = tau;
                    out->depth = delta;
                }
            }
        }
    }
    free(phi);
    return 0;
}

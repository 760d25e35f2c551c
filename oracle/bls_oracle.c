/*
 * bls_oracle.c -- plain, slow, FP64 box-least-squares (BLS) periodogram.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library; the product path never does.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes. Sec. 2.2.2 of the paper searches every light curve with a
 * "standard" BLS (Kovacs, Zucker & Mazeh 2002; Tingley 2003): phase the curve at
 * each trial period, test a range of box durations and phases, keep the best.
 * The paper prints no formula, so the definition is restated here from the cited
 * method:
 *
 *   weights   w_i = dy_i^-2 / W,  W = sum dy_i^-2            (unit weights if dy = NULL)
 *   flux      x_i = y_i - ybar,   ybar = sum w_i y_i          (so sum w_i x_i = 0)
 *   box B     r = sum_B w_i,  s = sum_B w_i x_i
 *   fit       level L = s/r in B, H = -s/(1-r) outside (weighted least squares)
 *   chi2_min  = sum w x^2 - s^2/(r(1-r))
 *   power     P = s^2/(r(1-r)),  SR = sqrt(P),  depth = H - L = -s/(r(1-r))
 *
 * Binned form: the folded phase is cut into nb equal bins and B runs over the
 * cyclic runs of k consecutive bins, kmin <= k <= kmax.  Readings where the paper
 * is silent (phase origin, bin clamp, kmin/kmax from q, dips-only sign, tie-break,
 * SNR, epoch) are the ones listed with the design notes; each is marked below.
 *
 * Arithmetic: IEEE FP64, round-to-nearest, and the file is compiled with
 * -ffp-contract=off so no multiply-add is fused.  Summation is plain, in point
 * order for the bins and in bin order for the box sums.
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int j;              /* frequency index, -1 if the slot is empty */
    double freq, period, epoch, duration, depth, snr, sr, power;
    int i1, k;          /* first bin and width (bins) of the best box */
    double sde;         /* signal detection efficiency of the peak */
} oracle_peak;

typedef struct {
    const double* t; const float* y; const float* dy; int n;
    const double* freqs; int nf; double fmin, df;
    int nb, kmin, kmax;
} oracle_curve;

/* Reading: kmin = max(1, floor(qmin*nb + 1e-9)), kmax = min(nb-1, ceil(qmax*nb - 1e-9)). */
int oracle_kminmax(int nb, double qmin, double qmax, int* kmin, int* kmax)
{
    if (nb < 2 || !(qmin > 0.0) || !(qmax >= qmin) || !(qmax < 1.0)) return -1;
    int lo = (int)floor(qmin * nb + 1e-9);
    int hi = (int)ceil(qmax * nb - 1e-9);
    if (lo < 1) lo = 1;
    if (hi > nb - 1) hi = nb - 1;
    if (hi < lo) hi = lo;
    *kmin = lo; *kmax = hi;
    return 0;
}

/* Uniform grid: f_j = fmin + j*df, both operations rounded (no fused multiply-add). */
double oracle_freq(int j, double fmin, double df)
{
    double jd = (double)j;
    double step = jd * df;
    return fmin + step;
}

/* Fold one time offset at frequency f into one of nb phase bins:
 * p = dt*f, phase = p - floor(p) in [0,1), bin = floor(phase*nb), clamped to nb-1
 * (reading: phase*nb can round up to nb). */
int oracle_fold(double dt, double f, int nb)
{
    double p = dt * f;
    double ph = p - floor(p);
    double u = ph * (double)nb;
    int b = (int)floor(u);
    if (b >= nb) b = nb - 1;
    if (b < 0) b = 0;
    return b;
}

/* Preparation of one curve.  Reading: phase origin t_ref = min t and dt = t - t_ref;
 * the weighted mean is taken about the first flux value, ybar = y0 + sum w (y - y0),
 * which is the same mean but returns exactly zero residuals for constant flux.
 * scal[0..3] = t_ref, W, ybar, sum w x^2. */
int oracle_prep(int n, const double* t, const float* y, const float* dy,
                double* dt, double* w, double* x, double* scal)
{
    if (n < 1) return -1;
    double tref = t[0];
    for (int i = 1; i < n; i++) if (t[i] < tref) tref = t[i];
    double W = 0.0;
    for (int i = 0; i < n; i++) {
        double inv = 1.0;
        if (dy) { double d = (double)dy[i]; inv = 1.0 / (d * d); }
        w[i] = inv;
        W += inv;
    }
    for (int i = 0; i < n; i++) w[i] = w[i] / W;
    double y0 = (double)y[0];
    double acc = 0.0;
    for (int i = 0; i < n; i++) acc += w[i] * ((double)y[i] - y0);
    double ybar = y0 + acc;
    double swx2 = 0.0;
    for (int i = 0; i < n; i++) {
        dt[i] = t[i] - tref;
        x[i] = (double)y[i] - ybar;
        swx2 += w[i] * x[i] * x[i];
    }
    scal[0] = tref; scal[1] = W; scal[2] = ybar; scal[3] = swx2;
    return 0;
}

/* Per-point bins of a curve for a list of frequencies: bins[q*n + i]. */
int oracle_bins(int n, const double* t, int nq, const double* f, int nb, int* bins)
{
    if (n < 1 || nb < 2) return -1;
    double tref = t[0];
    for (int i = 1; i < n; i++) if (t[i] < tref) tref = t[i];
    for (int q = 0; q < nq; q++)
        for (int i = 0; i < n; i++)
            bins[(size_t)q * n + i] = oracle_fold(t[i] - tref, f[q], nb);
    return 0;
}

/* Phase histograms of one frequency: Hw[b] = sum w_i, Hx[b] = sum w_i x_i, point order,
 * and Hn[b] = number of points in bin b. */
static void histogram(int n, const double* dt, const double* w, const double* x,
                      double f, int nb, double* Hw, double* Hx, int* Hn)
{
    for (int b = 0; b < nb; b++) { Hw[b] = 0.0; Hx[b] = 0.0; Hn[b] = 0; }
    for (int i = 0; i < n; i++) {
        int b = oracle_fold(dt[i], f, nb);
        Hw[b] += w[i];
        Hx[b] += w[i] * x[i];
        Hn[b] += 1;
    }
}

/* Box sweep of one histogram: every start i1 and width k, cyclic, sums taken bin by
 * bin from the start.  Reading: a box counts only when both levels of the step model
 * are defined, i.e. it holds at least one point and leaves at least one out (0 < r < 1
 * exactly); this is decided on point counts, not on the rounded weight sums.  With
 * sign = 0 only dips (s < 0) count; with sign = 1 both signs count.  The best box is
 * kept with a strict '>' while i1 and then k ascend, so equal powers resolve to the
 * smallest (i1, k); if no box has positive power the result is P = 0, (0, kmin). */
static double sweep(int n, int nb, int kmin, int kmax, int sign, const double* Hw,
                    const double* Hx, const int* Hn, int* bi1, int* bk)
{
    double best = 0.0;
    int b1 = 0, bkk = kmin;
    for (int i1 = 0; i1 < nb; i1++) {
        double r = 0.0, s = 0.0;
        int cnt = 0;
        for (int k = 1; k <= kmax; k++) {
            int m = (i1 + k - 1) % nb;
            r += Hw[m];
            s += Hx[m];
            cnt += Hn[m];
            if (k < kmin) continue;
            if (cnt == 0 || cnt == n) continue;
            if (sign == 0 && !(s < 0.0)) continue;
            double P = (s * s) / (r * (1.0 - r));
            if (P > best) { best = P; b1 = i1; bkk = k; }
        }
    }
    *bi1 = b1; *bk = bkk;
    return best;
}

/* Box sums (r, s) of one box, taken bin by bin exactly as in the sweep. */
static void box_sums(int nb, const double* Hw, const double* Hx, int i1, int k,
                     double* r, double* s)
{
    double rr = 0.0, ss = 0.0;
    for (int m = 0; m < k; m++) { rr += Hw[(i1 + m) % nb]; ss += Hx[(i1 + m) % nb]; }
    *r = rr; *s = ss;
}

/* Best box at one frequency from prepared arrays; also returns its (r, s). */
int oracle_power(int n, const double* dt, const double* w, const double* x, double f,
                 int nb, int kmin, int kmax, int sign, double* P, int* i1, int* k,
                 double* r, double* s)
{
    if (n < 1 || nb < 2 || kmin < 1 || kmax < kmin || kmax > nb) return -1;
    double* H = (double*)malloc(sizeof(double) * 2 * (size_t)nb);
    int* Hn = (int*)malloc(sizeof(int) * (size_t)nb);
    if (!H || !Hn) { free(H); free(Hn); return -2; }
    histogram(n, dt, w, x, f, nb, H, H + nb, Hn);
    *P = sweep(n, nb, kmin, kmax, sign, H, H + nb, Hn, i1, k);
    box_sums(nb, H, H + nb, *i1, *k, r, s);
    free(H);
    free(Hn);
    return 0;
}

/* Power of one given box (i1, k) at frequency f: P = s^2/(r(1-r)) with the sums taken bin
 * by bin as in the sweep; 0 when the box does not count (r outside (0,1), or s >= 0 with
 * dips only).  Also returns r and s. */
int oracle_box(int n, const double* dt, const double* w, const double* x, double f, int nb,
               int i1, int k, int sign, double* P, double* r, double* s)
{
    if (n < 1 || nb < 2 || i1 < 0 || i1 >= nb || k < 1 || k > nb) return -1;
    double* H = (double*)malloc(sizeof(double) * 2 * (size_t)nb);
    int* Hn = (int*)malloc(sizeof(int) * (size_t)nb);
    if (!H || !Hn) { free(H); free(Hn); return -2; }
    histogram(n, dt, w, x, f, nb, H, H + nb, Hn);
    box_sums(nb, H, H + nb, i1, k, r, s);
    int cnt = 0;
    for (int m = 0; m < k; m++) cnt += Hn[(i1 + m) % nb];
    free(H);
    free(Hn);
    double rr = *r, ss = *s;
    *P = 0.0;
    if (cnt > 0 && cnt < n && (sign == 1 || ss < 0.0)) *P = (ss * ss) / (rr * (1.0 - rr));
    return 0;
}

/* Reported quantities of one (frequency, box).  Reading: period = 1/f,
 * duration = k/(nb f), epoch = mid-box time t_ref + frac((i1 + k/2)/nb)/f,
 * depth = -s/(r(1-r)), SR = sqrt(P), SNR = depth/sigma_depth = SR*sqrt(W). */
static void derive(oracle_peak* pk, int j, double f, int nb, int i1, int k, double P,
                   double r, double s, double tref, double W)
{
    pk->j = j; pk->freq = f; pk->period = 1.0 / f; pk->i1 = i1; pk->k = k;
    pk->duration = (double)k / ((double)nb * f);
    double ph = ((double)i1 + 0.5 * (double)k) / (double)nb;
    ph = ph - floor(ph);
    pk->epoch = tref + ph / f;
    pk->power = P;
    if (P > 0.0) {
        pk->depth = -s / (r * (1.0 - r));
        pk->sr = sqrt(P);
        pk->snr = pk->sr * sqrt(W);
    } else {
        pk->depth = 0.0; pk->sr = 0.0; pk->snr = 0.0;
    }
}

/* Reading for the top-k: j is a peak if it is strictly above its left neighbour and
 * not below its right one (ends count as open); peaks rank by (P desc, j asc).  The
 * global argmax with the smallest index is always the first peak. */
static void top_peaks(int nf, const double* P, int topk, int* js)
{
    for (int q = 0; q < topk; q++) js[q] = -1;
    for (int j = 0; j < nf; j++) {
        if (j > 0 && !(P[j] > P[j - 1])) continue;
        if (j < nf - 1 && !(P[j] >= P[j + 1])) continue;
        /* insertion into the ranked list */
        int pos = topk;
        for (int q = 0; q < topk; q++) {
            if (js[q] < 0 || P[j] > P[js[q]]) { pos = q; break; }
        }
        if (pos == topk) continue;
        for (int q = topk - 1; q > pos; q--) js[q] = js[q - 1];
        js[pos] = j;
    }
    if (topk > 0 && js[0] < 0 && nf > 0) js[0] = 0;
}

typedef struct {
    int n; double* dt; double* w; double* x; double scal[4];
} prepped;

static int prep_curve(const oracle_curve* c, prepped* p)
{
    p->n = c->n;
    p->dt = (double*)malloc(sizeof(double) * 3 * (size_t)c->n);
    if (!p->dt) return -2;
    p->w = p->dt + c->n; p->x = p->w + c->n;
    return oracle_prep(c->n, c->t, c->y, c->dy, p->dt, p->w, p->x, p->scal);
}

static double grid_freq(const oracle_curve* c, int j)
{
    return c->freqs ? c->freqs[j] : oracle_freq(j, c->fmin, c->df);
}

/* Mean and population sd of SR = sqrt(P) over a spectrum (plain sums in frequency order),
 * the statistics of the signal detection efficiency. */
static void sr_stats(int nf, const double* P, double* mean_out, double* sd_out)
{
    double mean = 0.0, var = 0.0;
    for (int j = 0; j < nf; j++) mean += sqrt(P[j]);
    mean /= (double)nf;
    for (int j = 0; j < nf; j++) {
        double d = sqrt(P[j]) - mean;
        var += d * d;
    }
    *mean_out = mean;
    *sd_out = sqrt(var / (double)nf);
}

/* Full periodogram of one curve.  P, i1, k (length nf, each may be NULL) receive the
 * per-frequency best box; peaks (length topk) the ranked peaks. */
int oracle_bls(const oracle_curve* c, int sign, double* P, int* i1, int* k,
               int topk, oracle_peak* peaks)
{
    if (!c || c->n < 2 || c->nf < 1 || c->nb < 2 || c->kmin < 1 || c->kmax < c->kmin ||
        c->kmax > c->nb)
        return -1;
    prepped p;
    int rc = prep_curve(c, &p);
    if (rc) { free(p.dt); return rc; }
    int nb = c->nb, nf = c->nf;
    double* H = (double*)malloc(sizeof(double) * 2 * (size_t)nb);
    int* Hn = (int*)malloc(sizeof(int) * (size_t)nb);
    double* Pl = P ? P : (double*)malloc(sizeof(double) * (size_t)nf);
    int* I1 = i1 ? i1 : (int*)malloc(sizeof(int) * (size_t)nf);
    int* K = k ? k : (int*)malloc(sizeof(int) * (size_t)nf);
    for (int j = 0; j < nf; j++) {
        double f = grid_freq(c, j);
        histogram(p.n, p.dt, p.w, p.x, f, nb, H, H + nb, Hn);
        Pl[j] = sweep(p.n, nb, c->kmin, c->kmax, sign, H, H + nb, Hn, &I1[j], &K[j]);
    }
    if (topk > 0 && peaks) {
        /* signal detection efficiency (Kovacs, Zucker & Mazeh 2002, the BLS paper cited in
         * Sec. 2.2.2): SDE = (SR_peak - <SR>) / sd(SR) over the curve's whole spectrum,
         * sd the population standard deviation; 0 for a flat spectrum */
        double mean, sd;
        sr_stats(nf, Pl, &mean, &sd);
        int js[64];
        int kk = topk > 64 ? 64 : topk;
        top_peaks(nf, Pl, kk, js);
        for (int q = 0; q < kk; q++) {
            if (js[q] < 0) { memset(&peaks[q], 0, sizeof(oracle_peak)); peaks[q].j = -1; continue; }
            int j = js[q];
            double f = grid_freq(c, j), r, s;
            histogram(p.n, p.dt, p.w, p.x, f, nb, H, H + nb, Hn);
            box_sums(nb, H, H + nb, I1[j], K[j], &r, &s);
            derive(&peaks[q], j, f, nb, I1[j], K[j], Pl[j], r, s, p.scal[0], p.scal[1]);
            peaks[q].sde = sd > 0.0 ? (peaks[q].sr - mean) / sd : 0.0;
        }
    }
    if (!P) free(Pl);
    if (!i1) free(I1);
    if (!k) free(K);
    free(H);
    free(Hn);
    free(p.dt);
    return 0;
}

/* ---- multi-threaded driver over many curves (for timing the oracle as it stands) ---- */

typedef struct {
    int nc; const oracle_curve* cv; int sign;
    prepped* pp; double** Pc; int** I1c; int** Kc;
    int* item_curve; int* item_j0; int nitems; int chunk;
    atomic_int next; atomic_int err;
} many_ctx;

static void* many_worker(void* arg)
{
    many_ctx* m = (many_ctx*)arg;
    int nbmax = 2;
    for (int c = 0; c < m->nc; c++) if (m->cv[c].nb > nbmax) nbmax = m->cv[c].nb;
    double* H = (double*)malloc(sizeof(double) * 2 * (size_t)nbmax);
    int* Hn = (int*)malloc(sizeof(int) * (size_t)nbmax);
    if (!H || !Hn) { free(H); free(Hn); atomic_store(&m->err, -2); return NULL; }
    for (;;) {
        int it = atomic_fetch_add(&m->next, 1);
        if (it >= m->nitems) break;
        int c = m->item_curve[it], j0 = m->item_j0[it];
        const oracle_curve* cv = &m->cv[c];
        const prepped* p = &m->pp[c];
        int j1 = j0 + m->chunk; if (j1 > cv->nf) j1 = cv->nf;
        for (int j = j0; j < j1; j++) {
            double f = grid_freq(cv, j);
            histogram(p->n, p->dt, p->w, p->x, f, cv->nb, H, H + cv->nb, Hn);
            m->Pc[c][j] = sweep(p->n, cv->nb, cv->kmin, cv->kmax, m->sign, H, H + cv->nb, Hn,
                                &m->I1c[c][j], &m->Kc[c][j]);
        }
    }
    free(H);
    free(Hn);
    return NULL;
}

/* Periodograms of nc curves on nthreads POSIX threads, split into (curve, 256-frequency)
 * items.  P_all (sum of nf, may be NULL) receives the per-frequency powers back to back;
 * peaks (nc*topk) the ranked peaks of every curve. */
int oracle_bls_many(int nc, const oracle_curve* cv, int sign, int nthreads,
                    double* P_all, int topk, oracle_peak* peaks)
{
    if (nc < 1 || nthreads < 1) return -1;
    for (int c = 0; c < nc; c++) {
        const oracle_curve* q = &cv[c];
        if (q->n < 2 || q->nf < 1 || q->nb < 2 || q->kmin < 1 || q->kmax < q->kmin ||
            q->kmax > q->nb)
            return -1;
    }
    many_ctx m;
    memset(&m, 0, sizeof(m));
    m.nc = nc; m.cv = cv; m.sign = sign; m.chunk = 256;
    m.pp = (prepped*)calloc((size_t)nc, sizeof(prepped));
    m.Pc = (double**)calloc((size_t)nc, sizeof(double*));
    m.I1c = (int**)calloc((size_t)nc, sizeof(int*));
    m.Kc = (int**)calloc((size_t)nc, sizeof(int*));
    size_t nitems = 0, off = 0;
    int rc = 0;
    for (int c = 0; c < nc; c++) {
        if (prep_curve(&cv[c], &m.pp[c])) rc = -2;
        m.Pc[c] = P_all ? P_all + off : (double*)malloc(sizeof(double) * (size_t)cv[c].nf);
        m.I1c[c] = (int*)malloc(sizeof(int) * (size_t)cv[c].nf);
        m.Kc[c] = (int*)malloc(sizeof(int) * (size_t)cv[c].nf);
        off += (size_t)cv[c].nf;
        nitems += (size_t)((cv[c].nf + m.chunk - 1) / m.chunk);
    }
    m.item_curve = (int*)malloc(sizeof(int) * nitems);
    m.item_j0 = (int*)malloc(sizeof(int) * nitems);
    size_t it = 0;
    for (int c = 0; c < nc; c++)
        for (int j0 = 0; j0 < cv[c].nf; j0 += m.chunk) { m.item_curve[it] = c; m.item_j0[it] = j0; it++; }
    m.nitems = (int)nitems;
    atomic_store(&m.next, 0);
    atomic_store(&m.err, 0);
    if (rc == 0) {
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
        for (int q = 0; q < nthreads; q++) pthread_create(&th[q], NULL, many_worker, &m);
        for (int q = 0; q < nthreads; q++) pthread_join(th[q], NULL);
        free(th);
        rc = atomic_load(&m.err);
    }
    if (rc == 0 && topk > 0 && peaks) {
        int kk = topk > 64 ? 64 : topk;
        int js[64];
        for (int c = 0; c < nc; c++) {
            const oracle_curve* q = &cv[c];
            double* H = (double*)malloc(sizeof(double) * 2 * (size_t)q->nb);
            int* Hn = (int*)malloc(sizeof(int) * (size_t)q->nb);
            double mean, sd;
            sr_stats(q->nf, m.Pc[c], &mean, &sd);
            top_peaks(q->nf, m.Pc[c], kk, js);
            for (int e = 0; e < kk; e++) {
                oracle_peak* pk = &peaks[(size_t)c * topk + e];
                if (js[e] < 0) { memset(pk, 0, sizeof(*pk)); pk->j = -1; continue; }
                int j = js[e];
                double f = grid_freq(q, j), r, s;
                histogram(m.pp[c].n, m.pp[c].dt, m.pp[c].w, m.pp[c].x, f, q->nb, H, H + q->nb, Hn);
                box_sums(q->nb, H, H + q->nb, m.I1c[c][j], m.Kc[c][j], &r, &s);
                derive(pk, j, f, q->nb, m.I1c[c][j], m.Kc[c][j], m.Pc[c][j], r, s,
                       m.pp[c].scal[0], m.pp[c].scal[1]);
                pk->sde = sd > 0.0 ? (pk->sr - mean) / sd : 0.0;
            }
            free(H);
            free(Hn);
        }
    }
    for (int c = 0; c < nc; c++) {
        free(m.pp[c].dt);
        if (!P_all) free(m.Pc[c]);
        free(m.I1c[c]); free(m.Kc[c]);
    }
    free(m.pp); free(m.Pc); free(m.I1c); free(m.Kc); free(m.item_curve); free(m.item_j0);
    return rc;
}

/*
 * Oracle for Hercules exact k-NN query answering (Echihabi et al., "Hercules
 * Against Data Series Similarity Search", PVLDB 15(10), 2022).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU
 * restatement of what the query path computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Arithmetic: IEEE binary64, round to nearest, no FMA contraction (the file is
 * compiled with -ffp-contract=off), every sum taken sequentially in index
 * order.  Functions:
 *
 *   hko_dist2        squared Euclidean distance (Sec. 2, k-NN definition and
 *                    the Euclidean distance it is defined with)
 *   hko_knn_update   brute-force k-NN: running top-k by (distance, id)
 *                    (Sec. 2, k-NN query definition; ties broken by lower id)
 *   hko_seg_stats    mean and population standard deviation of a segment
 *                    (Sec. 3.2, EAPCA synopsis z_i)
 *   hko_lb_eapca     LB_EAPCA of a query to a node synopsis (Sec. 2; used by
 *                    Algorithms Approx-kNN and FindCandidateLeaves, Sec. 3.4;
 *                    the bound comes from DSTree and is restated below)
 *   hko_paa          Piecewise Aggregate Approximation (Sec. 2)
 *   hko_isax_bp      iSAX breakpoints: standard normal quantiles j/256
 *   hko_isax_symbol  iSAX symbol of a PAA value (alphabet 256, Sec. 2)
 *   hko_lb_sax       LB_SAX of a query PAA to an iSAX word (Sec. 3.4,
 *                    Algorithms CSWorker and CRWorker)
 *   hko_dtw2         DTW with a Sakoe-Chiba band (Sec. 2: any distance with
 *                    a lower bound, e.g. DTW), squared point costs
 *   hko_dtw_knn_update  brute-force k-NN under that DTW
 *   hko_envelope, hko_lb_keogh, hko_lb_keogh_eapca, hko_lb_keogh_sax
 *                    LB_Keogh (the lower bound the paper cites for DTW) and
 *                    its forms against a node synopsis and an iSAX word
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Squared Euclidean distance, summed in index order.                        */
/* D(q,x) = sum_{j=0}^{n-1} (q_j - x_j)^2, every operation in binary64.      */
/* ------------------------------------------------------------------------ */
double hko_dist2(const float *q, const float *x, int n)
{
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = (double)q[j] - (double)x[j];
        double t = d * d;
        s = s + t;
    }
    return s;
}

/* (d, id) < (d2, id2) lexicographically. */
static int pair_less(double d, int64_t id, double d2, int64_t id2)
{
    if (d < d2) return 1;
    if (d > d2) return 0;
    return id < id2;
}

/* Insert (d, id) into the ascending list (ds, ids) of length k if it beats
 * the last entry; the last entry falls off. */
static void topk_insert(double *ds, int64_t *ids, int k, double d, int64_t id)
{
    if (!pair_less(d, id, ds[k - 1], ids[k - 1])) return;
    int p = k - 1;
    while (p > 0 && pair_less(d, id, ds[p - 1], ids[p - 1])) {
        ds[p] = ds[p - 1];
        ids[p] = ids[p - 1];
        --p;
    }
    ds[p] = d;
    ids[p] = id;
}

double hko_dtw2(const float *q, const float *x, int n, int r);

typedef struct {
    const float *X;
    int64_t id0, cnt;
    int n;
    const float *Q;
    int k;
    int band;        /* < 0: Euclidean; >= 0: DTW with this band */
    int64_t *ids;
    double *d2;
    int q_begin, q_end;
} knn_job;

static void *knn_worker(void *arg)
{
    knn_job *J = (knn_job *)arg;
    for (int qi = J->q_begin; qi < J->q_end; ++qi) {
        const float *q = J->Q + (int64_t)qi * J->n;
        double *ds = J->d2 + (int64_t)qi * J->k;
        int64_t *is = J->ids + (int64_t)qi * J->k;
        for (int64_t r = 0; r < J->cnt; ++r) {
            double d = J->band < 0 ? hko_dist2(q, J->X + r * J->n, J->n)
                                   : hko_dtw2(q, J->X + r * J->n, J->n, J->band);
            topk_insert(ds, is, J->k, d, J->id0 + r);
        }
    }
    return NULL;
}

/* Initialise nq running top-k lists to (+inf, -1). */
void hko_knn_init(int nq, int k, int64_t *ids, double *d2)
{
    for (int64_t i = 0; i < (int64_t)nq * k; ++i) {
        ids[i] = -1;
        d2[i] = INFINITY;
    }
}

/* Brute-force k-NN, one block of consecutive series at a time.
 * X: cnt rows of n floats whose ids are id0, id0+1, ...; Q: nq rows of n
 * floats; ids/d2: nq*k running lists (ascending by (D, id)).  Calling this
 * over consecutive blocks of a collection gives the same lists as one call
 * over the whole collection: every series is offered to every query's list,
 * in id order.  Queries are divided among nthreads threads. */
static int knn_run(const float *X, int64_t id0, int64_t cnt, int n, const float *Q, int nq, int k,
                   int band, int64_t *ids, double *d2, int nthreads);

int hko_knn_update(const float *X, int64_t id0, int64_t cnt, int n,
                   const float *Q, int nq, int k, int64_t *ids, double *d2,
                   int nthreads)
{
    return knn_run(X, id0, cnt, n, Q, nq, k, -1, ids, d2, nthreads);
}

/* The same under DTW with a Sakoe-Chiba band of half-width band >= 0. */
int hko_dtw_knn_update(const float *X, int64_t id0, int64_t cnt, int n,
                       const float *Q, int nq, int k, int band, int64_t *ids,
                       double *d2, int nthreads)
{
    if (band < 0) return -1;
    return knn_run(X, id0, cnt, n, Q, nq, k, band, ids, d2, nthreads);
}

static int knn_run(const float *X, int64_t id0, int64_t cnt, int n, const float *Q, int nq, int k,
                   int band, int64_t *ids, double *d2, int nthreads)
{
    if (n <= 0 || nq < 0 || k <= 0 || cnt < 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nq) nthreads = nq > 0 ? nq : 1;
    knn_job *jobs = (knn_job *)calloc((size_t)nthreads, sizeof(knn_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        knn_job *J = &jobs[t];
        J->X = X; J->id0 = id0; J->cnt = cnt; J->n = n; J->Q = Q; J->k = k; J->band = band;
        J->ids = ids; J->d2 = d2;
        J->q_begin = (int)((int64_t)nq * t / nthreads);
        J->q_end = (int)((int64_t)nq * (t + 1) / nthreads);
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, knn_worker, &jobs[t]) != 0) break;
        started = t;
    }
    knn_worker(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    /* any job whose thread failed to start runs here */
    for (int t = started + 1; t < nthreads; ++t) knn_worker(&jobs[t]);
    free(jobs);
    free(th);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* EAPCA segment statistics (Sec. 3.2): mean and population standard         */
/* deviation of x[a..b).  Two passes: the mean, then the mean square          */
/* deviation from it.                                                         */
/* ------------------------------------------------------------------------ */
void hko_seg_stats(const float *x, int a, int b, double *mu, double *sd)
{
    double l = (double)(b - a);
    double s = 0.0;
    for (int j = a; j < b; ++j) s = s + (double)x[j];
    double m = s / l;
    double v = 0.0;
    for (int j = a; j < b; ++j) {
        double d = (double)x[j] - m;
        double t = d * d;
        v = v + t;
    }
    *mu = m;
    *sd = sqrt(v / l);
}

/* Segment statistics of many rows at once: rows[i] of X (row length n). */
void hko_seg_stats_rows(const float *X, const int64_t *rows, int64_t cnt, int n,
                        int a, int b, double *mu, double *sd)
{
    for (int64_t i = 0; i < cnt; ++i)
        hko_seg_stats(X + rows[i] * (int64_t)n, a, b, &mu[i], &sd[i]);
}

/* Distance from v to the closed interval [lo, hi] (0 inside). */
static double dist_to_range(double v, double lo, double hi)
{
    if (v < lo) return lo - v;
    if (v > hi) return v - hi;
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* LB_EAPCA (Sec. 2; Algorithms Approx-kNN and FindCandidateLeaves prune    */
/* with it, Sec. 3.4).  The paper takes the bound from DSTree unrestated.     */
/* For a node with segmentation r_1 < ... < r_m = n (r_0 = 0) and synopsis    */
/* z_i = {mu_min, mu_max, sd_min, sd_max} (Sec. 3.2), with                    */
/* l_i = r_i - r_{i-1} and the query's own segment mean and standard          */
/* deviation (mu_q,i, sd_q,i):                                                */
/*   LB^2 = sum_i l_i * ( dist(mu_q,i, [mu_min,mu_max])^2                     */
/*                      + dist(sd_q,i, [sd_min,sd_max])^2 )                   */
/* It lower-bounds D because, per segment, sum (q-x)^2 =                      */
/* l (mu_q - mu_x)^2 + |q~ - x~|^2 >= l (mu_q - mu_x)^2 + (|q~| - |x~|)^2     */
/* = l [(mu_q - mu_x)^2 + (sd_q - sd_x)^2]  (q~, x~ centred, |q~| = sqrt(l) sd) */
/* seg_end: m right endpoints; env: m*4 doubles (mu_min, mu_max, sd_min,      */
/* sd_max).  Returns the squared bound.                                       */
/* ------------------------------------------------------------------------ */
double hko_lb_eapca(const float *q, int m, const int32_t *seg_end,
                    const double *env)
{
    double lb = 0.0;
    int a = 0;
    for (int i = 0; i < m; ++i) {
        int b = seg_end[i];
        double mu, sd;
        hko_seg_stats(q, a, b, &mu, &sd);
        double dm = dist_to_range(mu, env[4 * i + 0], env[4 * i + 1]);
        double ds = dist_to_range(sd, env[4 * i + 2], env[4 * i + 3]);
        double l = (double)(b - a);
        double t = dm * dm + ds * ds;
        lb = lb + l * t;
        a = b;
    }
    return lb;
}

/* ------------------------------------------------------------------------ */
/* PAA (Sec. 2): w equal segments of length n/w, each the mean of its points.  */
/* ------------------------------------------------------------------------ */
void hko_paa(const float *x, int n, int w, double *out)
{
    int l = n / w;
    for (int i = 0; i < w; ++i) {
        double s = 0.0;
        for (int j = i * l; j < (i + 1) * l; ++j) s = s + (double)x[j];
        out[i] = s / (double)l;
    }
}

/* ------------------------------------------------------------------------ */
/* iSAX breakpoints for an alphabet of 256 (Sec. 2): beta_j with              */
/* Phi(beta_j) = j/256, j = 1..255, Phi the standard normal CDF,              */
/* Phi(b) = erfc(-b/sqrt(2))/2.  The lower half (j < 128, beta_j < 0) is      */
/* found by bisection on [-40, 0] until the bracket stops shrinking; the      */
/* normal's symmetry Phi(-x) = 1 - Phi(x) gives beta_128 = 0 and              */
/* beta_{256-j} = -beta_j (near 0, Phi is flat to binary64 precision, so      */
/* bisection alone cannot resolve beta_128).                                   */
/* ------------------------------------------------------------------------ */
static double std_normal_cdf(double b) { return 0.5 * erfc(-b / sqrt(2.0)); }

void hko_isax_bp(double *out /* 255 */)
{
    for (int j = 1; j < 128; ++j) {
        double target = (double)j / 256.0;
        double lo = -40.0, hi = 0.0;
        for (int it = 0; it < 400; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (std_normal_cdf(mid) < target) lo = mid; else hi = mid;
        }
        /* pick the end of the bracket whose CDF is closer to the target */
        double elo = fabs(std_normal_cdf(lo) - target);
        double ehi = fabs(std_normal_cdf(hi) - target);
        out[j - 1] = (elo <= ehi) ? lo : hi;
    }
    out[127] = 0.0;
    for (int j = 129; j <= 255; ++j) out[j - 1] = -out[256 - j - 1];
}

/* iSAX symbol of a PAA value: the number of breakpoints (given as float32,
 * promoted) that are <= v.  A value equal to a breakpoint takes the upper
 * cell.  Symbols run 0..255; cell s spans [beta_s, beta_{s+1}) with
 * beta_0 = -inf and beta_256 = +inf. */
int hko_isax_symbol(double v, const float *bp /* 255 */)
{
    int s = 0;
    for (int j = 0; j < 255; ++j)
        if ((double)bp[j] <= v) s = s + 1;
    return s;
}

/* LB_SAX (Sec. 3.4, Algorithm CSWorker): for a query PAA p (w segments) and an iSAX word
 * sym (w symbols) of a series of length n:
 *   LB^2 = (n/w) * sum_i dist(p_i, [beta_{s_i}, beta_{s_i+1}])^2
 * with beta_0 = -inf, beta_256 = +inf. */
double hko_lb_sax(const double *paa_q, const uint8_t *sym, int w, int n,
                  const float *bp /* 255 */)
{
    double acc = 0.0;
    for (int i = 0; i < w; ++i) {
        int s = sym[i];
        double lo = (s == 0) ? -INFINITY : (double)bp[s - 1];
        double hi = (s == 255) ? INFINITY : (double)bp[s];
        double d = dist_to_range(paa_q[i], lo, hi);
        acc = acc + d * d;
    }
    return ((double)n / (double)w) * acc;
}

/* ------------------------------------------------------------------------ */
/* DTW (Sec. 2: Hercules supports any distance with a lower-bounding          */
/* distance, e.g. DTW, with the lower bound of Keogh and Ratanamahatana,     */
/* KAIS 2005).  Squared point costs, a Sakoe-Chiba band of half-width r:     */
/*   D(i, j) = (q_i - x_j)^2 + min(D(i-1, j-1), D(i-1, j), D(i, j-1))        */
/* over |i - j| <= r, with D = +inf outside the band and D(-1,-1) = 0; the   */
/* distance is D(n-1, n-1).  Rows i ascending, columns j ascending; the     */
/* minimum is exact, the cost and the addition are rounded once each.        */
/* With r = 0 the only path is the diagonal and D equals hko_dist2.          */
/* ------------------------------------------------------------------------ */
double hko_dtw2(const float *q, const float *x, int n, int r)
{
    double *prev = (double *)malloc(sizeof(double) * (size_t)n);
    double *cur = (double *)malloc(sizeof(double) * (size_t)n);
    if (!prev || !cur) { free(prev); free(cur); return NAN; }
    for (int j = 0; j < n; ++j) prev[j] = INFINITY;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) cur[j] = INFINITY;
        int jlo = i - r < 0 ? 0 : i - r;
        int jhi = i + r > n - 1 ? n - 1 : i + r;
        for (int j = jlo; j <= jhi; ++j) {
            double best;
            if (i == 0 && j == 0) {
                best = 0.0;
            } else {
                double a = (i > 0 && j > 0) ? prev[j - 1] : INFINITY;
                double b = i > 0 ? prev[j] : INFINITY;
                double c = j > 0 ? cur[j - 1] : INFINITY;
                best = a < b ? a : b;
                best = c < best ? c : best;
            }
            double d = (double)q[i] - (double)x[j];
            double t = d * d;
            cur[j] = t + best;
        }
        double *sw = prev; prev = cur; cur = sw;
    }
    double out = prev[n - 1];
    free(prev);
    free(cur);
    return out;
}

/* Envelope of q for band r (Keogh 2005): L_j = min, U_j = max of q over
 * positions j-r .. j+r inside [0, n). */
void hko_envelope(const float *q, int n, int r, float *L, float *U)
{
    for (int j = 0; j < n; ++j) {
        int a = j - r < 0 ? 0 : j - r;
        int b = j + r > n - 1 ? n - 1 : j + r;
        float lo = q[a], hi = q[a];
        for (int t = a + 1; t <= b; ++t) {
            if (q[t] < lo) lo = q[t];
            if (q[t] > hi) hi = q[t];
        }
        L[j] = lo;
        U[j] = hi;
    }
}

/* LB_Keogh^2(q, x) = sum_j dist(x_j, [L_j, U_j])^2, index order: every
 * warping path matches x_j to some q_i with |i - j| <= r, which lies in
 * [L_j, U_j], so each term is at most that path's cost at x_j. */
double hko_lb_keogh(const float *q, const float *x, int n, int r)
{
    float *L = (float *)malloc(sizeof(float) * (size_t)n);
    float *U = (float *)malloc(sizeof(float) * (size_t)n);
    if (!L || !U) { free(L); free(U); return NAN; }
    hko_envelope(q, n, r, L, U);
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = dist_to_range((double)x[j], (double)L[j], (double)U[j]);
        s = s + d * d;
    }
    free(L);
    free(U);
    return s;
}

/* Distance between the closed intervals [a1, b1] and [a2, b2]. */
static double interval_gap(double a1, double b1, double a2, double b2)
{
    if (a1 > b2) return a1 - b2;
    if (a2 > b1) return a2 - b1;
    return 0.0;
}

/* Mean of v[a..b), binary64, sequential. */
static double mean_f(const float *v, int a, int b)
{
    double s = 0.0;
    for (int j = a; j < b; ++j) s = s + (double)v[j];
    return s / (double)(b - a);
}

/* LB_Keogh against a node synopsis (a reading: the paper gives no formula).
 * dist(x_j, [L_j, U_j])^2 is jointly convex in (x_j, L_j, U_j), so over a
 * segment of l points its sum is at least l times its value at the means
 * (Jensen): l dist(mean x, [mean L, mean U])^2, and with the node's series'
 * segment means in [mu_min, mu_max] at least
 * l gap([mu_min, mu_max], [mean L, mean U])^2.  Segments in order. */
double hko_lb_keogh_eapca(const float *q, int n, int r, int m, const int32_t *seg_end, const double *env)
{
    float *L = (float *)malloc(sizeof(float) * (size_t)n);
    float *U = (float *)malloc(sizeof(float) * (size_t)n);
    if (!L || !U) { free(L); free(U); return NAN; }
    hko_envelope(q, n, r, L, U);
    double acc = 0.0;
    int a = 0;
    for (int i = 0; i < m; ++i) {
        int b = seg_end[i];
        double lm = mean_f(L, a, b), um = mean_f(U, a, b);
        double g = interval_gap(env[4 * i], env[4 * i + 1], lm, um);
        double l = (double)(b - a);
        acc = acc + l * (g * g);
        a = b;
    }
    free(L);
    free(U);
    return acc;
}

/* LB_Keogh against an iSAX word: the same argument over the 16 PAA segments,
 * with the series' PAA inside its symbol's cell [beta_s, beta_{s+1}):
 * (n/16) sum_i gap(cell_i, [PAA(L)_i, PAA(U)_i])^2. */
double hko_lb_keogh_sax(const float *q, int n, int r, const uint8_t *sym, const float *bp /* 255 */)
{
    float *L = (float *)malloc(sizeof(float) * (size_t)n);
    float *U = (float *)malloc(sizeof(float) * (size_t)n);
    if (!L || !U) { free(L); free(U); return NAN; }
    hko_envelope(q, n, r, L, U);
    int w = 16, l = n / w;
    double acc = 0.0;
    for (int i = 0; i < w; ++i) {
        double lm = mean_f(L, i * l, (i + 1) * l), um = mean_f(U, i * l, (i + 1) * l);
        int s = sym[i];
        double lo = s == 0 ? -INFINITY : (double)bp[s - 1];
        double hi = s == 255 ? INFINITY : (double)bp[s];
        double g = interval_gap(lo, hi, lm, um);
        acc = acc + g * g;
    }
    free(L);
    free(U);
    return (double)l * acc;
}

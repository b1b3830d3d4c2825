/*
 * O2 -- triangle-inequality (group / point filtered) K-means in FP64.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference leg may load this library.  It
 * shares no code with the brute-force oracle (lloyd.c) or with the CUDA
 * library.
 *
 * What it computes.  KPynq's accelerator (Sec. I) is a "Multi-level Filters"
 * stage -- a group-level and a point-level filter that remove distance
 * computations -- followed by a "Distance Calculator" for the pairs that
 * survive.  The paper gives no formulas; the filter vocabulary is that of
 * Yinyang K-means (Ding et al., ICML 2015), whose last author is also KPynq's.
 * This file takes the steps in that order, in FP64:
 *
 *   state    a(x) label, u(x) >= d(x, c_a) upper bound, lb_g(x) <= d(x, c)
 *            for every c != a(x) in centroid group g (Euclidean distances).
 *   t = 0    all K distances: a = argmin (lowest index on ties),
 *            u = d(x, c_a), lb_g = min over c in g, c != a of d(x, c).
 *   update   c'_k = mean of its points (empty: unchanged), drift
 *            delta_k = ||c'_k - c_k||, group drift delta_g = max over g.
 *   t >= 1   bound update:  u += delta_a;  lb_g^new = lb_g - delta_g
 *            global filter: min_g lb_g^new > u        -> label kept
 *            tighten:       u = d(x, c_a), test again -> label kept
 *            group filter:  skip group g if lb_g^new > best-so-far
 *            point filter:  inside a surviving group skip c if
 *                           lb_g^old - delta_c > best-so-far
 *            distance calculator: d(x, c) for the remaining c
 *            bound refresh: lb_g = min over c in g, c != new label, of the
 *                           computed distance or the point-filter bound
 *                           (the old label's tightened distance joins its
 *                           group when the label moves).
 *
 * A filter skips only when the bound exceeds the best distance by the
 * relative margin RHO, which covers the FP64 rounding of the bound
 * arithmetic, so every centroid that could tie or beat the current best is
 * evaluated.  Distances are summed exactly as in the brute-force oracle
 * (i ascending, no fused multiply-add), so both pick the same label.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define RHO 9.094947017729282e-13 /* 2^-40 */

/* skip counters, per iteration */
enum {
    CNT_GLOBAL = 0,   /* points kept by the global filter before tightening */
    CNT_TIGHT = 1,    /* points kept by the global filter after tightening */
    CNT_GROUP = 2,    /* (point, group) pairs removed by the group filter */
    CNT_POINT = 3,    /* (point, centroid) pairs removed by the point filter */
    CNT_DIST = 4,     /* distance evaluations, tightening included */
    CNT_CHANGED = 5,  /* labels changed */
    CNT_N = 6
};

/* squared Euclidean distance, i ascending; the label is chosen on these
   values (as in the brute-force oracle) and the bounds on their roots */
static double dist2(const double *x, const double *c, int32_t D)
{
    double s = 0.0;
    for (int32_t i = 0; i < D; ++i) {
        double t = x[i] - c[i];
        s = s + t * t;
    }
    return s;
}

/* bound b rules centroid out against best distance bd */
static int beyond(double b, double bd) { return b > bd * (1.0 + RHO); }

/* iteration 0: every distance; sets a, u, lb (N x G, row per point) */
void o2_init_assign(const double *X, int64_t N, int32_t D, const double *C,
                    int32_t K, int32_t G, const int32_t *grp, int32_t *a,
                    double *u, double *lb, int64_t *cnt)
{
    double *s = (double *)malloc((size_t)K * sizeof(double));
    if (!s) return;
    memset(cnt, 0, CNT_N * sizeof(int64_t));
    for (int64_t n = 0; n < N; ++n) {
        const double *x = X + n * (int64_t)D;
        int32_t best = 0;
        for (int32_t k = 0; k < K; ++k) {
            s[k] = dist2(x, C + (int64_t)k * D, D);
            if (s[k] < s[best]) best = k;
        }
        cnt[CNT_DIST] += K;
        double *row = lb + n * (int64_t)G;
        for (int32_t g = 0; g < G; ++g) row[g] = INFINITY;
        for (int32_t k = 0; k < K; ++k)
            if (k != best && sqrt(s[k]) < row[grp[k]]) row[grp[k]] = sqrt(s[k]);
        a[n] = best;
        u[n] = sqrt(s[best]);
    }
    cnt[CNT_CHANGED] = N;
    free(s);
}

/*
 * Iteration t >= 1.  C holds C^t; delta[k] and delta_g[g] are the drifts from
 * C^{t-1} to C^t.  a, u, lb hold the state left by iteration t-1 and are
 * updated in place.  cnt receives the CNT_* counters.
 */
void o2_assign(const double *X, int64_t N, int32_t D, const double *C,
               int32_t K, int32_t G, const int32_t *grp, const double *delta,
               const double *delta_g, int32_t *a, double *u, double *lb,
               int64_t *cnt)
{
    double *lbo = (double *)malloc((size_t)G * sizeof(double));
    double *lbn = (double *)malloc((size_t)G * sizeof(double));
    double *cand = (double *)malloc((size_t)K * sizeof(double));
    char *scanned = (char *)malloc((size_t)G);
    if (!lbo || !lbn || !cand || !scanned) goto out;
    memset(cnt, 0, CNT_N * sizeof(int64_t));
    for (int64_t n = 0; n < N; ++n) {
        const double *x = X + n * (int64_t)D;
        double *row = lb + n * (int64_t)G;
        int32_t al = a[n];
        /* bound update after drift */
        double ub = u[n] + delta[al];
        double m = INFINITY;
        for (int32_t g = 0; g < G; ++g) {
            lbo[g] = row[g];
            lbn[g] = row[g] - delta_g[g];
            if (lbn[g] < m) m = lbn[g];
        }
        /* global filter */
        if (beyond(m, ub)) {
            cnt[CNT_GLOBAL] += 1;
            u[n] = ub;
            memcpy(row, lbn, (size_t)G * sizeof(double));
            continue;
        }
        /* tighten the upper bound and test again */
        double sa = dist2(x, C + (int64_t)al * D, D);
        double da = sqrt(sa);
        cnt[CNT_DIST] += 1;
        if (beyond(m, da)) {
            cnt[CNT_TIGHT] += 1;
            u[n] = da;
            memcpy(row, lbn, (size_t)G * sizeof(double));
            continue;
        }
        /* group filter, point filter, distance calculator */
        int32_t best = al;
        double bs = sa, bd = da; /* best squared distance and its root */
        cand[al] = da;
        for (int32_t g = 0; g < G; ++g) {
            scanned[g] = 0;
            if (beyond(lbn[g], bd)) {
                cnt[CNT_GROUP] += 1;
                continue;
            }
            scanned[g] = 1;
            for (int32_t c = 0; c < K; ++c) {
                if (grp[c] != g || c == al) continue;
                double bound = lbo[g] - delta[c];
                if (beyond(bound, bd)) {
                    cand[c] = bound;
                    cnt[CNT_POINT] += 1;
                    continue;
                }
                double sc = dist2(x, C + (int64_t)c * D, D);
                cnt[CNT_DIST] += 1;
                cand[c] = sqrt(sc);
                if (sc < bs || (sc == bs && c < best)) {
                    best = c;
                    bs = sc;
                    bd = cand[c];
                }
            }
        }
        /* bound refresh */
        for (int32_t g = 0; g < G; ++g) {
            if (scanned[g]) {
                double v = INFINITY;
                for (int32_t c = 0; c < K; ++c)
                    if (grp[c] == g && c != best && cand[c] < v) v = cand[c];
                row[g] = v;
            } else {
                row[g] = lbn[g];
                if (g == grp[al] && best != al && da < row[g]) row[g] = da;
            }
        }
        if (best != al) cnt[CNT_CHANGED] += 1;
        a[n] = best;
        u[n] = bd;
    }
out:
    free(lbo);
    free(lbn);
    free(cand);
    free(scanned);
}

/*
 * Centroid update with drift.  C_new = means (empty cluster: unchanged),
 * delta[k] = ||C_new[k] - C_old[k]||, delta_g[g] = max over the group.
 * Returns J(a, C_old).
 */
double o2_update(const double *X, int64_t N, int32_t D, const int32_t *a,
                 const double *C_old, int32_t K, int32_t G, const int32_t *grp,
                 double *C_new, double *delta, double *delta_g)
{
    double *S = (double *)calloc((size_t)K * (size_t)D, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    double J = 0.0;
    if (!S || !cnt) {
        J = NAN;
        goto out;
    }
    for (int64_t n = 0; n < N; ++n) {
        const double *x = X + n * (int64_t)D;
        const double *c = C_old + (int64_t)a[n] * D;
        double s = 0.0;
        for (int32_t i = 0; i < D; ++i) {
            S[(int64_t)a[n] * D + i] += x[i];
            double t = x[i] - c[i];
            s = s + t * t;
        }
        J += s;
        cnt[a[n]] += 1;
    }
    for (int32_t g = 0; g < G; ++g) delta_g[g] = 0.0;
    for (int32_t k = 0; k < K; ++k) {
        double dd = 0.0;
        for (int32_t i = 0; i < D; ++i) {
            int64_t j = (int64_t)k * D + i;
            C_new[j] = cnt[k] > 0 ? S[j] / (double)cnt[k] : C_old[j];
            double t = C_new[j] - C_old[j];
            dd = dd + t * t;
        }
        delta[k] = sqrt(dd);
        if (delta[k] > delta_g[grp[k]]) delta_g[grp[k]] = delta[k];
    }
out:
    free(S);
    free(cnt);
    return J;
}

/*
 * Full filtered run.  Same stopping rule and outputs as the brute-force
 * oracle's o1_fit.  labels_hist (nullable, max_iter x N) receives the
 * assignment of every iteration, J_hist (nullable, max_iter) J_t, cnt_hist
 * (nullable, max_iter x CNT_N) the counters.  Returns the number of
 * iterations, or -1 on allocation failure.
 */
int32_t o2_fit(const double *X, int64_t N, int32_t D, const double *C0,
               int32_t K, int32_t G, const int32_t *grp, int32_t max_iter,
               double tol, int32_t *labels, double *C, int32_t *labels_hist,
               double *J_hist, int64_t *cnt_hist, double *J_final)
{
    size_t csz = (size_t)K * (size_t)D;
    double *Cn = (double *)malloc(csz * sizeof(double));
    double *u = (double *)malloc((size_t)N * sizeof(double));
    double *lb = (double *)malloc((size_t)N * (size_t)G * sizeof(double));
    double *delta = (double *)malloc((size_t)K * sizeof(double));
    double *delta_g = (double *)malloc((size_t)G * sizeof(double));
    int64_t cnt[CNT_N];
    int32_t n_iter = -1;
    if (!Cn || !u || !lb || !delta || !delta_g) goto out;
    memcpy(C, C0, csz * sizeof(double));
    n_iter = 0;
    double J_prev = 0.0;
    for (int32_t t = 0; t < max_iter; ++t) {
        if (t == 0)
            o2_init_assign(X, N, D, C, K, G, grp, labels, u, lb, cnt);
        else
            o2_assign(X, N, D, C, K, G, grp, delta, delta_g, labels, u, lb, cnt);
        double J = o2_update(X, N, D, labels, C, K, G, grp, Cn, delta, delta_g);
        memcpy(C, Cn, csz * sizeof(double));
        if (labels_hist) memcpy(labels_hist + (int64_t)t * N, labels, (size_t)N * sizeof(int32_t));
        if (J_hist) J_hist[t] = J;
        if (cnt_hist) memcpy(cnt_hist + (int64_t)t * CNT_N, cnt, sizeof(cnt));
        n_iter = t + 1;
        int stop = (cnt[CNT_CHANGED] == 0) || (t >= 1 && (J_prev - J) < tol * J_prev);
        J_prev = J;
        if (stop) break;
    }
    /* final assignment to the returned centroids, through the filters */
    if (n_iter > 0) {
        o2_assign(X, N, D, C, K, G, grp, delta, delta_g, labels, u, lb, cnt);
        if (J_final) {
            double J = 0.0;
            for (int64_t n = 0; n < N; ++n) {
                const double *x = X + n * (int64_t)D;
                const double *c = C + (int64_t)labels[n] * D;
                double s = 0.0;
                for (int32_t i = 0; i < D; ++i) {
                    double t = x[i] - c[i];
                    s = s + t * t;
                }
                J += s;
            }
            *J_final = J;
        }
    }
out:
    free(Cn);
    free(u);
    free(lb);
    free(delta);
    free(delta_g);
    return n_iter;
}

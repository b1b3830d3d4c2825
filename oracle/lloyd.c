/*
 * O1 -- brute-force Lloyd K-means in FP64.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference leg may load this library.  The CUDA
 * library never links, includes or calls it, and this file includes nothing
 * from the CUDA side.
 *
 * What it computes.  KPynq (Abstract; Sec. I) is a work-efficient
 * triangle-inequality K-means: its multi-level filters only discard distance
 * evaluations that cannot change a point's nearest centroid, and its distance
 * calculator evaluates the rest.  Its result is therefore that of the
 * "CPU-based standard K-means" it is compared against (Abstract; Sec. II),
 * i.e. Lloyd's algorithm.  This file is Lloyd's algorithm written out from
 * its definition, with the readings the paper leaves open fixed as follows:
 *
 *   assign   a(x) = argmin_k  sum_i (x_i - c_{k,i})^2   (FP64, i ascending,
 *            no fused multiply-add), ties to the LOWEST index k.
 *   update   c'_k = (sum of x with a(x) = k) / |{x : a(x) = k}|, sums in
 *            point order; an empty cluster keeps its previous centroid.
 *   J        J(a, C) = sum_x ||x - c_{a(x)}||^2 with the centroids C that
 *            produced the assignment.
 *   loop     iteration t assigns from C^t and updates to C^{t+1}; stop after
 *            max_iter iterations, or when no label changed, or (t >= 1) when
 *            J_{t-1} - J_t < tol * J_{t-1}.
 *   finish   labels = assignment to the returned centroids; J_final = J of
 *            that pair.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off [-fopenmp].  The OpenMP
 * pragma only splits the independent per-point argmins across threads; the
 * arithmetic of each point is unchanged, so results do not depend on it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* squared Euclidean distance, summed over i = 0..D-1 in order */
static double sqdist(const double *x, const double *c, int32_t D)
{
    double s = 0.0;
    for (int32_t i = 0; i < D; ++i) {
        double t = x[i] - c[i];
        s = s + t * t;
    }
    return s;
}

/*
 * Nearest centroid of every point.  labels[n] = argmin (lowest index on
 * ties).  d1sq/d2sq (nullable) receive the smallest and second-smallest
 * squared distances (d2sq = +inf when K = 1).  prev (nullable) is the previous
 * assignment; the return value is the number of labels that differ from it
 * (N when prev is NULL).
 */
int64_t o1_assign(const double *X, int64_t N, int32_t D, const double *C,
                  int32_t K, const int32_t *prev, int32_t *labels,
                  double *d1sq, double *d2sq)
{
    int64_t changed = 0;
#pragma omp parallel for schedule(static) reduction(+ : changed)
    for (int64_t n = 0; n < N; ++n) {
        const double *x = X + n * (int64_t)D;
        int32_t best = 0;
        double b1 = INFINITY, b2 = INFINITY;
        for (int32_t k = 0; k < K; ++k) {
            double s = sqdist(x, C + (int64_t)k * D, D);
            if (s < b1) {          /* strict: an equal later k never wins */
                b2 = b1;
                b1 = s;
                best = k;
            } else if (s < b2) {
                b2 = s;
            }
        }
        labels[n] = best;
        if (d1sq) d1sq[n] = b1;
        if (d2sq) d2sq[n] = b2;
        if (!prev || prev[n] != best) changed += 1;
    }
    return changed;
}

/* J(a, C): sum over points of the squared distance to the assigned centroid */
double o1_objective(const double *X, int64_t N, int32_t D, const int32_t *labels,
                    const double *C, int32_t K)
{
    (void)K;
    double J = 0.0;
    for (int64_t n = 0; n < N; ++n)
        J += sqdist(X + n * (int64_t)D, C + (int64_t)labels[n] * D, D);
    return J;
}

/*
 * Centroid update.  C_new[k] = mean of the points labelled k (sums in point
 * order); an empty cluster keeps C_old[k].  counts (nullable) receives the
 * cluster sizes.  Returns J(labels, C_old).
 */
double o1_update(const double *X, int64_t N, int32_t D, const int32_t *labels,
                 const double *C_old, int32_t K, double *C_new, int64_t *counts)
{
    double *S = (double *)calloc((size_t)K * (size_t)D, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    if (!S || !cnt) {
        free(S);
        free(cnt);
        return NAN;
    }
    for (int64_t n = 0; n < N; ++n) {
        const double *x = X + n * (int64_t)D;
        double *s = S + (int64_t)labels[n] * D;
        for (int32_t i = 0; i < D; ++i) s[i] += x[i];
        cnt[labels[n]] += 1;
    }
    for (int32_t k = 0; k < K; ++k) {
        for (int32_t i = 0; i < D; ++i) {
            int64_t j = (int64_t)k * D + i;
            C_new[j] = cnt[k] > 0 ? S[j] / (double)cnt[k] : C_old[j];
        }
        if (counts) counts[k] = cnt[k];
    }
    double J = o1_objective(X, N, D, labels, C_old, K);
    free(S);
    free(cnt);
    return J;
}

/*
 * Full Lloyd run from C0.  On return C holds the final centroids, labels the
 * final assignment to them and *J_final its objective.  J_hist[t] = J_t and
 * changed_hist[t] = labels changed at iteration t (both nullable, max_iter
 * entries).  Returns the number of iterations performed, or -1 on allocation
 * failure.
 */
int32_t o1_fit(const double *X, int64_t N, int32_t D, const double *C0,
               int32_t K, int32_t max_iter, double tol, int32_t *labels,
               double *C, double *J_hist, int64_t *changed_hist, double *J_final)
{
    size_t csz = (size_t)K * (size_t)D;
    double *Cn = (double *)malloc(csz * sizeof(double));
    int32_t *prev = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!Cn || !prev) {
        free(Cn);
        free(prev);
        return -1;
    }
    memcpy(C, C0, csz * sizeof(double));
    int32_t n_iter = 0;
    double J_prev = 0.0;
    for (int32_t t = 0; t < max_iter; ++t) {
        int64_t changed = o1_assign(X, N, D, C, K, t == 0 ? NULL : prev,
                                    labels, NULL, NULL);
        double J = o1_update(X, N, D, labels, C, K, Cn, NULL);
        memcpy(C, Cn, csz * sizeof(double));
        memcpy(prev, labels, (size_t)N * sizeof(int32_t));
        if (J_hist) J_hist[t] = J;
        if (changed_hist) changed_hist[t] = changed;
        n_iter = t + 1;
        int stop = (changed == 0) || (t >= 1 && (J_prev - J) < tol * J_prev);
        J_prev = J;
        if (stop) break;
    }
    o1_assign(X, N, D, C, K, NULL, labels, NULL, NULL);
    if (J_final) *J_final = o1_objective(X, N, D, labels, C, K);
    free(Cn);
    free(prev);
    return n_iter;
}

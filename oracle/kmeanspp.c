/*
 * O4 -- k-means++ seeding in FP64.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference leg may load this library.  It
 * shares no code with the other oracles or with the CUDA library.
 *
 * What it computes.  The paper takes its initial centroids as given; the
 * library offers the D^2 seeding of k-means++ (Arthur and Vassilvitskii,
 * SODA 2007) as an alternative initialisation: the first centre is a point
 * drawn uniformly, and each further centre is a point drawn with probability
 * proportional to D(x)^2, its squared distance to the nearest centre chosen
 * so far.  Random numbers are inputs (u[j] in [0, 1), one per centre), and
 * the draw is made exactly reproducible:
 *
 *   D(x)^2   sum_i (x_i - c_i)^2 in FP64, i ascending, no fused multiply-add,
 *            minimised over the centres chosen so far;
 *   weights  q(x) = floor(D(x)^2 * 2^s) as 64-bit integers, where 2^s is the
 *            power of two with max_x D(x)^2 * 2^s in [2^31, 2^32) (exact
 *            scaling; weights below 2^-32 of the largest become 0);
 *   draw     T = floor(u[j] * W), W = sum_x q(x) (integer sum, exact in any
 *            order; T = W - 1 if the product rounds up to W); the centre is
 *            the first point in index order whose running sum of q exceeds T;
 *            when W = 0 (every point already a centre) the draw is uniform:
 *            floor(u[j] * N);
 *   first    floor(u[0] * N).
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static double sq(const double *x, const double *c, int32_t D)
{
    double s = 0.0;
    for (int32_t i = 0; i < D; ++i) {
        double t = x[i] - c[i];
        s = s + t * t;
    }
    return s;
}

static int64_t uniform_index(double u, int64_t N)
{
    int64_t i = (int64_t)floor(u * (double)N);
    if (i < 0) i = 0;
    if (i >= N) i = N - 1;
    return i;
}

/*
 * Chooses K centre indices into idx[K].  dmin (nullable, N) receives the
 * final D(x)^2 (to the K chosen centres).  Returns 0, or -1 on bad
 * arguments or allocation failure.
 */
int32_t o4_kmeanspp(const double *X, int64_t N, int32_t D, int32_t K, const double *u, int64_t *idx,
                    double *dmin)
{
    if (N < 1 || D < 1 || K < 1 || K > N) return -1;
    double *d = (double *)malloc((size_t)N * sizeof(double));
    if (!d) return -1;
    for (int64_t n = 0; n < N; ++n) d[n] = INFINITY;
    for (int32_t j = 0; j < K; ++j) {
        int64_t pick;
        if (j == 0) {
            pick = uniform_index(u[0], N);
        } else {
            double wmax = 0.0;
            for (int64_t n = 0; n < N; ++n)
                if (d[n] > wmax) wmax = d[n];
            uint64_t W = 0;
            int e = 0;
            if (wmax > 0.0) {
                frexp(wmax, &e); /* wmax = m 2^e, m in [0.5, 1) */
                for (int64_t n = 0; n < N; ++n) W += (uint64_t)floor(ldexp(d[n], 32 - e));
            }
            if (W == 0) {
                pick = uniform_index(u[j], N);
            } else {
                uint64_t T = (uint64_t)floor(u[j] * (double)W);
                if (T >= W) T = W - 1;
                uint64_t run = 0;
                pick = N - 1;
                for (int64_t n = 0; n < N; ++n) {
                    run += (uint64_t)floor(ldexp(d[n], 32 - e));
                    if (run > T) {
                        pick = n;
                        break;
                    }
                }
            }
        }
        idx[j] = pick;
        const double *c = X + pick * (int64_t)D;
        for (int64_t n = 0; n < N; ++n) {
            double s = sq(X + n * (int64_t)D, c, D);
            if (s < d[n]) d[n] = s;
        }
    }
    if (dmin)
        for (int64_t n = 0; n < N; ++n) dmin[n] = d[n];
    free(d);
    return 0;
}

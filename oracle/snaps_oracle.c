/*
 * FP64 brute-force oracle for the SNAPS outlier-detection hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never calls it and shares no code with it.
 *
 * What it computes (Gowanlock et al., arXiv 2405.20176):
 *   - feature normalisation to [0, 1] (Sec. 3.3), with missing values
 *     (NaN) replaced by the column mean first (Sec. 2.1);
 *   - for one feature subspace S (a bitmask over the features, Eq. 1):
 *       * the distance similarity self-join (DSSJ, Sec. 3.5): for each query
 *         point, the number of other points within eps and the sum of their
 *         Euclidean distances (Sec. 3.5.1 metrics 1 and 2);
 *       * the k-nearest-neighbour self-join (kNNSJ, Sec. 3.6): the k nearest
 *         other points, nearest first (the kNN graph of Fig. 1b).
 *
 * Readings of the paper taken here:
 *   - distance is Euclidean over the subspace's features (Sec. 3.1 terms;
 *     the Table 2 values reproduce only with it);
 *   - a point is never its own neighbour (Table 2: point 10 has 0 eps
 *     neighbours and in-degree 0);
 *   - eps is inclusive, tested on squared distances: d2 <= eps2;
 *   - kNN order is by (squared distance, index) ascending, so exact ties go
 *     to the lower index (Fig. 1b draws the tie of point 1 to point 2);
 *   - all arithmetic is IEEE double; inputs are taken as given.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC snaps_oracle.c -o libsnaps_oracle.so
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Column-wise min-max normalisation (Sec. 3.3), rounded to float32.
 * x: n x f row-major doubles.  out: n x f row-major floats.
 * nan_to_mean != 0: a NaN becomes the mean of the column's non-NaN values
 * before min and max are taken (Sec. 2.1).  A constant column maps to 0.
 * Returns 0, or -1 on bad sizes. */
int snaps_oracle_normalise(const double *x, int64_t n, int f, int nan_to_mean,
                           float *out)
{
    if (n < 1 || f < 1) return -1;
    double *col = (double *)malloc((size_t)n * sizeof(double));
    if (!col) return -1;
    for (int c = 0; c < f; ++c) {
        for (int64_t i = 0; i < n; ++i) col[i] = x[i * f + c];
        if (nan_to_mean) {
            double s = 0.0;
            int64_t m = 0;
            for (int64_t i = 0; i < n; ++i)
                if (!isnan(col[i])) { s += col[i]; ++m; }
            double mean = m > 0 ? s / (double)m : 0.0;
            for (int64_t i = 0; i < n; ++i)
                if (isnan(col[i])) col[i] = mean;
        }
        double lo = col[0], hi = col[0];
        for (int64_t i = 1; i < n; ++i) {
            if (col[i] < lo) lo = col[i];
            if (col[i] > hi) hi = col[i];
        }
        double span = hi - lo;
        for (int64_t i = 0; i < n; ++i) {
            double v = span > 0.0 ? (col[i] - lo) / span : 0.0;
            out[i * f + c] = (float)v;
        }
    }
    free(col);
    return 0;
}

/* Squared Euclidean distance between rows a and b over the features in mask. */
static double dist2(const double *x, int f, uint32_t mask, int64_t a, int64_t b)
{
    double s = 0.0;
    for (int c = 0; c < f; ++c) {
        if (mask & (1u << c)) {
            double d = x[a * f + c] - x[b * f + c];
            s += d * d;
        }
    }
    return s;
}

/* Is (d2, j) ordered before (e2, l)?  Distance first, then index. */
static int before(double d2, int64_t j, double e2, int64_t l)
{
    return d2 < e2 || (d2 == e2 && j < l);
}

/* Self-join of one subspace by brute force over all pairs.
 *
 * x: n x f row-major doubles (normalised features).  mask: the subspace.
 * queries: the query rows to evaluate (NULL means all n rows, in order);
 * nq: their count.  Every query is joined against all n rows.
 * k > 0: writes knn_idx / knn_d2 (nq x k): the k nearest other rows, by
 *   (squared distance, index).  Requires k <= n - 1.
 * eps2 >= 0: writes eps_count (nq) = #{j != i : d2 <= eps2} and
 *   eps_sum (nq) = sum of sqrt(d2) over those j.
 * nthreads > 0 sets the OpenMP thread count.
 * Returns 0, or -1 on bad arguments. */
int snaps_oracle_join(const double *x, int64_t n, int f, uint32_t mask, int k,
                      double eps2, const int64_t *queries, int64_t nq,
                      int32_t *knn_idx, double *knn_d2, int64_t *eps_count,
                      double *eps_sum, int nthreads)
{
    if (n < 1 || f < 1 || f > 32 || mask == 0 || nq < 0) return -1;
    if (f < 32 && (mask >> f) != 0) return -1;
    if (k < 0 || (k > 0 && (int64_t)k > n - 1)) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = queries ? queries[q] : q;
        if (i < 0 || i >= n) { failed = 1; continue; }
        /* the k best seen so far, kept sorted nearest first */
        double *bd = k > 0 ? knn_d2 + q * k : NULL;
        int32_t *bj = k > 0 ? knn_idx + q * k : NULL;
        int filled = 0;
        int64_t cnt = 0;
        double sum = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d2 = dist2(x, f, mask, i, j);
            if (eps2 >= 0.0 && d2 <= eps2) {
                cnt += 1;
                sum += sqrt(d2);
            }
            if (k > 0) {
                if (filled < k) {
                    int p = filled++;
                    while (p > 0 && before(d2, j, bd[p - 1], bj[p - 1])) {
                        bd[p] = bd[p - 1];
                        bj[p] = bj[p - 1];
                        --p;
                    }
                    bd[p] = d2;
                    bj[p] = (int32_t)j;
                } else if (before(d2, j, bd[k - 1], bj[k - 1])) {
                    int p = k - 1;
                    while (p > 0 && before(d2, j, bd[p - 1], bj[p - 1])) {
                        bd[p] = bd[p - 1];
                        bj[p] = bj[p - 1];
                        --p;
                    }
                    bd[p] = d2;
                    bj[p] = (int32_t)j;
                }
            }
        }
        if (eps2 >= 0.0) {
            eps_count[q] = cnt;
            eps_sum[q] = sum;
        }
    }
    return failed ? -1 : 0;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int snaps_oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

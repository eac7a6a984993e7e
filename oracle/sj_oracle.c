/*
 * Oracle for the Euclidean distance similarity self-join — TEST INFRASTRUCTURE.
 *
 * This file is the plain, slow, obviously correct CPU statement of what the
 * join computes.  It exists only to check the CUDA library: tests, the smoke
 * check and the CPU-baseline leg of the benchmark may call it; the product
 * path never does.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Definition followed (Sec. II-A, Eq. 1): for points a, b of a d-dimensional
 * set V, dist(a, b) = sqrt(sum_i (a_i - b_i)^2); the self-join returns every
 * ordered pair (a, b) in V x V with dist(a, b) <= eps.  Self pairs belong to
 * the result (Sec. IV-A defines the selectivity as (|R| - |V|) / |V|, so |R|
 * counts each point finding itself).
 *
 * Arithmetic (binding readings):
 *   e2 = eps * eps rounded once (IEEE binary64, round to nearest);
 *   s  = 0; for k = 0..d-1: t = x_i[k] - x_j[k]; s = s + t * t
 *        (sequential k, every operation rounded separately: this file must be
 *        compiled with -ffp-contract=off so no multiply-add is fused);
 *   (i, j) is in the result iff s <= e2; its distance is sqrt(s), correctly
 *   rounded.
 * Comparing s with fl(eps^2) instead of sqrt(s) with eps is a reading of the
 * paper (its tensor-core algorithm of Fig. 2 produces squared sums and never
 * takes the root); the two differ only for pairs within a relative 1e-15 of
 * eps.
 *
 * Also here: a double-double evaluation of the same sum (error-free
 * transformations TwoSum, Knuth; TwoProduct via fma, Ogita-Rump-Oishi 2005)
 * used to classify a pair as "borderline" when its exact squared distance
 * lies within a relative 1e-9 of eps.
 *
 * Layout: points are row-major n x d binary64.  Pairs are reported as 64-bit
 * keys (i << 32) | j, ascending, which is the natural order of the loops.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double sq_dist(const double* a, const double* b, int32_t d) {
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = a[k] - b[k];
        double t2 = t * t;
        s = s + t2;
    }
    return s;
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    return nthreads;
#else
    (void)nthreads;
    return 1;
#endif
}

/* Number of threads the oracle runs with for a request of `nthreads`
 * (<= 0 means all available). */
int sjo_threads(int nthreads) { return set_threads(nthreads); }

/* Per-query neighbour counts (Sec. II-A: |V| range queries).  counts[i] =
 * #{ j : s(i, j) <= e2 }.  Returns the total |R|. */
int64_t sjo_count(const double* x, int64_t n, int32_t d, double eps,
                  int64_t* counts, int nthreads) {
    const double e2 = eps * eps;
    int nt = set_threads(nthreads);
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        const double* a = x + i * (int64_t)d;
        for (int64_t j = 0; j < n; ++j) {
            double s = sq_dist(a, x + j * (int64_t)d, d);
            if (s <= e2) ++c;
        }
        if (counts) counts[i] = c;
        total += c;
    }
    return total;
}

/* The full result set, ascending by (i, j).  `counts` must hold the output of
 * sjo_count for the same inputs; keys_out has room for the total, dist_out is
 * NULL or has the same room.  Returns the number of pairs written. */
int64_t sjo_join(const double* x, int64_t n, int32_t d, double eps,
                 const int64_t* counts, int64_t* keys_out, double* dist_out,
                 int nthreads) {
    const double e2 = eps * eps;
    int nt = set_threads(nthreads);
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!start) return -1;
    start[0] = 0;
    for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + counts[i];
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        int64_t w = start[i];
        const double* a = x + i * (int64_t)d;
        for (int64_t j = 0; j < n; ++j) {
            double s = sq_dist(a, x + j * (int64_t)d, d);
            if (s <= e2) {
                keys_out[w] = (int64_t)(((uint64_t)i << 32) | (uint64_t)(uint32_t)j);
                if (dist_out) dist_out[w] = sqrt(s);
                ++w;
            }
        }
    }
    int64_t total = start[n];
    free(start);
    return total;
}

/* Rows of the result for a list of query indices (used to check very large
 * inputs one query at a time).  For query q = queries[r], writes row_counts[r]
 * and, when keys_out is not NULL, its neighbours j ascending into
 * keys_out[row_start[r] ..] where row_start is the prefix of row_counts
 * computed by the caller from a previous call with keys_out == NULL. */
int64_t sjo_rows(const double* x, int64_t n, int32_t d, double eps,
                 const int64_t* queries, int64_t nq, int64_t* row_counts,
                 const int64_t* row_start, int64_t* keys_out, double* dist_out,
                 int nthreads) {
    const double e2 = eps * eps;
    int nt = set_threads(nthreads);
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total) num_threads(nt)
    for (int64_t r = 0; r < nq; ++r) {
        int64_t i = queries[r];
        const double* a = x + i * (int64_t)d;
        int64_t c = 0;
        int64_t w = (keys_out && row_start) ? row_start[r] : 0;
        for (int64_t j = 0; j < n; ++j) {
            double s = sq_dist(a, x + j * (int64_t)d, d);
            if (s <= e2) {
                if (keys_out && row_start) {
                    keys_out[w] = (int64_t)(((uint64_t)i << 32) | (uint64_t)(uint32_t)j);
                    if (dist_out) dist_out[w] = sqrt(s);
                    ++w;
                }
                ++c;
            }
        }
        row_counts[r] = c;
        total += c;
    }
    return total;
}

/* All n squared distances from query q, in the oracle's operation order
 * (used to calibrate eps from sampled queries and to check single values). */
void sjo_sqdist_row(const double* x, int64_t n, int32_t d, int64_t q, double* out) {
    const double* a = x + q * (int64_t)d;
    for (int64_t j = 0; j < n; ++j) out[j] = sq_dist(a, x + j * (int64_t)d, d);
}

/* ---- double-double (error-free transformations) ------------------------ */

static void two_sum(double a, double b, double* s, double* e) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

static void two_prod(double a, double b, double* p, double* e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* (hi, lo) += (bh, bl), accurate double-double addition. */
static void dd_add(double* hi, double* lo, double bh, double bl) {
    double s, e, t, f;
    two_sum(*hi, bh, &s, &e);
    two_sum(*lo, bl, &t, &f);
    e += t;
    double s2 = s + e;
    e = e - (s2 - s);
    e += f;
    double s3 = s2 + e;
    *lo = e - (s3 - s2);
    *hi = s3;
}

/* Squared distance of points i and j in double-double: the difference of two
 * binary64 numbers is exact as a double-double (TwoSum), its square is formed
 * with TwoProduct plus the cross terms, and the sum is accumulated in
 * double-double.  Relative error about 2^-100. */
void sjo_sqdist_dd(const double* x, int32_t d, int64_t i, int64_t j,
                   double* hi_out, double* lo_out) {
    const double* a = x + i * (int64_t)d;
    const double* b = x + j * (int64_t)d;
    double hi = 0.0, lo = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double th, tl;
        two_sum(a[k], -b[k], &th, &tl);
        double ph, pl;
        two_prod(th, th, &ph, &pl);
        /* (th + tl)^2 = th^2 + 2 th tl + tl^2 */
        double cross = 2.0 * th * tl + tl * tl;
        pl += cross;
        dd_add(&hi, &lo, ph, pl);
    }
    *hi_out = hi;
    *lo_out = lo;
}

/* 1 iff the exact squared distance of (i, j) lies in
 * [ (eps (1 - rel))^2, (eps (1 + rel))^2 ], i.e. dist within a relative `rel`
 * of eps.  The band edges are formed in double-double too. */
int sjo_is_borderline(const double* x, int32_t d, int64_t i, int64_t j,
                      double eps, double rel) {
    double sh, sl;
    sjo_sqdist_dd(x, d, i, j, &sh, &sl);
    double lo_f = eps * (1.0 - rel), hi_f = eps * (1.0 + rel);
    double lh, ll, hh, hl;
    two_prod(lo_f, lo_f, &lh, &ll);
    two_prod(hi_f, hi_f, &hh, &hl);
    /* signs of the double-double differences s - lo^2 and hi^2 - s; a
     * normalised double-double has the sign of its high part */
    double ah = sh, al = sl;
    dd_add(&ah, &al, -lh, -ll);
    double bh = hh, bl = hl;
    dd_add(&bh, &bl, -sh, -sl);
    int ge_lo = (ah > 0) || (ah == 0 && al >= 0);
    int le_hi = (bh > 0) || (bh == 0 && bl >= 0);
    return ge_lo && le_hi;
}

/*
 * knor_oracle.c -- FP64 CPU oracle for Lloyd's k-means with MTI pruning.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent, slow, plainly
 * written reference that the CUDA library is checked against.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or helper with the CUDA library: it reads the
 * same FP32 input bits and computes in FP64.
 *
 * What it computes, and where in the paper (Mhembere et al., "knor: A NUMA-
 * Optimized In-Memory, Distributed and Semi-External-Memory k-means Library",
 * HPDC'17, arXiv 1606.08905) each piece is defined:
 *
 *   - Euclidean distance d(v,c) with the square root, and the centroid drift
 *     f(c^t) = d(c^t, c^{t-1}):  section "Nomenclature".
 *   - Lloyd's iteration: Phase I assigns each point to its nearest centroid,
 *     Phase II sets each centroid to the mean of its members, repeated until
 *     nothing changes:  section "Parallel Lloyd's Algorithm", the two-phase
 *     list, and Algorithm 1 (||Lloyd's) whose per-point scan keeps the first
 *     centroid on ties because it only replaces the best on a strict "<".
 *   - MTI pruning, Clauses 1-3, and the upper bound u^t maintained through
 *     the drift:  section "Minimal Triangle Inequality (MTI) Pruning".
 *   - The O(k^2) centroid-to-centroid table:  section "Asymptotic Memory
 *     Consumption".
 *
 * Readings taken where the paper is silent or garbled (each is listed with
 * its reason in the design notes of the repository):
 *   R1  The clauses compare u with centroid-to-centroid distances without a
 *       factor 1/2 and with the minimum taken over all centroids (which
 *       includes the zero self-distance).  Pruning is only sound with Elkan's
 *       half distances, so s(a) = 1/2 min_{c != a} d(c_a, c) and the per-
 *       centroid test uses 1/2 d(c_a, c).
 *   R2  u^t is read as Elkan's running bound: u is set to an exact distance
 *       when a point is scanned and grows by the drift of its centroid every
 *       iteration.
 *   R3  Ties go to the lowest centroid index in every full scan; every MTI
 *       test is a strict "<" with a rounding slack, so that no pruning
 *       decision rests on a tie and pruned runs assign exactly like unpruned
 *       ones.
 *   R4  Floating point: every bound is inflated (u, f) or deflated (1/2 d)
 *       by a factor that covers the FP64 rounding of the quantity.
 *   R5  Initialisation (the paper states none): Forgy, k distinct row indices
 *       drawn by Floyd's sampling algorithm driven by SplitMix64(seed);
 *       C^0 is those rows in drawn order.
 *   R6  Convergence: stop when no assignment changes (equivalent to "the
 *       centroids no longer change" under R7), or at max_iters.
 *   R7  An empty cluster keeps its previous centroid.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -shared -fPIC.
 * -ffp-contract=off keeps every a*b+c as two roundings, as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_EPS64 (1.1102230246251565e-16) /* 2^-53, FP64 unit roundoff */

/* Planted mistakes, for the test that shows the pins catch them.  None is
 * defined in a normal build; the test compiles throwaway variants with one
 * of them defined and checks that some pin fails. */
#ifdef ORACLE_PLANT_NO_HALF          /* prune on d(c_a,c) instead of 1/2 d */
#define ORACLE_HALF 1.0
#else
#define ORACLE_HALF 0.5
#endif
#ifdef ORACLE_PLANT_DROP_LAST_DIM    /* distance ignores the last coordinate */
#define ORACLE_DIMS(d) ((d) - 1)
#else
#define ORACLE_DIMS(d) (d)
#endif

/* ------------------------------------------------------------------ */
/* Random numbers for the Forgy initialisation (reading R5).           */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the state advances by the
 * golden-ratio increment and the output is the state passed through the
 * published 64-bit finaliser (shifts 30/27/31, two odd multipliers). */
uint64_t oracle_splitmix64_next(uint64_t *state) {
    uint64_t z;
    *state = *state + 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* An integer uniform on [0, m) from one 64-bit draw: the high 64 bits of the
 * 128-bit product r*m (Lemire's multiply-shift reduction). */
static uint64_t oracle_below(uint64_t *state, uint64_t m) {
    uint64_t r = oracle_splitmix64_next(state);
    unsigned __int128 p = (unsigned __int128)r * (unsigned __int128)m;
    return (uint64_t)(p >> 64);
}

/* Floyd's algorithm (Bentley and Floyd, CACM 1987) for k distinct indices of
 * [0, n): for j = n-k .. n-1 draw t uniform on [0, j]; keep t unless it was
 * already chosen, in which case keep j.  idx_out receives the indices in the
 * order they were kept.  Membership is a linear search: slow and plain.
 * Returns 0, or -1 if the arguments are out of range. */
int oracle_forgy_indices(int64_t n, int32_t k, uint64_t seed, int64_t *idx_out) {
    uint64_t state = seed;
    int32_t have = 0;
    int64_t j;
    if (n <= 0 || k <= 0 || (int64_t)k > n) return -1;
    for (j = n - k; j < n; ++j) {
        int64_t t = (int64_t)oracle_below(&state, (uint64_t)(j + 1));
        int32_t q, seen = 0;
        for (q = 0; q < have; ++q)
            if (idx_out[q] == t) { seen = 1; break; }
        idx_out[have++] = seen ? j : t;
    }
    return 0;
}

/* The library's FP32 squared distance, restated (see oracle_assign_f32 for
 * the order): two chains over even and odd coordinates, fmaf, then e + o. */
static float oracle_dist2_f32(const float *x, const float *c, int32_t d) {
    float e = 0.0f, o = 0.0f;
    int32_t q;
    for (q = 0; q < d; ++q) {
        float t = x[q] - c[q];
        if (q % 2 == 0) e = fmaf(t, t, e);
        else o = fmaf(t, t, o);
    }
    return e + o;
}

/* k-means++ seeding (Arthur and Vassilvitskii, SODA 2007; the paper lists it
 * among the variants to come): the first centroid is a uniformly drawn point,
 * every further one a point drawn with probability proportional to its
 * squared distance D^2 to the nearest centroid chosen so far.  Readings that
 * make a draw reproducible bit for bit:
 *   - D^2 is the FP32 squared distance above (the one every scan uses),
 *     between the FP32 rows of the point and of the chosen points;
 *   - the weights are D^2 quantised onto a power-of-two grid fixed per round:
 *     w(x) = floor(D^2(x) 2^E) with E = 32 - e, e the smallest integer with
 *     max D^2 < 2^e, so every weight is an exact integer below 2^32 and the
 *     total an exact 64-bit integer;
 *   - each draw is the next SplitMix64(seed) output r reduced by the
 *     multiply-shift: the first index floor(r n / 2^64), then t = floor(r T /
 *     2^64) with T the total weight, and the chosen point is the first whose
 *     running weight sum exceeds t (a point of weight 0 is never chosen);
 *   - if every weight is 0 (all points sit on chosen centroids) the next index
 *     is drawn uniformly like the first.
 * idx_out receives the k indices in the order drawn.  Returns 0, or -1 for
 * bad arguments. */
int oracle_kmeanspp_indices(const float *X, int64_t n, int32_t d, int32_t k, uint64_t seed,
                            int64_t *idx_out) {
    uint64_t state = seed;
    float *D2;
    uint64_t *w;
    int32_t j;
    int64_t i;
    if (n <= 0 || k <= 0 || d <= 0 || (int64_t)k > n) return -1;
    D2 = (float *)malloc((size_t)n * sizeof(float));
    w = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    idx_out[0] = (int64_t)oracle_below(&state, (uint64_t)n);
    for (i = 0; i < n; ++i) D2[i] = INFINITY;
    for (j = 1; j < k; ++j) {
        const float *c = X + (size_t)idx_out[j - 1] * d;
        float m = 0.0f;
        uint64_t T = 0, t, run = 0;
        int e = 0;
        for (i = 0; i < n; ++i) {
            float v = oracle_dist2_f32(X + (size_t)i * d, c, d);
            if (v < D2[i]) D2[i] = v;
            if (D2[i] > m) m = D2[i];
        }
        if (m > 0.0f) {
            (void)frexpf(m, &e); /* m = f 2^e, f in [0.5, 1): m < 2^e */
            for (i = 0; i < n; ++i) {
#ifdef ORACLE_PLANT_KPP_LINEAR /* weights in proportion to D instead of D^2 */
                w[i] = (uint64_t)floor(ldexp(sqrt((double)D2[i]) / sqrt((double)m), 32));
#else
                w[i] = (uint64_t)floor(ldexp((double)D2[i], 32 - e));
#endif
                T += w[i];
            }
        }
        if (T == 0) {
            idx_out[j] = (int64_t)oracle_below(&state, (uint64_t)n);
            continue;
        }
        t = oracle_below(&state, T);
        for (i = 0; i < n; ++i) {
            run += w[i];
            if (run > t) break;
        }
        idx_out[j] = i;
    }
    free(D2);
    free(w);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Distances ("Nomenclature").                                          */
/* ------------------------------------------------------------------ */

/* Squared Euclidean distance between FP32 point x and FP64 centroid c,
 * summed in index order in FP64. */
static double oracle_dist2(const float *x, const double *c, int32_t d) {
    double s = 0.0;
    int32_t i;
    for (i = 0; i < ORACLE_DIMS(d); ++i) {
        double t = (double)x[i] - c[i];
        s += t * t;
    }
    return s;
}

/* The squared distance over every dimension (used only to check the bounds,
 * so that a planted mistake in oracle_dist2 cannot hide itself). */
static double oracle_dist2_exactish(const float *x, const double *c, int32_t d) {
    double s = 0.0;
    int32_t i;
    for (i = 0; i < d; ++i) {
        double t = (double)x[i] - c[i];
        s += t * t;
    }
    return s;
}

static double oracle_dist2_cc(const double *a, const double *b, int32_t d) {
    double s = 0.0;
    int32_t i;
    for (i = 0; i < d; ++i) {
        double t = a[i] - b[i];
        s += t * t;
    }
    return s;
}

/* Relative error bound of the FP64 squared distance above, with room for the
 * square root and the scaling multiply: gamma_m = m*eps/(1-m*eps), m = 2d+8. */
static double oracle_gamma(int32_t d) {
    double m = 2.0 * (double)d + 8.0;
    return m * ORACLE_EPS64 / (1.0 - m * ORACLE_EPS64);
}

/* Upper bound on an exact distance from its computed square (reading R4). */
static double oracle_dist_up(double s2, double g) {
    return sqrt(s2) * (1.0 + 2.0 * g) + 1e-300;
}
/* Lower bound on an exact distance from its computed square (reading R4). */
static double oracle_dist_down(double s2, double g) {
    double v = sqrt(s2) * (1.0 - 2.0 * g) - 1e-300;
    return v > 0.0 ? v : 0.0;
}
/* Upper bound on the exact sum of two non-negative bounds. */
static double oracle_add_up(double a, double b) {
    return (a + b) * (1.0 + 8.0 * ORACLE_EPS64);
}

/* ------------------------------------------------------------------ */
/* Phase I (assignment) and Phase II (means) of Lloyd's algorithm.      */
/* ------------------------------------------------------------------ */

/* Nearest centroid of one point: scan c = 0..k-1 and replace the best only
 * when strictly closer, so ties keep the lowest index (Algorithm 1). */
static int32_t oracle_nearest(const float *x, const double *C, int32_t d, int32_t k,
                              double *best_d2) {
    int32_t c, best = 0;
    double bd = oracle_dist2(x, C, d);
    for (c = 1; c < k; ++c) {
        double v = oracle_dist2(x, C + (size_t)c * d, d);
#ifdef ORACLE_PLANT_TIE_HIGH         /* ties go to the highest index */
        if (v <= bd) { bd = v; best = c; }
#else
        if (v < bd) { bd = v; best = c; }
#endif
    }
    if (best_d2) *best_d2 = bd;
    return best;
}

/* Phase I for all points.  Also returns, per point, the two smallest squared
 * distances (d1 <= d2) and ||x||^2 + ||c_best||^2, which the parity rule uses
 * to recognise near-ties.  Any output pointer may be NULL. */
void oracle_assign(const float *X, int64_t n, int32_t d, int32_t k, const double *C,
                   int32_t *a_out, double *d1_out, double *d2_out, double *scale_out,
                   int nthreads) {
    int64_t i;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (i = 0; i < n; ++i) {
        const float *x = X + (size_t)i * d;
        int32_t c, best = 0;
        double b1 = INFINITY, b2 = INFINITY;
        for (c = 0; c < k; ++c) {
            double v = oracle_dist2(x, C + (size_t)c * d, d);
#ifdef ORACLE_PLANT_TIE_HIGH
            if (v <= b1) { b2 = b1; b1 = v; best = c; }
#else
            if (v < b1) { b2 = b1; b1 = v; best = c; }
#endif
            else if (v < b2) { b2 = v; }
        }
        if (a_out) a_out[i] = best;
        if (d1_out) d1_out[i] = b1;
        if (d2_out) d2_out[i] = b2;
        if (scale_out) {
            double xn = 0.0, cn = 0.0;
            int32_t q;
            for (q = 0; q < d; ++q) {
                xn += (double)x[q] * (double)x[q];
                cn += C[(size_t)best * d + q] * C[(size_t)best * d + q];
            }
            scale_out[i] = xn + cn;
        }
    }
}

/* Phase II: each centroid becomes the FP64 mean of its members; an empty
 * cluster keeps C_prev (reading R7).  The sum is recomputed from scratch.
 * As in ||Lloyd's, each thread sums a contiguous block of points into its own
 * copy and the copies are added in thread order afterwards. */
void oracle_means(const float *X, int64_t n, int32_t d, int32_t k, const int32_t *a,
                  const double *C_prev, double *C_out, int64_t *cnt_out) {
    double *S = (double *)calloc((size_t)k * d, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int nt = 1, t;
    int32_t c, q;
    double *St;
    int64_t *ct;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    St = (double *)calloc((size_t)nt * k * d, sizeof(double));
    ct = (int64_t *)calloc((size_t)nt * k, sizeof(int64_t));
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int me = 0, all = 1;
        int64_t lo, hi, i;
#ifdef _OPENMP
        me = omp_get_thread_num();
        all = omp_get_num_threads();
#endif
        lo = n * me / all;
        hi = n * (me + 1) / all;
        for (i = lo; i < hi; ++i) {
            const float *x = X + (size_t)i * d;
            int32_t ci = a[i], qq;
            ct[(size_t)me * k + ci] += 1;
            for (qq = 0; qq < d; ++qq) St[((size_t)me * k + ci) * d + qq] += (double)x[qq];
        }
    }
    for (t = 0; t < nt; ++t)
        for (c = 0; c < k; ++c) {
            cnt[c] += ct[(size_t)t * k + c];
            for (q = 0; q < d; ++q) S[(size_t)c * d + q] += St[((size_t)t * k + c) * d + q];
        }
    free(St);
    free(ct);
    for (c = 0; c < k; ++c) {
        for (q = 0; q < d; ++q) {
            size_t e = (size_t)c * d + q;
#ifdef ORACLE_PLANT_EMPTY_ZERO       /* empty clusters collapse to the origin */
            C_out[e] = cnt[c] > 0 ? S[e] / (double)cnt[c] : 0.0 * C_prev[e];
#else
            C_out[e] = cnt[c] > 0 ? S[e] / (double)cnt[c] : C_prev[e];
#endif
        }
        if (cnt_out) cnt_out[c] = cnt[c];
    }
    free(S);
    free(cnt);
}

/* Sum of squared distances of every point to its assigned centroid. */
double oracle_objective(const float *X, int64_t n, int32_t d, const double *C,
                        const int32_t *a) {
    double obj = 0.0;
    int64_t i;
    for (i = 0; i < n; ++i) obj += oracle_dist2(X + (size_t)i * d, C + (size_t)a[i] * d, d);
    return obj;
}

/* ------------------------------------------------------------------ */
/* MTI pruning ("Minimal Triangle Inequality (MTI) Pruning").           */
/* ------------------------------------------------------------------ */

/* Per-iteration centroid quantities, from the FP64 centroids:
 *   halfD[a*k+c] <= 1/2 d(c_a, c_c)   (c != a; the diagonal is unused)
 *   s[a]         <= 1/2 min_{c != a} d(c_a, c_c)   (+inf when k == 1)
 *   f[c]         >= d(c^t, c^{t-1})   (the drift; 0 when C_prev is NULL) */
void oracle_mti_tables(const double *C, const double *C_prev, int32_t d, int32_t k,
                       double *halfD, double *s, double *f) {
    double g = oracle_gamma(d);
    int32_t a, c;
    for (a = 0; a < k; ++a) {
        double m = INFINITY;
        for (c = 0; c < k; ++c) {
            double h;
            if (c == a) { halfD[(size_t)a * k + c] = 0.0; continue; }
            h = ORACLE_HALF * oracle_dist_down(oracle_dist2_cc(C + (size_t)a * d, C + (size_t)c * d, d), g);
            halfD[(size_t)a * k + c] = h;
            if (h < m) m = h;
        }
        s[a] = m;
        f[a] = C_prev ? oracle_dist_up(oracle_dist2_cc(C + (size_t)a * d, C_prev + (size_t)a * d, d), g)
                      : 0.0;
    }
}

/* One MTI iteration over all points, in the paper's clause order.
 *   a[i]   in: assignment from the previous iteration (-1: none yet)
 *          out: new assignment
 *   u[i]   in/out: upper bound on d(x_i, c_{a[i]}) (ignored while a[i] < 0)
 * The slack kappa and the absolute floor tau make every test strict with
 * room for the FP64 rounding of the distances it protects (reading R3), so
 * every pruned centroid is strictly farther, in computed FP64 values, than
 * the assigned one, and the result equals the unpruned scan exactly.
 * Counters (may be NULL): points skipped by Clause 1, distance evaluations. */
int64_t oracle_mti_iter(const float *X, int64_t n, int32_t d, int32_t k, const double *C,
                        const double *halfD, const double *s, const double *f,
                        int32_t *a, double *u, int64_t *skipped_out, int64_t *evals_out,
                        int nthreads) {
    double g = oracle_gamma(d);
    double kappa = 2.0 * g;
    double tau = 1e-280;
    int64_t changed = 0, skipped = 0, evals = 0;
    int64_t i;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static) reduction(+ : changed, skipped, evals)
#endif
    for (i = 0; i < n; ++i) {
        const float *x = X + (size_t)i * d;
        int32_t ai = a[i], c, best;
        double ui, bd;
        int tight = 0;
        if (ai < 0) {
            /* No assignment yet: a full scan (every distance is computed). */
            best = oracle_nearest(x, C, d, k, &bd);
            evals += k;
            a[i] = best;
            u[i] = oracle_dist_up(bd, g);
            changed += 1;
            continue;
        }
        /* u^t = u^{t-1} + f(c_a): the bound follows the centroid's drift. */
#ifdef ORACLE_PLANT_NO_DRIFT         /* the bound ignores centroid drift */
        ui = u[i];
#else
        ui = oracle_add_up(u[i], f[ai]);
#endif
        /* Clause 1: u below half the distance from c_a to every other
         * centroid, so v keeps its cluster and nothing else is read. */
        if (ui * (1.0 + kappa) + tau < s[ai]) {
            u[i] = ui;
            skipped += 1;
            continue;
        }
        best = ai;
        bd = 0.0; /* d^2(x, c_a) once computed */
        for (c = 0; c < k; ++c) {
            double v;
            if (c == ai) continue;
            /* Clause 2: the loose bound already rules c out. */
            if (ui * (1.0 + kappa) + tau < halfD[(size_t)ai * k + c]) continue;
            if (!tight) {
                /* Clause 3: tighten u to the exact d(v, c_a) and retest. */
                bd = oracle_dist2(x, C + (size_t)ai * d, d);
                evals += 1;
                ui = oracle_dist_up(bd, g);
                tight = 1;
                if (ui * (1.0 + kappa) + tau < halfD[(size_t)ai * k + c]) continue;
            }
            v = oracle_dist2(x, C + (size_t)c * d, d);
            evals += 1;
            /* Lowest index wins an exact tie, as in the unpruned scan. */
            if (v < bd || (v == bd && c < best)) { bd = v; best = c; }
        }
        if (best != ai) changed += 1;
        a[i] = best;
        u[i] = tight ? oracle_dist_up(bd, g) : ui;
    }
    if (skipped_out) *skipped_out = skipped;
    if (evals_out) *evals_out = evals;
    return changed;
}

/* ------------------------------------------------------------------ */
/* Elkan's algorithm: MTI plus per-centroid lower bounds.               */
/* ------------------------------------------------------------------ */

/* A lower bound on a - b for a >= 0, b >= 0 (0 when negative). */
static double oracle_sub_down(double a, double b) {
    double v = (a - b) * (1.0 - 8.0 * ORACLE_EPS64);
    return v > 0.0 ? v : 0.0;
}

/* One iteration of Elkan's algorithm (Elkan 2003, the source the paper cites
 * for its pruning; the paper's MTI keeps Elkan's first three tests and
 * leaves out the fourth, whose n x k lower bounds it finds too costly, and
 * does not measure it).  Besides MTI's upper bound u(x) >= d(x, c_a) every
 * point keeps lower bounds l(x, c) <= d(x, c), one per centroid, set when
 * the distance is computed and lowered by the centroid's drift each
 * iteration (triangle inequality).  A centroid is ruled out when u is below
 * 1/2 d(c_a, c) (MTI's Clause 2) or below l(x, c) (the fourth test); Clause 1
 * and the tightening of u (Clause 3) are MTI's.
 *   l        n*k lower bounds (row per point), updated in place
 *   a, u     as for oracle_mti_iter
 *   viol_out NULL, or receives the number of bounds found wrong before
 *            the tests use them: some l(x, c) above d(x, c), or u below
 *            d(x, c_a) (exact distances in FP64, with a rounding margin);
 *            always 0 for correct bounds.
 * Returns the number of points whose assignment changed. */
int64_t oracle_elkan_iter(const float *X, int64_t n, int32_t d, int32_t k, const double *C,
                          const double *halfD, const double *s, const double *f, int32_t *a,
                          double *u, double *l, int64_t *skipped_out, int64_t *evals_out,
                          int64_t *viol_out, int nthreads) {
    double g = oracle_gamma(d);
    double kappa = 2.0 * g;
    double tau = 1e-280;
    int64_t changed = 0, skipped = 0, evals = 0, viol = 0;
    int64_t i;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static) reduction(+ : changed, skipped, evals, viol)
#endif
    for (i = 0; i < n; ++i) {
        const float *x = X + (size_t)i * d;
        double *li = l + (size_t)i * k;
        int32_t ai = a[i], c, best;
        double ui, bd;
        int tight = 0;
        if (ai < 0) {
            /* No assignment yet: every distance, and every lower bound. */
            best = 0;
            bd = INFINITY;
            for (c = 0; c < k; ++c) {
                double v = oracle_dist2(x, C + (size_t)c * d, d);
                li[c] = oracle_dist_down(v, g);
                if (v < bd) { bd = v; best = c; }
            }
            evals += k;
            a[i] = best;
            u[i] = oracle_dist_up(bd, g);
            changed += 1;
            continue;
        }
        ui = oracle_add_up(u[i], f[ai]);
#ifndef ORACLE_PLANT_ELKAN_NO_LB_DRIFT /* lower bounds ignore centroid drift */
        for (c = 0; c < k; ++c) li[c] = oracle_sub_down(li[c], f[c]);
#endif
        if (viol_out) {
            for (c = 0; c < k; ++c) {
                double e = sqrt(oracle_dist2_exactish(x, C + (size_t)c * d, d));
                if (li[c] > e * (1.0 + 4.0 * g) + 1e-300) viol += 1;
                if (c == ai && ui < e * (1.0 - 4.0 * g)) viol += 1;
            }
        }
        /* Clause 1: nothing else is read. */
        if (ui * (1.0 + kappa) + tau < s[ai]) {
            u[i] = ui;
            skipped += 1;
            continue;
        }
        best = ai;
        bd = 0.0;
        for (c = 0; c < k; ++c) {
            double v, thr;
            if (c == ai) continue;
            /* Clause 2 (1/2 d(c_a, c)) and the fourth test (l(x, c)). */
            thr = halfD[(size_t)ai * k + c] > li[c] ? halfD[(size_t)ai * k + c] : li[c];
            if (ui * (1.0 + kappa) + tau < thr) continue;
            if (!tight) {
                /* Clause 3: tighten u to the exact d(v, c_a) and retest. */
                bd = oracle_dist2(x, C + (size_t)ai * d, d);
                evals += 1;
                ui = oracle_dist_up(bd, g);
                li[ai] = oracle_dist_down(bd, g);
                tight = 1;
                if (ui * (1.0 + kappa) + tau < thr) continue;
            }
            v = oracle_dist2(x, C + (size_t)c * d, d);
            evals += 1;
            li[c] = oracle_dist_down(v, g);
            if (v < bd || (v == bd && c < best)) { bd = v; best = c; }
        }
        if (best != ai) changed += 1;
        a[i] = best;
        u[i] = tight ? oracle_dist_up(bd, g) : ui;
    }
    if (skipped_out) *skipped_out = skipped;
    if (evals_out) *evals_out = evals;
    if (viol_out) *viol_out = viol;
    return changed;
}

/* ------------------------------------------------------------------ */
/* A whole run.                                                         */
/* ------------------------------------------------------------------ */

/* Lloyd's algorithm from C0 for at most max_iters iterations, stopping after
 * the first iteration in which no assignment changes (reading R6).
 *   prune       0: unpruned scans; 1: MTI; 2: Elkan (MTI plus lower bounds).
 *   C_out       k*d final centroids.
 *   a_out       n final assignments.
 *   a_hist      NULL or max_iters*n: assignments after each iteration.
 *   C_hist      NULL or (max_iters+1)*k*d: C^0 then the centroids after each
 *               iteration.
 *   changed/skipped/evals  NULL or max_iters per-iteration counters.
 *   viol_out    NULL or max_iters: Elkan's bound check (see oracle_elkan_iter);
 *               0 for the other modes.
 * Returns the number of iterations executed. */
int oracle_run(const float *X, int64_t n, int32_t d, int32_t k, const double *C0,
               int32_t max_iters, int prune, double *C_out, int32_t *a_out,
               int32_t *a_hist, double *C_hist, int64_t *changed_out, int64_t *skipped_out,
               int64_t *evals_out, int64_t *viol_out, int nthreads) {
    size_t kd = (size_t)k * d;
    double *C = (double *)malloc(kd * sizeof(double));
    double *Cp = (double *)malloc(kd * sizeof(double));
    double *Cn = (double *)malloc(kd * sizeof(double));
    double *halfD = (double *)malloc((size_t)k * k * sizeof(double));
    double *s = (double *)malloc((size_t)k * sizeof(double));
    double *f = (double *)malloc((size_t)k * sizeof(double));
    int32_t *a = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *an = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    double *u = (double *)malloc((size_t)n * sizeof(double));
    double *l = prune == 2 ? (double *)malloc((size_t)n * k * sizeof(double)) : NULL;
    int32_t t, iters = 0;
    int64_t i;
    memcpy(C, C0, kd * sizeof(double));
    if (C_hist) memcpy(C_hist, C0, kd * sizeof(double));
    for (i = 0; i < n; ++i) { a[i] = -1; u[i] = INFINITY; }
    for (t = 0; t < max_iters; ++t) {
        int64_t changed = 0, skipped = 0, evals = 0, viol = 0;
        if (prune == 2) {
            oracle_mti_tables(C, t > 0 ? Cp : NULL, d, k, halfD, s, f);
            changed = oracle_elkan_iter(X, n, d, k, C, halfD, s, f, a, u, l, &skipped, &evals,
                                        viol_out ? &viol : NULL, nthreads);
        } else if (prune) {
            oracle_mti_tables(C, t > 0 ? Cp : NULL, d, k, halfD, s, f);
            changed = oracle_mti_iter(X, n, d, k, C, halfD, s, f, a, u, &skipped, &evals,
                                      nthreads);
        } else {
            oracle_assign(X, n, d, k, C, an, NULL, NULL, NULL, nthreads);
            for (i = 0; i < n; ++i) {
                if (an[i] != a[i]) changed += 1;
                a[i] = an[i];
            }
            evals = n * (int64_t)k;
        }
        oracle_means(X, n, d, k, a, C, Cn, NULL);
        memcpy(Cp, C, kd * sizeof(double));
        memcpy(C, Cn, kd * sizeof(double));
        if (a_hist) memcpy(a_hist + (size_t)t * n, a, (size_t)n * sizeof(int32_t));
        if (C_hist) memcpy(C_hist + (size_t)(t + 1) * kd, C, kd * sizeof(double));
        if (changed_out) changed_out[t] = changed;
        if (skipped_out) skipped_out[t] = skipped;
        if (evals_out) evals_out[t] = evals;
        if (viol_out) viol_out[t] = viol;
        iters = t + 1;
        if (changed == 0) break;
    }
    memcpy(C_out, C, kd * sizeof(double));
    memcpy(a_out, a, (size_t)n * sizeof(int32_t));
    free(C); free(Cp); free(Cn); free(halfD); free(s); free(f);
    free(a); free(an); free(u); free(l);
    return iters;
}

/* The assignment decision restated in FP32, for callers that want to compare
 * an FP32 argmin in the same precision.  The paper computes in FP64 and fixes
 * no FP32 summation order; this restates the order the library documents for
 * its FP32 distance: two chains, e over even i and o over odd i, each in
 * increasing i with e (or o) = fmaf(x_i - c_i, x_i - c_i, e), then
 * d^2 = e + o; every operation rounded to nearest FP32; lowest index wins
 * ties. */
void oracle_assign_f32(const float *X, int64_t n, int32_t d, int32_t k, const float *C32,
                       int32_t *a_out, int nthreads) {
    int64_t i;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (i = 0; i < n; ++i) {
        const float *x = X + (size_t)i * d;
        int32_t c, q, best = 0;
        float bd = INFINITY;
        for (c = 0; c < k; ++c) {
            float e = 0.0f, o = 0.0f, acc;
            for (q = 0; q < d; ++q) {
                float t = x[q] - C32[(size_t)c * d + q];
                if (q % 2 == 0) e = fmaf(t, t, e);
                else o = fmaf(t, t, o);
            }
            acc = e + o;
            if (acc < bd) { bd = acc; best = c; }
        }
        a_out[i] = best;
    }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

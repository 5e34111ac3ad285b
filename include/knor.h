/*
 * knor.h -- C ABI of libknor.so: Lloyd's k-means with MTI pruning on one
 * GB300 (sm_103a).
 *
 * Paper: Mhembere, Zheng, Priebe, Vogelstein, Burns, "knor: A NUMA-Optimized
 * In-Memory, Distributed and Semi-External-Memory k-means Library", HPDC'17,
 * arXiv 1606.08905.  Section references below are to that paper:
 *   "Nomenclature"                        V in R^{n x d}, k, iteration t,
 *                                         Euclidean d(v, c), drift f(c^t)
 *   "Parallel Lloyd's Algorithm"          Phase I / Phase II, Algorithm 1
 *   "Minimal Triangle Inequality (MTI)
 *    Pruning"                             Clauses 1-3, the upper bound u^t
 *   "Asymptotic Memory Consumption"       the k x k centroid table, O(n) bound
 *
 * Conventions (every function):
 *   - Returns a knor_status; never aborts the process.  On error the context
 *     stays valid and destroyable, and knor_last_error() describes the error.
 *   - Pointers marked "host or device" may point to host memory (pageable or
 *     pinned) or to device memory of the context's GPU; the library tells
 *     them apart with cudaPointerGetAttributes.  Inputs are copied (except the
 *     points under knor_opts.points_in_host); the caller keeps ownership of
 *     every buffer it passes.  Outputs go to caller-owned
 *     buffers and are complete when the call returns.
 *   - All arrays are dense and row-major.  Points are FP32; centroids are
 *     returned as FP64 (the master copy) or FP32 (the copy the scan used).
 *   - A context is not thread-safe.  It owns all its device memory and one
 *     CUDA stream, created on the device current at knor_create.
 *   - Assignments follow Algorithm 1's scan: the nearest centroid, ties to the
 *     lowest index.  Iteration 1 starts from "no assignment", so every point
 *     counts as changed in it.
 *   - Tuning switches, read from the environment by knor_create, change how
 *     the work is grouped, not the assignments or centroids: KNOR_SEL_M (Clause-1
 *     selection: a point whose bound would leave it this many Clause-2
 *     candidates or more is scored against every centroid in a batch of its
 *     own; default k / 3 from k = 8 on, 0 never), KNOR_SEL_MULT=1 (one
 *     selection warp per scan warp instead of two where two fit),
 *     KNOR_MTI_KERNEL=1 (the one-kernel MTI scan instead of the split
 *     selection / scan / delta kernels).
 */
#ifndef KNOR_H
#define KNOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct knor_ctx knor_ctx; /* opaque; owns all device memory */

typedef enum {
    KNOR_OK = 0,
    KNOR_ERR_ARG = -1,     /* invalid argument (sizes, NULL, NaN/Inf input, ...) */
    KNOR_ERR_OOM = -2,     /* a device or host allocation failed */
    KNOR_ERR_CUDA = -3,    /* a CUDA call failed; the message names it */
    KNOR_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up */
    KNOR_ERR_STATE = -5    /* call not valid in the context's current state */
} knor_status;

typedef enum {
    KNOR_INIT_FORGY = 0,    /* k distinct rows chosen from the seed (below) */
    KNOR_INIT_EXPLICIT = 1, /* caller supplies C^0 with knor_set_init_centroids */
    KNOR_INIT_KMEANSPP = 2  /* k-means++ seeding from the seed (below) */
} knor_init;

typedef enum {
    KNOR_PREC_FP32 = 0, /* FP32 distances, direct form sum_i (x_i - c_i)^2 */
    KNOR_PREC_BF16 = 1, /* tensor-core BF16 distance block + exact FP32 recheck */
    KNOR_PREC_FP8 = 2,  /* tensor-core FP8 e4m3 (power-of-two per-dimension scales,
                           x_j / sigma_j and c_j sigma_j) + exact FP32 recheck; d = 128 */
    KNOR_PREC_FP16 = 3  /* tensor-core FP16 distance block (points and centroids
                           scaled by powers of two into range) + exact FP32 recheck */
} knor_precision;
/* Every tensor-core form returns exactly the assignments of KNOR_PREC_FP32:
 * a point whose two smallest approximate distances are further apart than
 * twice a proven bound on their error keeps the approximate argmin, every
 * other point is re-scored in FP32 over the centroids that can still be
 * nearest.  They need d = 64 or 128 (FP8: 128); k is limited by shared memory
 * (8192 at d = 128).  They never prune (every point is scanned each
 * iteration). */

/* Options.  A zero-initialised struct gives the defaults: MTI pruning on,
 * FP32 distances, sums maintained by deltas, no debug checks. */
typedef struct {
    int32_t no_prune;             /* 0: MTI pruning; 1: plain Lloyd (every distance) */
    int32_t precision;            /* knor_precision */
    int32_t full_recompute_every; /* 0: never; m > 0: rebuild the cluster sums
                                     from all points every m-th iteration */
    int32_t debug_invariants;     /* 1: after each MTI iteration, check on the
                                     GPU that every bound u >= d(x, c_a) (with
                                     elkan, also every lower bound) and count
                                     violations into knor_iter_stats.violations */
    int32_t elkan;                /* 1: Elkan's algorithm instead of MTI -- MTI's
                                     tests plus a lower bound l(x, c) per point and
                                     centroid (the fourth test, which the paper's
                                     MTI leaves out: c is ruled out when u <
                                     l(x, c)); an ablation that keeps an n x k FP32
                                     matrix (4nk bytes).  Needs FP32 distances,
                                     pruning, full_recompute_every = 0, d in {8,
                                     16, 32, 64}, k <= 110 and k*d <= 8192;
                                     KNOR_ERR_ARG otherwise.  Assignments equal
                                     MTI's and plain Lloyd's. */
    int32_t points_in_host;       /* 1: the points stay where the caller has them,
                                     in host memory (pinned or pageable; a pageable
                                     buffer is registered with the CUDA driver for
                                     the context's lifetime): no n x d copy in HBM,
                                     the scans read rows over the host link (NVLink-
                                     C2C on Grace), so the rows Clause 1 skips are
                                     never transferred -- the in-memory analogue of
                                     the paper's semi-external mode.  The caller
                                     keeps the buffer alive and unchanged until
                                     knor_destroy.  Needs FP32 distances, a 16-byte
                                     aligned host buffer; KNOR_ERR_ARG otherwise
                                     (or if points is device memory). */
} knor_opts;

/* Per-iteration counters. */
typedef struct {
    int64_t changed;         /* points whose assignment changed */
    int64_t clause1_skipped; /* points skipped by MTI Clause 1 (nothing read) */
    int64_t dist_evals;      /* point-centroid distances computed */
    int64_t rechecked;       /* precision forms: rows re-scored exactly in FP32 */
    int32_t empty;           /* clusters with no member after the iteration */
    int32_t iteration;       /* 1-based iteration number */
    int64_t violations;      /* debug_invariants: MTI bounds found below the true distance,
                                or (precision forms) points whose assignment differs from a
                                full FP32 scan; precision forms always: points left without a
                                new assignment; batched form always: points that found their
                                cluster's segment full (the sort-segmented MTI scan).  Always 0
                                unless the library is faulty. */
} knor_iter_stats;

/* Creates a context holding a copy of the n x d FP32 points (host or device)
 * and the initial centroids C^0.
 *   init = KNOR_INIT_FORGY: C^0 = rows idx[0..k-1] in drawn order, where idx
 *     are k distinct indices of [0, n) drawn by Floyd's sampling algorithm
 *     (for j = n-k .. n-1: t = floor(r * (j+1) / 2^64) with r the next
 *     SplitMix64 output of state `seed`; keep t unless already kept, else j).
 *     The paper states no initialisation; this one is reproducible.
 *   init = KNOR_INIT_KMEANSPP: k-means++ (Arthur and Vassilvitskii 2007; the
 *     paper names it among the variants to come), reproducible bit for bit:
 *     with r_1, r_2, ... the SplitMix64 outputs of state `seed` and
 *     below(r, m) = floor(r * m / 2^64), the first index is below(r_1, n);
 *     then D^2(x) = min over the chosen points p of the FP32 squared distance
 *     of the scans (even/odd fma chains) between the rows x and p; with e the
 *     smallest integer such that max D^2 < 2^e, the weights are
 *     w(x) = floor(D^2(x) * 2^(32 - e)) and T their sum; the next index is the
 *     first point whose running weight sum exceeds below(r_j, T), or
 *     below(r_j, n) when T = 0.  C^0 = the rows in drawn order.
 *   init = KNOR_INIT_EXPLICIT: C^0 must be set with knor_set_init_centroids
 *     before the first iteration (KNOR_ERR_STATE otherwise).
 * Errors: KNOR_ERR_ARG if points or out is NULL, n < 1, d < 1, k < 1, k > n,
 * n > 2^31, n*d > 2^40, or any coordinate is NaN, infinite or of magnitude above 1e15
 * (so no squared distance can overflow FP32).  opts may be NULL (defaults).
 * On success *out owns the context; free it with knor_destroy. */
knor_status knor_create(const float *points, int64_t n, int32_t d, int32_t k, knor_init init,
                        uint64_t seed, const knor_opts *opts, knor_ctx **out);

/* Sets C^0 (k x d FP64, host or device) and resets the run: no assignment, u
 * unset, iteration 0.  Valid for any init mode.  Coordinates must be finite. */
knor_status knor_set_init_centroids(knor_ctx *ctx, const double *c_kxd);

/* Returns the context to C^0 and iteration 0 (no assignment). */
knor_status knor_reset(knor_ctx *ctx);

/* One Lloyd iteration ("Parallel Lloyd's Algorithm"): Phase I with MTI
 * pruning (Clauses 1-3) unless no_prune, then Phase II (means; an empty
 * cluster keeps its centroid).  `out` may be NULL. */
knor_status knor_iterate(knor_ctx *ctx, knor_iter_stats *out);

/* Iterates until an iteration changes no assignment or max_iters iterations
 * have run in this call (the paper's "repeat until converged").  The loop
 * runs on the device (one CUDA graph launch).  *iters_done (may be NULL)
 * receives the number of iterations executed, including the final one that
 * changed nothing; per_iter (may be NULL) must hold max_iters records. */
knor_status knor_run(knor_ctx *ctx, int32_t max_iters, int32_t *iters_done,
                     knor_iter_stats *per_iter);

/* Current assignments, n int32 (host or device buffer).  -1 before the first
 * iteration. */
knor_status knor_get_assignments(const knor_ctx *ctx, int32_t *out_n);

/* Current centroids: the FP64 master copy (k x d) or the FP32 copy (k x d,
 * each the FP64 value rounded to nearest) that the next scan uses.  Host or
 * device buffers. */
knor_status knor_get_centroids(const knor_ctx *ctx, double *out_kxd);
knor_status knor_get_centroids_f32(const knor_ctx *ctx, float *out_kxd);

/* The Forgy or k-means++ row indices (k int64, host buffer), in drawn order.
 * KNOR_ERR_STATE for KNOR_INIT_EXPLICIT contexts. */
knor_status knor_get_init_indices(const knor_ctx *ctx, int64_t *out_k);

/* Iterations completed since the last reset. */
knor_status knor_get_iteration(const knor_ctx *ctx, int32_t *out);

/* The CUDA stream (a cudaStream_t) every kernel of this context runs on. */
void *knor_stream(const knor_ctx *ctx);

/* Per-kernel timing.  With profiling on, knor_iterate and knor_run launch the
 * iteration's kernels one by one (no graph; the run loop moves to the host,
 * one synchronisation per iteration) and bracket each with CUDA events on the
 * context's stream.  knor_get_profile returns the launches and the summed
 * event durations per kernel since the last reset of the profile
 * (reset_after = 1 clears them after reading). */
typedef enum {
    KNOR_KERNEL_DENSE = 0,  /* full scan + fresh sums (plain Lloyd, MTI iteration 1);
                               the certifying tensor-core scan of all points in the
                               precision form */
    KNOR_KERNEL_MTI = 1,    /* Clause-1 test + pruned scan + delta sums */
    KNOR_KERNEL_REDUCE = 2, /* ordered FP64 merge of per-CTA sums, new centroids */
    KNOR_KERNEL_TABLE = 3,  /* drift, k x k half-distance table, s(c) */
    KNOR_KERNEL_RECHECK = 4, /* precision form: the uncertified points -- gather, tensor-core
                                candidate pass, exact FP32 re-score of the candidates */
    KNOR_KERNEL_SUMS = 5,   /* precision form: delta cluster sums of the changed points */
    KNOR_KERNEL_SELECT = 6, /* split MTI scan: Clause 1 and the per-cluster batch records
                               (KNOR_KERNEL_MTI is then the scan of those records) */
    KNOR_KERNEL_DELTA = 7,  /* split scans: cluster sums moved by the rows of the points
                               that changed cluster */
    KNOR_KERNEL_COUNT = 8
} knor_kernel;
typedef struct {
    int64_t launches[KNOR_KERNEL_COUNT];
    double ms[KNOR_KERNEL_COUNT];
} knor_profile;
knor_status knor_set_profiling(knor_ctx *ctx, int32_t on);
/* Name of the CUDA kernel that implements `kernel` (a knor_kernel) for this
 * context, e.g. "k_mti_w<32>": the variant chosen from d and the shared-memory
 * footprint of k x d.  Valid for the context's lifetime; "" for bad input. */
const char *knor_kernel_name(const knor_ctx *ctx, int32_t kernel);
knor_status knor_get_profile(knor_ctx *ctx, knor_profile *out, int32_t reset_after);

/* Checkpoint.  knor_get_state with buf == NULL stores the needed size in
 * *size; otherwise it writes the state (header, FP64 centroids and sums,
 * counts, drift table, assignments and bounds) into the host buffer buf of
 * *size bytes.  knor_set_state restores a state taken from a context with the
 * same n, d, k and options; continuing from it reproduces the original run
 * bit for bit. */
knor_status knor_get_state(const knor_ctx *ctx, void *buf, size_t *size);
knor_status knor_set_state(knor_ctx *ctx, const void *buf, size_t size);

/* One plain Lloyd step on caller-owned device buffers, allocating no device
 * memory.  (Not from the paper, which has no counterpart: it exists for
 * callers that cannot allocate, such as code whose device memory belongs to
 * another allocator that has reserved most of HBM, or loops that must not
 * call cudaMalloc/cudaFree because those calls synchronise the device.)
 *   points      n x d FP32, device
 *   centroids   k x d FP32, device: the centroids of this step
 *   assign_out  n int32, device: nearest centroid of each point (FP32
 *               direct-form distance, lowest index on ties; the same values
 *               knor_iterate computes from the same FP32 centroids)
 *   sums_out    k x d FP64, device: per-cluster sums of the assigned points
 *   counts_out  k int64, device: per-cluster member counts
 *   stream      cudaStream_t to run on (NULL: the legacy default stream);
 *               the call returns after the stream has finished the step.
 * The means are sums_out / counts_out (the caller keeps the old centroid of
 * an empty cluster).  Working memory is a fixed 8 MiB array inside the
 * library's device image, held by every GPU that loads the library until the
 * process exits; it limits k * (d + 1) to 4096 (larger sizes return
 * KNOR_ERR_ARG).  The first call on each device looks the array's device
 * address up (cudaGetSymbolAddress).  All calls share the array: calls that overlap on
 * the GPU (other streams, other threads) race and give wrong results.
 * Errors: KNOR_ERR_ARG for NULL or non-device buffers and bad sizes,
 * KNOR_ERR_CUDA for CUDA failures; the message is knor_last_error(NULL). */
knor_status knor_lloyd_step_noalloc(const float *points, int64_t n, int32_t d, int32_t k,
                                    const float *centroids, int32_t *assign_out, double *sums_out,
                                    int64_t *counts_out, void *stream);

/* Fault injection, for tests of the error paths (the paper has no
 * counterpart).  They make a failure happen on the host; neither faults,
 * traps nor blocks the GPU.
 *   knor_test_fail_alloc(after): the device allocation made after `after`
 *     more successful ones (0: the next one) fails as if the device were out
 *     of memory (the call reports KNOR_ERR_OOM); once only.  after < 0
 *     cancels a pending failure.  Process-wide.
 *   knor_test_raise_error_flag(ctx): sets the context's device error flag,
 *     the flag a bounded device-side wait sets when it gives up; the next
 *     knor_iterate / knor_run then returns KNOR_ERR_TIMEOUT and clears it. */
knor_status knor_test_fail_alloc(int32_t after);
knor_status knor_test_raise_error_flag(knor_ctx *ctx);

/* Measurement helper (the paper has no counterpart: it measures the roof that
 * the FP32-bound scans are judged against).  Times, with CUDA events on a
 * private stream of the current device, a kernel that issues only fused
 * multiply-adds (eight independent chains per thread, 8 CTAs of 256 threads
 * per SM): kind 0 FP32 fma.rn.f32, 1 packed fma.rn.f32x2 (two FP32 FMAs per
 * instruction), 2 FP64.  *tflops_out receives the best of three timed runs
 * after one warm-up, counting 2 flops per FMA; *ms_out (may be NULL) that
 * run's time.  Allocates nothing on the device.  Errors: KNOR_ERR_ARG (bad
 * kind or NULL output), KNOR_ERR_CUDA; message from knor_last_error(NULL). */
knor_status knor_probe_alu(int32_t kind, double *tflops_out, float *ms_out);

/* Message for the last error on this context ("" if none).  Valid until the
 * next call on the context.  ctx may be NULL for errors of knor_create. */
const char *knor_last_error(const knor_ctx *ctx);

/* Frees the context and all its device memory.  NULL is ignored. */
void knor_destroy(knor_ctx *ctx);

/* Library version, "major.minor.patch". */
const char *knor_version(void);

/* ------------------------------------------------------------------------
 * Batched form: m independent problems advanced together.
 *
 * Each step runs one Lloyd iteration (with MTI pruning unless opts->no_prune)
 * of every instance that has not converged, as one persistent scan launch
 * over work units (instance, point range) taken longest-first from a device
 * queue -- the GPU counterpart of the paper's task queue with work stealing
 * ("Parallel Lloyd's Algorithm"; NUMA-aware task scheduling) -- followed by
 * batched merge and table launches.  An instance gets the same assignments
 * it would get alone from the same centroids; its sums are updated by FP64
 * atomics, so centroids agree with the single-instance path to FP64
 * rounding (not bit for bit).  An instance whose iteration changed no point
 * is converged and skipped from then on.
 * ---------------------------------------------------------------------- */
typedef struct knor_batch knor_batch;

typedef struct {
    int64_t n;             /* points */
    int32_t d, k;
    int32_t iterations;    /* iterations run since the last reset */
    int32_t converged;     /* 1 once an iteration changed no assignment */
    int64_t changed_last;  /* points that changed cluster in its last iteration */
} knor_batch_instance;

/* points[i]: row-major n[i] x d[i] FP32 (host or device, copied; the caller
 * keeps ownership).  Limits per instance: 1 <= k[i] <= min(n[i], 256), d[i]
 * in {8, 16, 32, 64}; coordinates finite with |x| <= 1e15.  C^0 of instance
 * i is Forgy with seed + i (as knor_create with that seed).  opts: NULL or
 * FP32 distances with full_recompute_every = 0 (no_prune selects plain
 * Lloyd).  Creation tunes the work-unit size per (d, k) bucket and the CTAs
 * per SM by timing dry scans (set KNOR_AUTOTUNE=0 to skip; results are cached
 * per device and bucket for the process and, if KNOR_AUTOTUNE_CACHE names a
 * file, across processes).  Errors: KNOR_ERR_ARG (message from
 * knor_last_error(NULL)), KNOR_ERR_OOM, KNOR_ERR_CUDA. */
knor_status knor_batch_create(int32_t m, const float *const *points, const int64_t *n, const int32_t *d,
                              const int32_t *k, uint64_t seed, const knor_opts *opts, knor_batch **out);
/* C^0 of one instance, k x d FP64 (host or device); resets the whole batch
 * to iteration 0. */
knor_status knor_batch_set_init_centroids(knor_batch *b, int32_t instance, const double *c_kxd);
/* Back to C^0 for every instance. */
knor_status knor_batch_reset(knor_batch *b);
/* One iteration of every active instance; *out (may be NULL) sums the
 * counters over the instances that ran. */
knor_status knor_batch_iterate(knor_batch *b, knor_iter_stats *out);
/* Up to max_iters iterations as one graph launch, stopping on the device once
 * every instance has converged; per_iter (NULL or max_iters records) as for
 * knor_iterate. */
knor_status knor_batch_run(knor_batch *b, int32_t max_iters, int32_t *iters_done, knor_iter_stats *per_iter);
/* Per-instance results into caller buffers (host or device): n int32
 * assignments, k x d FP64 centroids, k x d FP32 scan copy, k int64 Forgy
 * indices, and the instance record. */
knor_status knor_batch_get_assignments(const knor_batch *b, int32_t instance, int32_t *out_n);
knor_status knor_batch_get_centroids(const knor_batch *b, int32_t instance, double *out_kxd);
knor_status knor_batch_get_centroids_f32(const knor_batch *b, int32_t instance, float *out_kxd);
knor_status knor_batch_get_init_indices(const knor_batch *b, int32_t instance, int64_t *out_k);
knor_status knor_batch_get_instance(const knor_batch *b, int32_t instance, knor_batch_instance *out);
/* Work since the last reset: point-iterations (sum over the iterations of the
 * points of every instance that ran in it) and the scan's algorithmic bytes
 * (8 per point for the state read; 4d + 8 more per point not skipped by
 * Clause 1: its row and the state write). */
knor_status knor_batch_get_work(const knor_batch *b, int64_t *point_iterations, int64_t *scan_bytes);
/* Profiling as for a context; the batch fills the KNOR_KERNEL_MTI (scan),
 * KNOR_KERNEL_REDUCE (merge) and KNOR_KERNEL_TABLE (bookkeeping + table)
 * slots. */
knor_status knor_batch_set_profiling(knor_batch *b, int32_t on);
knor_status knor_batch_get_profile(knor_batch *b, knor_profile *out, int32_t reset_after);
const char *knor_batch_kernel_name(const knor_batch *b, int32_t kernel);
/* The tuned launch shape, as text (valid for the batch's lifetime). */
const char *knor_batch_describe(const knor_batch *b);
/* The batch's CUDA stream (cudaStream_t). */
void *knor_batch_stream(const knor_batch *b);
const char *knor_batch_last_error(const knor_batch *b);
void knor_batch_destroy(knor_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* KNOR_H */

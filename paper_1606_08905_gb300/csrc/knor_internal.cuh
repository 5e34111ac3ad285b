// knor_internal.cuh -- types and launch parameters shared by the kernels and
// the host runtime of libknor.so.  Not part of the public ABI (include/knor.h).
#pragma once
#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

namespace knor {

// Threads per CTA of the point kernels, and points per row tile.
constexpr int NT = 256;
// Points tested per thread and step by the MTI bound test (phase A).
constexpr int PA = 8;
// Capacity of the MTI active-point ring queue (leftover < NT plus one chunk).
constexpr int QCAP = NT * PA + NT;

// Warp-autonomous kernels (k_dense_w, k_mti_w): warps per CTA, points per
// lane and per warp chunk of the bound test, capacity of each per-cluster
// bucket of k_mti_w (fewer than 32 left plus one append of 32; a power of
// two, used as a ring) and state chunks in flight per warp.
constexpr int WPC = 4;
constexpr int WPA = 4;
constexpr int WCH = 32 * WPA;
constexpr int WBCAP = 64;
constexpr int WSTAGES = 2;

// Split MTI scan: ints per batch record (144 bytes, 16-byte aligned:
// cluster, count, two unused, 32 point indices).
constexpr int SP_REC = 36;
#ifndef KNOR_SP_WPB
#define KNOR_SP_WPB 4
#endif
constexpr int SP_WPB = KNOR_SP_WPB; // warps per CTA of both split kernels
#ifndef KNOR_DS_P
#define KNOR_DS_P 1
#endif
constexpr int DS_ROWS = 32 * KNOR_DS_P; // rows per tile of the split dense scan (KNOR_DS_P per lane)

// Per-point MTI state, packed so that the bound test reads 8 bytes per point.
//   a   assignment (-1 before the first iteration)
//   ub  u - F[a] rounded up, where u >= d(x, c_a) was exact-plus-rounding when
//       stored and F[a] is the cluster's cumulative drift at that time.  The
//       current bound is u^t = ub + F^t[a] (rounded up): the paper's running
//       update u^t = u^{t-1} + f(c_a) without rewriting ub every iteration.
struct __align__(8) PtState {
    float ub;
    int32_t a;
};

// Device counters of the iteration in flight (zeroed when snapshotted).
struct Counters {
    unsigned long long changed;
    unsigned long long skipped;
    unsigned long long evals;
    unsigned long long rechecked;
    unsigned long long empty;
    unsigned long long violations;
};

// One record per completed iteration; layout identical to knor_iter_stats.
struct IterStats {
    long long changed;
    long long clause1_skipped;
    long long dist_evals;
    long long rechecked;
    int32_t empty;
    int32_t iteration;
    long long violations;
};

// Parameters of the point kernels (dense scan and MTI scan).
struct IterParams {
    const float *X;        // n x d points
    int64_t n;
    int32_t d, k;
    PtState *st;           // n
    const float *C32;      // k x d current centroids (FP32 scan copy)
    const float *halfD;    // k x k, lower bounds on 1/2 d(c_a, c)
    const float *s;        // k, lower bounds on 1/2 min_{c != a} d(c_a, c)
    const float *F;        // k, cumulative drift (upper bound)
    double *part_S;        // [k*d][part_stride] per-CTA FP64 partial sums
    long long *part_cnt;   // [k][part_stride]  per-CTA member-count partials
    int32_t part_stride;   // = number of partial slots (grid size, or 1)
    Counters *ctr;
    float onepk;           // 1 + kappa, rounded up: pruning slack
    float tau;             // absolute pruning floor
    float g_up;            // >= 1 / (1 - (d+2) 2^-24): FP32 distance error bound
    float tiny;            // >= d * 2^-149: underflow allowance
    int32_t acc_global;    // 1: cluster sums go straight to part_S slot 0 by FP64 atomics
    int32_t cent_smem;     // 1: centroids staged in shared memory
    int32_t halfD_smem;    // 1: k x k table staged in shared memory
    int32_t mti;           // dense kernel: also write the MTI bound
    // shared-memory layout (byte offsets; off_s / off_F are -1 when the
    // per-cluster arrays are read from global memory instead)
    int32_t off_acc_hi, off_acc_lo, off_cnt, off_cent, off_halfD, off_s, off_F;
    int32_t off_tb, off_ta, off_ti, off_tile, off_queue, off_misc;
    int32_t dpad;          // floats per staged row (d + 4)
    int32_t stages;        // row tiles in flight (dense kernel)
    // warp-autonomous kernels: warp w's private region starts at
    // w_base + w * w_stride; offsets below are within that region
    int32_t warp_kernels;  // 1: k_dense_w / k_mti_w; 3: the split MTI scan; 0: the CTA kernels
    int32_t w_base, w_stride;
    int32_t w_acc_hi, w_acc_lo, w_cnt, w_tile, w_bucket, w_state;
    // k_mti_w: when non-null, each warp's TwoSum accumulators (hi then lo,
    // k x d each) live in this global array, slot blockIdx.x * WPC + warp,
    // instead of shared memory (few points change cluster in an MTI
    // iteration; the freed shared memory holds more warps per SM)
    float *wacc;
    // split MTI scan: the row stride of a staged batch, in floats (d + 4)
    int32_t sp_rs;
    int32_t *err;          // set when a bounded wait gives up (KNOR_ERR_TIMEOUT)
    // split MTI scan (k_mti_sel + k_mti_scan): per k_mti_sel warp a list of
    // batch records (SP_REC ints each: cluster, count, 32 point indices,
    // padding), rec_cap records each, rec_cnt[list] records written;
    // k_mti_sel runs sel_mult (1 or 2) warps per scan warp, scan warp w taking
    // lists w sel_mult, w sel_mult + 1 in order (their ranges make up its
    // own); warps per CTA and the per-warp shared-memory region of the scan
    // (two row slots, then the warp's member counts)
    int32_t *rec;
    int32_t *rec_cnt;
    int64_t rec_cap;
    int32_t sel_mult;
    int32_t sp_wpb;
    int32_t sp_off_warp, sp_warp_stride, sp_off_cnt;
    // change lists (point, new cluster << 16 | old cluster), chg_cap entries
    // per scan warp, chg_cnt[warp] entries written; the delta kernel's
    // per-warp shared-memory region (accumulators and counts) and the number
    // of its warps that share one list
    int2 *chg;
    int32_t *chg_cnt;
    int64_t chg_cap;
    int32_t dl_warp_stride, dl_split; // k_mti_delta: per-warp region, warps per change list
    int32_t dl_off_rows;   // k_mti_delta: the two 32-row slots within the per-warp region
    int32_t dl_dense;      // 1: dense iterations sum by change lists (k_dense_scan)
    int32_t dl_mti;        // 1: MTI iterations sum by change lists (k_mti_scan)
    // Elkan's lower bounds (ablation of MTI): n x k FP32, cluster-major
    // (lb[c n + i]); each stored as l + F(c) rounded down, where l <= d(x_i, c)
    // when stored and F is the cumulative drift, so that lb - F^t(c) bounds
    // d(x_i, c^t) from below; null when not kept
    float *lb;
    float ginv_dn;         // <= (1 - (d+2) 2^-24): turns a computed d^2 into a lower bound
    // k_mti_sel's heavy points: a surviving point of cluster a whose Clause-1
    // test value reaches theta[a] goes to the mixed bucket (null: no split);
    // off_th: the thresholds' place in k_mti_sel's shared memory
    const float *theta;
    int32_t off_th;
};

// Parameters of the reduction / finalize kernels.
struct FinParams {
    const double *part_S;
    const long long *part_cnt;
    int32_t part_stride;
    int32_t k, d;
    double *S;              // k x d running sums
    const long long *cnt;   // k member counts before this iteration
    long long *cnt_next;    // k member counts after
    double *C64;            // k x d master centroids
    float *C32;             // k x d scan copy (current; replaced by K1)
    float *C32n;            // k x d scan copy (next)
    float *halfD, *s, *F;
    long long *cnt_out;     // where K1 commits cnt_next
    Counters *ctr;
    IterStats *stats;       // per-run records
    int32_t *run_iter;      // iterations done in this run
    int32_t *total_iter;    // iterations since reset
    const int32_t *max_iters_dev; // run limit (for the device-side loop)
    int32_t snapshot;       // 1: record stats (0 for the table at reset)
    unsigned long long cond_handle; // cudaGraphConditionalHandle, 0 if none
    // k_mti_sel's heavy thresholds (null when not used): theta[a] = the
    // th_M-th smallest of 1/2 d(c_a, c) over c != a (+inf when th_M > k - 1)
    float *theta;
    int32_t th_M;
};

// Candidate slots per re-scored point in the precision form (count + 8,
// padded to 12 ints = three int4).
constexpr int PREC_CANDS = 16;

// Per-iteration quantities of the precision form, written on the device
// before the tensor-core scan: norms and the centroid scale.
struct PrecIter {
    float cnorm_max; // max ||c|| rounded up (atomicMax on the bits)
    float cabs_max;  // max |c_j sigma_j| (atomicMax on the bits)
    float cdnorm_max; // max ||c . sigma|| rounded up (FP8: per-dimension scales; else = cnorm_max)
    float neg2inv;   // -2 / (s_x s_c): a power of two
    float eta_c;     // sqrt(d) * (absolute rounding error of a scaled coordinate) / s_c, rounded up
};

// Operand format of the precision form's tensor-core scan.
enum PrecFormat : int32_t { PREC_FMT_BF16 = 0, PREC_FMT_FP16 = 1, PREC_FMT_FP8 = 2 };

// Parameters of the precision-form assignment (precision.cu).
struct PrecParams {
    int64_t n;
    int32_t d, k;
    const float *xn;     // n: ||x||^2 (FP64 sum rounded to FP32)
    const float *xdn;    // n: ||x / sigma||^2 (FP8: per-dimension scales; else = xn)
    const float *rxdn;   // mode 1: the same for the gathered points
    int32_t fp8;         // operands are FP8 e4m3 (kind::f8f6f4), else 16-bit (kind::f16)
    int32_t nkc;         // 128-byte K chunks per row (d x operand bytes / 128)
    int32_t tkb;         // operand elements per 128-byte chunk
    const float *cn;     // k: ||c||^2
    const PrecIter *it;  // this iteration's centroid quantities
    int32_t *a_next;     // n: new assignment of certified points
    int32_t *rlist;      // points to re-score exactly
    int32_t *rcand;      // per listed point: two lists (one per half of the columns), each a
                         // count (-1: too many) and up to 7 centroids
    float *rm1;          // per listed point: its smallest d~^2
    const float *rxn;    // mode 1: ||x||^2 of the gathered points
    int32_t mode;        // 0: all points, certify or list; 1: listed points, record candidates
    unsigned *rcount;
    uint32_t idesc;      // tcgen05 instruction descriptor (operand format)
    // error bound E(x) (prec_error_constants): unit roundoff of the operand
    // format, sqrt(d) * absolute error of a scaled point coordinate / s_x,
    // tensor-core accumulation factor, FP32 epilogue and distance factors
    float uq, eta_x, gtc, eA32, eB;
    int32_t *err;        // set when a bounded wait gives up
};

// Launchers implemented in kernels.cu.
// mode_dense selects which scan runs (the other returns at once); the scan
// that runs records how many partial slots it wrote and whether the sums are
// fresh (dense) or deltas (MTI).
cudaError_t launch_dense(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                         const int32_t *mode_dense, int32_t *nslots, int32_t *fresh);
cudaError_t launch_mti(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                       const int32_t *mode_dense, int32_t *nslots, int32_t *fresh);
cudaError_t dense_attr(int dv, size_t smem, int *blocks_per_sm);
cudaError_t mti_attr(int dv, size_t smem, int *blocks_per_sm);
// warp-autonomous variants (templated widths only), WPC warps per CTA
cudaError_t launch_dense_w(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                           const int32_t *mode_dense, int32_t *nslots, int32_t *fresh);
cudaError_t launch_mti_w(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                         const int32_t *mode_dense, int32_t *nslots, int32_t *fresh);
cudaError_t dense_w_attr(int dv, size_t smem, int *blocks_per_sm);
cudaError_t mti_w_attr(int dv, size_t smem, int *blocks_per_sm);
// split MTI scan: Clause 1 + batch records, then the scan of the records
cudaError_t launch_mti_sel(const IterParams &p, int grid, size_t smem, cudaStream_t s, const int32_t *mode_dense);
cudaError_t mti_sel_attr(int wpb, size_t smem, int *blocks_per_sm);
cudaError_t launch_mti_scan(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                            const int32_t *mode_dense, int32_t *nslots, int32_t *fresh);
cudaError_t mti_scan_attr(int dv, int wpb, size_t smem, int *blocks_per_sm);
cudaError_t launch_mti_delta(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                             const int32_t *mode_dense, int32_t *nslots, int32_t *fresh);
cudaError_t mti_delta_attr(int dv, size_t smem, int split, int *blocks_per_sm);
cudaError_t launch_dense_scan(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                              const int32_t *mode_dense);
cudaError_t dense_scan_attr(int dv, size_t smem, int *blocks_per_sm);
// Elkan's scan (MTI plus lower bounds) on the split grid, and its bound check
cudaError_t launch_elkan_scan(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                              const int32_t *mode_dense);
cudaError_t elkan_scan_attr(int dv, size_t smem, int *blocks_per_sm);
cudaError_t launch_elkan_check(int dv, const IterParams &p, IterStats *stats, const int32_t *run_iter,
                               cudaStream_t s);
cudaError_t launch_reduce(const FinParams &f, const int32_t *nslots, const int32_t *fresh, cudaStream_t s);
cudaError_t launch_theta(const FinParams &f, cudaStream_t s);
cudaError_t launch_table(const FinParams &f, int32_t *mode_dense, int need_table, int recompute_every,
                         int always_dense, cudaStream_t s);
cudaError_t launch_validate(const float *X, int64_t count, unsigned long long *bad, cudaStream_t s);
cudaError_t launch_init_state(PtState *st, int64_t n, cudaStream_t s);
cudaError_t launch_gather_rows(const float *X, int32_t d, const int64_t *idx, int32_t k, double *C64,
                               cudaStream_t s);
cudaError_t launch_round_c32(const double *C64, float *C32, int64_t kd, cudaStream_t s);
cudaError_t launch_extract_assign(const PtState *st, int64_t n, int32_t *out, cudaStream_t s);
cudaError_t launch_check_bounds(const float *X, int64_t n, int32_t d, const PtState *st,
                                const float *C32, const float *F, IterStats *stats,
                                const int32_t *run_iter, cudaStream_t s);
int supported_dv(int d); // template width used for d (0 = generic)
void set_global_error(const char *msg); // message for knor_last_error(NULL)
// k-means++ seeding (kmeanspp.cu): one round's D^2 update (with the round's
// largest D^2 as float bits), the weight sums over the fixed CTA ranges, and
// the search of one range for the drawn point
cudaError_t kpp_update(int dv, const float *X, int64_t n, int32_t d, const float *c, float *D2, int first,
                       unsigned *maxbits, int grid, cudaStream_t s);
cudaError_t kpp_sums(const float *D2, int64_t n, double scale, unsigned long long *sums, int grid, cudaStream_t s);
cudaError_t kpp_find(const float *D2, int64_t lo, int64_t hi, double scale, unsigned long long t, int64_t *out,
                     cudaStream_t s);
// Forgy initialisation: k distinct indices of [0, n) (Floyd's sampling on
// SplitMix64(seed)), in the order drawn (knor_ctx.cu).
std::vector<int64_t> forgy_indices(int64_t n, int32_t k, uint64_t seed);
float f32_up(double v); // smallest float >= v

// precision form (precision.cu)
size_t prec_smem_bytes(int d, int k, int esize);
cudaError_t prec_absmax(const float *X, int64_t count, float *out, cudaStream_t s);
cudaError_t prec_dim_absmax(const float *X, int64_t n, int32_t d, float *out, cudaStream_t s);
cudaError_t prec_points(const float *X, int64_t n, int32_t d, int32_t fmt, float sx, const float *sigma_inv,
                        void *Xb, float *xn, float *xdn, cudaStream_t s);
cudaError_t prec_prep(const float *C32, int32_t k, int32_t d, int32_t fmt, float sx, const float *sigma, void *Cb,
                      float *cn, PrecIter *it, cudaStream_t s);
int prec_point_scale_exp(int32_t fmt, float absmax); // s_x = 2^this
cudaError_t prec_assign_attr(size_t smem);
// tmX / tmC point to CUtensorMap objects (cuda.h) over the BF16 points / centroids
cudaError_t prec_assign(const void *tmX, const void *tmC, const PrecParams &p, int grid, size_t smem, cudaStream_t s);
void prec_error_constants(int32_t fmt, int d, float sx, PrecParams &p);
cudaError_t prec_recheck(int dv, const float *X, const float *C32, int32_t k, const int32_t *rlist,
                         const int32_t *rcand, const unsigned *rcount, int32_t *a_next, Counters *ctr, int grid,
                         cudaStream_t s);
cudaError_t prec_gather(int row_bytes, const void *Xb, const float *xn, const float *xdn, const int32_t *rlist,
                        const unsigned *rcount, void *Xc, float *rxn, float *rxdn, int grid, cudaStream_t s);
cudaError_t prec_verify(const float *X, int64_t n, int32_t d, const float *C32, int32_t k, const int32_t *a_next,
                        unsigned long long *viol, cudaStream_t s);
cudaError_t prec_delta_sums(const float *X, int64_t n, int32_t d, PtState *st, const int32_t *a_next, double *S,
                            long long *cnt, Counters *ctr, int32_t k, int32_t *nslots, int32_t *fresh, int grid,
                            cudaStream_t s);

} // namespace knor

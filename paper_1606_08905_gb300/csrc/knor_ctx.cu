// knor_ctx.cu -- host runtime of libknor.so: the C ABI of include/knor.h.
//
// A context owns the points, the per-point MTI state, the centroid tables and
// one CUDA stream.  One Lloyd iteration is the launch sequence
//   k_dense | k_mti  ->  k_reduce  ->  k_table  [-> k_check_bounds]
// captured once into a CUDA graph (knor_iterate) and once into the body of a
// conditional WHILE node (knor_run), so a whole run is a single graph launch
// and the loop stops on the device when an iteration changes nothing.
#include "knor.h"
#include "knor_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_set>
#include <vector>

using namespace knor;

namespace {

constexpr int kStatsCap = 1 << 16; // records per knor_run call
constexpr uint32_t kStateMagic = 0x4b4e4f52u; // "KNOR"
constexpr uint32_t kStateVersion = 1;

// Device flags (int32 each).
enum Flag { F_RUN_ITER = 0, F_TOTAL_ITER, F_MAX_ITERS, F_MODE_DENSE, F_NSLOTS, F_FRESH, F_ERR, F_COUNT };

} // namespace

namespace knor {

// SplitMix64 (Steele, Lea and Flood 2014): golden-ratio increment, then the
// published finaliser.
uint64_t splitmix64(uint64_t &state) {
    state += 0x9E3779B97F4A7C15ULL;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Floyd's sampling (Bentley and Floyd 1987): k distinct indices of [0, n) in
// the order they are kept; the uniform draw on [0, j] is the high word of
// r * (j + 1).
std::vector<int64_t> forgy_indices(int64_t n, int32_t k, uint64_t seed) {
    std::vector<int64_t> out;
    out.reserve((size_t)k);
    std::unordered_set<int64_t> kept;
    uint64_t state = seed;
    for (int64_t j = n - k; j < n; ++j) {
        const uint64_t r = splitmix64(state);
        const int64_t t = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(j + 1)) >> 64);
        const int64_t v = kept.count(t) ? j : t;
        kept.insert(v);
        out.push_back(v);
    }
    return out;
}

// k-means++ row indices (the rule of knor.h's KNOR_INIT_KMEANSPP): D^2 and
// the weights on the GPU, the draws and exact integer sums on the host.
static cudaError_t kmeanspp_indices(const float *X, int64_t n, int32_t d, int32_t k, uint64_t seed, int dv,
                                    int num_sms, cudaStream_t s, std::vector<int64_t> &out) {
    out.clear();
    uint64_t state = seed;
    auto below = [&](uint64_t m) {
        const uint64_t r = splitmix64(state);
        return (uint64_t)(((unsigned __int128)r * (unsigned __int128)m) >> 64);
    };
    out.push_back((int64_t)below((uint64_t)n));
    if (k == 1) return cudaSuccess;
    const int grid = 8 * num_sms;
    float *D2 = nullptr;
    unsigned *maxbits = nullptr;
    unsigned long long *sums = nullptr;
    int64_t *found = nullptr;
    cudaError_t e = cudaMalloc((void **)&D2, sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&maxbits, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&sums, sizeof(unsigned long long) * grid);
    if (e == cudaSuccess) e = cudaMalloc((void **)&found, sizeof(int64_t));
    std::vector<unsigned long long> hs((size_t)grid);
    for (int32_t j = 1; j < k && e == cudaSuccess; ++j) {
        unsigned mb = 0;
        e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned), s);
        if (e == cudaSuccess)
            e = kpp_update(dv, X, n, d, X + (size_t)out.back() * d, D2, j == 1 ? 1 : 0, maxbits, grid, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&mb, maxbits, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        float m;
        std::memcpy(&m, &mb, sizeof(m));
        unsigned long long T = 0;
        double scale = 0.0;
        if (m > 0.0f) {
            int ex = 0;
            std::frexp(m, &ex); // m = f 2^ex, f in [0.5, 1): m < 2^ex
            scale = std::ldexp(1.0, 32 - ex);
            e = kpp_sums(D2, n, scale, sums, grid, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hs.data(), sums, sizeof(unsigned long long) * grid, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            for (unsigned long long v : hs) T += v;
        }
        if (T == 0) {
            out.push_back((int64_t)below((uint64_t)n));
            continue;
        }
        unsigned long long t = below(T), before = 0;
        int b = 0;
        while (b < grid - 1 && before + hs[(size_t)b] <= t) before += hs[(size_t)b++];
        // CTA b's range, as block_range on the device splits [0, n)
        const int64_t lo = (int64_t)((unsigned __int128)n * b / grid);
        const int64_t hi = (int64_t)((unsigned __int128)n * (b + 1) / grid);
        int64_t idx = -1;
        e = kpp_find(D2, lo, hi, scale, t - before, found, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&idx, found, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && (idx < lo || idx >= hi)) e = cudaErrorUnknown; // cannot happen: the sums say so
        out.push_back(idx);
    }
    cudaFree(D2);
    cudaFree(maxbits);
    cudaFree(sums);
    cudaFree(found);
    return e;
}

float f32_up(double v) { // smallest float >= v
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}

} // namespace knor

namespace {

int getenv_int(const char *name, int dflt) {
    const char *v = std::getenv(name);
    return v && *v ? std::atoi(v) : dflt;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct StateHeader {
    uint32_t magic, version;
    int64_t n;
    int32_t d, k;
    int32_t no_prune, precision, recompute, total_iter, mode_dense, pad; // pad: the elkan option
};

} // namespace

struct knor_ctx {
    int dev = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    int32_t d = 0, k = 0;
    knor_opts opts{};
    knor_init init = KNOR_INIT_FORGY;
    uint64_t seed = 0;
    std::vector<int64_t> init_idx;
    bool c0_set = false;
    mutable std::string err;

    float *X = nullptr;
    PtState *st = nullptr;
    double *C0 = nullptr, *C64 = nullptr, *S = nullptr, *part_S = nullptr;
    float *C32 = nullptr, *C32n = nullptr, *halfD = nullptr, *s = nullptr, *F = nullptr;
    long long *cnt = nullptr, *cnt_next = nullptr, *part_cnt = nullptr;
    Counters *ctr = nullptr;
    IterStats *stats = nullptr;
    int32_t *flags = nullptr;
    int64_t *d_idx = nullptr;
    unsigned long long *d_bad = nullptr;
    IterStats *h_stats = nullptr; // pinned

    int dv = 0;
    int part_stride = 1;
    size_t smem_dense = 0, smem_mti = 0;
    int grid_dense = 0, grid_mti = 0;
    IterParams ip_dense{}, ip_mti{};
    FinParams fp{};

    cudaGraphExec_t iter_exec = nullptr, run_exec = nullptr;

    // precision form (BF16 tensor-core distances + exact FP32 recheck)
    bool prec = false;
    void *Xb = nullptr, *Cb = nullptr, *Xc = nullptr;
    float *rm1 = nullptr, *rxn = nullptr;
    alignas(64) unsigned char tmXc[128] = {};
    PrecParams pp2{};
    float *wacc = nullptr; // k_mti_w warp accumulators
    int32_t *rec = nullptr, *rec_cnt = nullptr, *chg_cnt = nullptr; // split MTI scan: batch records
    int2 *chg = nullptr;                                                // and change lists
    float *lb = nullptr;                                                // Elkan's lower bounds
    bool X_on_host = false;          // points_in_host: X is the device address of the caller's buffer
    float *host_registered = nullptr; // ... registered by knor_create (pageable memory)
    IterParams ip_sel{}, ip_delta{};
    size_t smem_sel = 0;
    int sel_M = 0;                   // k_mti_sel: heavy from the sel_M-th smallest 1/2 d(c_a, c) (0: no split)
    int sel_mult = 1;                // k_mti_sel warps per scan warp (1 or 2)
    float *theta = nullptr;          // k heavy thresholds
    bool mti_split = false, dense_split = false; // the split kernels run the MTI / dense scans
    int grid_split = 0;
    float *xdn = nullptr, *rxdn = nullptr; // FP8: norms of x / sigma (else aliases of xn, rxn)
    float *sigma = nullptr;                // FP8: sigma_j, then 1 / sigma_j (d each)
    float *xn = nullptr, *cn = nullptr, *absmax = nullptr;
    PrecIter *pit = nullptr;
    int32_t fmt = PREC_FMT_BF16;
    float sx = 1.0f; // point scale (a power of two)
    int32_t *a_next = nullptr, *rlist = nullptr, *rcand = nullptr;
    unsigned *rcount = nullptr;
    alignas(64) unsigned char tmX[128] = {}, tmC[128] = {}; // CUtensorMap
    PrecParams pp{};
    int prec_grid = 0;
    size_t prec_smem = 0;

    // profiling (host-driven loop, CUDA events around every kernel)
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    knor_profile prof{};
    int32_t host_total_iter = 0;
    std::string kname[KNOR_KERNEL_COUNT];
};

static thread_local std::string g_create_err;

namespace knor {
// Error message for calls that have no context (read by knor_last_error(NULL)).
void set_global_error(const char *msg) { g_create_err = msg ? msg : ""; }
} // namespace knor

#define KNOR_CUDA(ctx, call)                                                                    \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return e_ == cudaErrorMemoryAllocation ? KNOR_ERR_OOM : KNOR_ERR_CUDA;              \
        }                                                                                       \
    } while (0)

static knor_status fail(const knor_ctx *c, knor_status st, const std::string &msg) {
    c->err = msg;
    return st;
}

// Pending injected allocation failure (knor_test_fail_alloc): the number
// of allocations still to succeed before one fails; -1: none.
static std::atomic<int64_t> g_fail_alloc_after{-1};

template <class T>
static knor_status dalloc(knor_ctx *c, T **p, size_t count) {
    if (count == 0) count = 1;
    int64_t left = g_fail_alloc_after.load();
    while (left >= 0 && !g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
    }
    if (left == 0) {
        *p = nullptr;
        return fail(c, KNOR_ERR_OOM, "cudaMalloc(" + std::to_string(count * sizeof(T)) +
                                         " bytes): injected failure (knor_test_fail_alloc)");
    }
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, KNOR_ERR_OOM, std::string("cudaMalloc(") + std::to_string(count * sizeof(T)) +
                                         " bytes): " + cudaGetErrorString(e));
    }
    return KNOR_OK;
}

static void free_all(knor_ctx *c) {
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    if (c->iter_exec) cudaGraphExecDestroy(c->iter_exec);
    if (c->run_exec) cudaGraphExecDestroy(c->run_exec);
    if (c->host_registered) cudaHostUnregister(c->host_registered);
    void *bufs[] = {c->X_on_host ? nullptr : c->X, c->st,     c->C0,       c->C64,  c->S,     c->part_S, c->C32,  c->C32n,
                    c->halfD,  c->s,      c->F,        c->cnt,  c->cnt_next, c->part_cnt, c->ctr, c->stats,
                    c->flags,  c->d_idx,  c->d_bad,    c->Xb,   c->Cb,    c->xn,     c->cn,   c->absmax, c->pit,
                    c->a_next, c->rlist,  c->rcount, c->rcand, c->Xc, c->rm1, c->rxn, c->wacc, c->sigma, c->rec, c->rec_cnt, c->chg, c->chg_cnt, c->lb, c->theta,
                    c->xdn != c->xn ? c->xdn : nullptr, c->rxdn != c->rxn ? c->rxdn : nullptr};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (c->h_stats) cudaFreeHost(c->h_stats);
    if (c->stream) cudaStreamDestroy(c->stream);
}

// A 2-D TMA descriptor over a row-major rows x inner BF16 matrix, boxes of
// 64 columns (128 bytes) x box_rows rows, 128-byte swizzle, zero fill outside.
// TMA map of a row-major matrix of operands (rows x inner; 16-bit or FP8),
// 128-byte-wide boxes of box_rows rows, 128-byte swizzle.
static knor_status encode_op_map(knor_ctx *c, void *out, void *base, uint64_t inner, uint64_t rows,
                                 uint32_t box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q{};
        void *f = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f)
            return fail(c, KNOR_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    const int esize = c->fmt == PREC_FMT_FP8 ? 1 : 2;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * esize};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esize), box_rows}; // 128-byte rows
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapDataType dt = c->fmt == PREC_FMT_FP8    ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : c->fmt == PREC_FMT_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                             : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = fn(static_cast<CUtensorMap *>(out), dt, 2, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, KNOR_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return KNOR_OK;
}

// Shared-memory layout of a point kernel; returns the byte size.
static size_t plan_layout(const knor_ctx *c, bool mti, IterParams &p) {
    const int d = c->d, k = c->k, dv = c->dv;
    const size_t kd = (size_t)k * d;
    size_t off = 0;
    auto take = [&](size_t bytes) -> int32_t {
        const size_t o = off;
        off = (off + bytes + 15) & ~(size_t)15;
        return (int32_t)o;
    };
    const size_t budget = 200 * 1024;
    // fixed parts first
    p.dpad = d + 4;
    size_t tile_bytes = 0;
    p.stages = 1;
    if (dv > 0) {
        const size_t one = (size_t)NT * p.dpad * sizeof(float);
        p.stages = (!mti && 2 * one <= 110 * 1024) ? 2 : 1;
        tile_bytes = p.stages * one;
    }
    size_t fixed = tile_bytes + 3 * NT * sizeof(int) + 256 + (mti ? QCAP * sizeof(int2) : 0);
    p.cent_smem = (kd * sizeof(float) <= 64 * 1024 && fixed + kd * 4 <= budget) ? 1 : 0;
    if (p.cent_smem) fixed += kd * 4;
    p.halfD_smem = 0;
    if (mti && (size_t)k * k * 4 <= 48 * 1024 && fixed + (size_t)k * k * 4 <= budget) {
        p.halfD_smem = 1;
        fixed += (size_t)k * k * 4;
    }
    const bool sf = (size_t)k * 8 <= 32 * 1024 && fixed + (size_t)k * 8 <= budget;
    if (sf) fixed += (size_t)k * 8;
    p.acc_global = (fixed + 2 * kd * 4 + (size_t)k * 4 > budget) ? 1 : 0;

    p.off_acc_hi = take(p.acc_global ? 0 : kd * 4);
    p.off_acc_lo = take(p.acc_global ? 0 : kd * 4);
    p.off_cnt = take(p.acc_global ? 0 : (size_t)k * 4);
    p.off_cent = take(p.cent_smem ? kd * 4 : 0);
    p.off_halfD = take(p.halfD_smem ? (size_t)k * k * 4 : 0);
    p.off_s = sf ? take((size_t)k * 4) : -1;
    p.off_F = sf ? take((size_t)k * 4) : -1;
    p.off_tb = take(NT * 4);
    p.off_ta = take(NT * 4);
    p.off_ti = take(NT * 4);
    p.off_tile = take(tile_bytes);
    p.off_queue = take(mti ? QCAP * sizeof(int2) : 0);
    p.off_misc = take(256);
    return off;
}

// Shared-memory layout of a warp-autonomous kernel (CTA tables, then WPC
// private warp regions); returns 0 when the variant does not apply.
static size_t plan_layout_warp(const knor_ctx *c, bool mti, IterParams &p) {
    const int d = c->d, k = c->k, dv = c->dv;
    if (dv == 0) return 0;
    const size_t kd = (size_t)k * d;
    size_t off = 0;
    auto take = [&](size_t bytes) -> int32_t {
        const size_t o = off;
        off = (off + bytes + 15) & ~(size_t)15;
        return (int32_t)o;
    };
    p.dpad = d + 4;
    // the warp kernels keep every table in shared memory (else: CTA kernels)
    if (kd * 4 > 32 * 1024 || (mti && (size_t)k * k * 4 > 16 * 1024) || (size_t)k * 8 > 8 * 1024) return 0;
    p.cent_smem = 1;
    p.off_cent = take(kd * 4);
    p.halfD_smem = mti ? 1 : 0;
    p.off_halfD = take(mti ? (size_t)k * k * 4 : 0);
    p.off_s = take((size_t)k * 4);
    p.off_F = take((size_t)k * 4);
    p.w_base = take(0);
    size_t woff = 0;
    auto wtake = [&](size_t bytes) -> int32_t {
        const size_t o = woff;
        woff = (woff + bytes + 15) & ~(size_t)15;
        return (int32_t)o;
    };
    // the MTI kernel keeps its warps' accumulators in global memory
    p.w_acc_hi = mti ? 0 : wtake(kd * 4);
    p.w_acc_lo = mti ? 0 : wtake(kd * 4);
    p.w_cnt = wtake((size_t)k * 4);
    p.w_tile = wtake(mti ? 0 : 2 * 32 * (size_t)p.dpad * 4); // dense: two row tiles
    // MTI: k + 1 point buckets (one per cluster, one for unassigned points)
    // of WBCAP local indices, then their heads and counts
    p.w_bucket = wtake(mti ? (size_t)(k + 1) * (WBCAP + 2) * 4 : 0);
    p.w_state = wtake(mti ? (size_t)WSTAGES * WCH * sizeof(PtState) : 0);
    p.w_stride = (int32_t)woff;
    const size_t total = off + (size_t)WPC * woff;
    if (total > 110 * 1024) return 0; // keep at least two CTAs per SM
    p.warp_kernels = 1;
    p.acc_global = 0;
    p.stages = 2;
    return total;
}

// Shared-memory layouts of the split MTI scan: k_mti_sel (s and F, then per
// warp its buckets and state chunks) and k_mti_scan (centroids, k x k table,
// F, then per warp two row slots and its member counts).  0 when the split
// does not apply.
static size_t plan_layout_sel(const knor_ctx *c, IterParams &p) {
    const int k = c->k;
    size_t off = 0;
    auto take = [&](size_t bytes) -> int32_t {
        const size_t o = off;
        off = (off + bytes + 15) & ~(size_t)15;
        return (int32_t)o;
    };
    p.off_s = take((size_t)k * 4);
    p.off_F = take((size_t)k * 4);
    p.off_th = take((size_t)k * 4);
    p.w_base = take(0);
    p.w_bucket = 0;
    // k + 1 buckets (one per cluster, and the mixed one) of 32 slots and a count
    const size_t bucket = (((size_t)(k + 1) * (32 + 1) * 4) + 15) & ~(size_t)15;
    p.w_state = (int32_t)bucket;
    p.w_stride = (int32_t)(bucket + (size_t)WSTAGES * WCH * sizeof(PtState));
    p.sp_wpb = SP_WPB;
    return off + (size_t)SP_WPB * p.w_stride;
}
static size_t plan_layout_scan(const knor_ctx *c, IterParams &p) {
    const int d = c->d, k = c->k, dv = c->dv;
    if (dv != 8 && dv != 16 && dv != 32 && dv != 64) return 0;
    const size_t kd = (size_t)k * d;
    if (kd * 4 > 32 * 1024 || (size_t)k * k * 4 > 48 * 1024) return 0;
    size_t off = 0;
    auto take = [&](size_t bytes) -> int32_t {
        const size_t o = off;
        off = (off + bytes + 15) & ~(size_t)15;
        return (int32_t)o;
    };
    p.cent_smem = 1;
    p.halfD_smem = 1;
    p.off_cent = take(kd * 4);
    p.off_halfD = take((size_t)k * k * 4);
    p.off_F = take((size_t)k * 4);
    p.off_s = take((size_t)k * 4);
    // rows padded by 16 bytes: lane l reads its row at l * (4d + 16) bytes,
    // so the 8 lanes of a 16-byte shared load hit distinct banks
    p.sp_rs = d + 4;
    p.sp_off_warp = take(0);
    p.sp_off_cnt = 2 * 32 * p.sp_rs * 4;
    p.sp_warp_stride = (int32_t)((p.sp_off_cnt + (size_t)k * 4 + 15) & ~(size_t)15);
    p.sp_wpb = SP_WPB;
    const size_t total = off + (size_t)SP_WPB * p.sp_warp_stride;
    if (total > 112 * 1024) return 0; // keep at least two CTAs per SM
    // k_mti_delta: per warp, TwoSum accumulators and counts, then two slots
    // of 32 rows; each change list split over up to 4 warps while two CTAs
    // fit on an SM
    p.dl_off_rows = (int32_t)(((size_t)2 * kd * 4 + (size_t)k * 4 + 15) & ~(size_t)15);
    p.dl_warp_stride = p.dl_off_rows + 2 * 32 * d * 4;
    p.dl_split = 4;
    while (p.dl_split > 1 && (size_t)SP_WPB * p.dl_split * p.dl_warp_stride > 113 * 1024) p.dl_split /= 2;
    if ((size_t)SP_WPB * p.dl_split * p.dl_warp_stride > 227 * 1024) return 0;
    p.warp_kernels = 3;
    p.acc_global = 0;
    return total;
}

static void fill_common(knor_ctx *c, IterParams &p) {
    p.X = c->X;
    p.n = c->n;
    p.d = c->d;
    p.k = c->k;
    p.st = c->st;
    p.C32 = c->C32;
    p.halfD = c->halfD;
    p.s = c->s;
    p.F = c->F;
    p.part_S = c->part_S;
    p.part_cnt = c->part_cnt;
    p.ctr = c->ctr;
    // FP32 error bound of the direct-form squared distance: relative
    // (1 - (d+2) u)^-1 - 1 with u = 2^-24, plus d 2^-150 absolute.
    const double u = std::ldexp(1.0, -24);
    const double g = (c->d + 2) * u / (1.0 - (c->d + 2) * u);
    p.g_up = f32_up(1.0 / (1.0 - (c->d + 2) * u));
    p.onepk = f32_up(1.0 + g);
    p.tau = std::ldexp(1.0f, -40);
    p.tiny = (float)std::ldexp((double)std::min(c->d, 1 << 20), -149);
    p.mti = c->opts.no_prune ? 0 : 1;
    p.err = c->flags + F_ERR;
}

static cudaError_t scan_dense(knor_ctx *c, cudaStream_t s) {
    int32_t *fl = c->flags;
    if (c->dense_split) return launch_dense_scan(c->dv, c->ip_dense, c->grid_split, c->smem_dense, s, fl + F_MODE_DENSE);
    if (c->ip_dense.warp_kernels)
        return launch_dense_w(c->dv, c->ip_dense, c->grid_dense, c->smem_dense, s, fl + F_MODE_DENSE,
                              fl + F_NSLOTS, fl + F_FRESH);
    return launch_dense(c->dv, c->ip_dense, c->grid_dense, c->smem_dense, s, fl + F_MODE_DENSE, fl + F_NSLOTS,
                        fl + F_FRESH);
}

static cudaError_t scan_mti(knor_ctx *c, cudaStream_t s) {
    int32_t *fl = c->flags;
    if (c->mti_split && c->opts.elkan)
        return launch_elkan_scan(c->dv, c->ip_mti, c->grid_split, c->smem_mti, s, fl + F_MODE_DENSE);
    if (c->mti_split)
        return launch_mti_scan(c->dv, c->ip_mti, c->grid_split, c->smem_mti, s, fl + F_MODE_DENSE, fl + F_NSLOTS,
                               fl + F_FRESH);
    if (c->ip_mti.warp_kernels)
        return launch_mti_w(c->dv, c->ip_mti, c->grid_mti, c->smem_mti, s, fl + F_MODE_DENSE, fl + F_NSLOTS,
                            fl + F_FRESH);
    return launch_mti(c->dv, c->ip_mti, c->grid_mti, c->smem_mti, s, fl + F_MODE_DENSE, fl + F_NSLOTS,
                      fl + F_FRESH);
}

// Clause 1 and the batch records of the split MTI scan.
static cudaError_t scan_select(knor_ctx *c, cudaStream_t s) {
    if (!c->mti_split || c->opts.elkan) return cudaSuccess;
    return launch_mti_sel(c->ip_sel, c->grid_split * c->sel_mult, c->smem_sel, s, c->flags + F_MODE_DENSE);
}

// Phase II from the change lists of the split scans (a no-op in a dense
// iteration whose scan summed for itself).
static cudaError_t scan_delta(knor_ctx *c, cudaStream_t s) {
    if (!c->mti_split && !c->dense_split) return cudaSuccess;
    int32_t *fl = c->flags;
    return launch_mti_delta(c->dv, c->ip_delta, c->grid_split,
                            (size_t)SP_WPB * c->ip_delta.dl_split * c->ip_delta.dl_warp_stride, s,
                            fl + F_MODE_DENSE, fl + F_NSLOTS, fl + F_FRESH);
}

// The precision form's iteration: BF16 centroids, tensor-core scan with
// certification, exact FP32 re-score of the rest, delta sums, merge, table.
// With events != nullptr each stage is bracketed by CUDA events (profiling).
static knor_status enqueue_prec(knor_ctx *c, cudaStream_t s, unsigned long long cond, cudaEvent_t *ev) {
    int32_t *fl = c->flags;
    auto mark = [&](int i) -> cudaError_t { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
    KNOR_CUDA(c, cudaMemsetAsync(c->part_S, 0, sizeof(double) * (size_t)c->k * c->d, s));
    KNOR_CUDA(c, cudaMemsetAsync(c->part_cnt, 0, sizeof(long long) * (size_t)c->k, s));
    KNOR_CUDA(c, cudaMemsetAsync(c->rcount, 0, sizeof(unsigned), s));
    // every point gets a new assignment from the scan or the recheck; -1
    // marks one that did not (k_delta_sums counts it as a violation)
    KNOR_CUDA(c, cudaMemsetAsync(c->a_next, 0xFF, sizeof(int32_t) * (size_t)c->n, s));
    KNOR_CUDA(c, mark(0));
    KNOR_CUDA(c, prec_prep(c->C32, c->k, c->d, c->fmt, c->sx, c->sigma, c->Cb, c->cn, c->pit, s));
    KNOR_CUDA(c, prec_assign(c->tmX, c->tmC, c->pp, c->prec_grid, c->prec_smem, s));
    KNOR_CUDA(c, mark(1));
    // the points left uncertified: candidate pass over their gathered rows,
    // then the exact FP32 re-score
    KNOR_CUDA(c, mark(8));
    KNOR_CUDA(c, prec_gather(c->d * (c->fmt == PREC_FMT_FP8 ? 1 : 2), c->Xb, c->xn, c->xdn, c->rlist, c->rcount,
                             c->Xc, c->rxn, c->rxdn, 8 * c->num_sms, s));
    KNOR_CUDA(c, prec_assign(c->tmXc, c->tmC, c->pp2, c->prec_grid, c->prec_smem, s));
    KNOR_CUDA(c, prec_recheck(c->dv, c->X, c->C32, c->k, c->rlist, c->rcand, c->rcount, c->a_next, c->ctr,
                              4 * c->num_sms, s));
    if (c->opts.debug_invariants)
        KNOR_CUDA(c, prec_verify(c->X, c->n, c->d, c->C32, c->k, c->a_next, &c->ctr->violations, s));
    KNOR_CUDA(c, mark(9));
    KNOR_CUDA(c, mark(10));
    KNOR_CUDA(c, prec_delta_sums(c->X, c->n, c->d, c->st, c->a_next, c->part_S, c->part_cnt, c->ctr, c->k,
                                 fl + F_NSLOTS, fl + F_FRESH, 8 * c->num_sms, s));
    KNOR_CUDA(c, mark(11));
    KNOR_CUDA(c, mark(4));
    KNOR_CUDA(c, launch_reduce(c->fp, fl + F_NSLOTS, fl + F_FRESH, s));
    KNOR_CUDA(c, mark(5));
    FinParams f = c->fp;
    f.snapshot = 1;
    f.cond_handle = cond;
    KNOR_CUDA(c, mark(6));
    KNOR_CUDA(c, launch_table(f, fl + F_MODE_DENSE, 0, 0, 1, s));
    KNOR_CUDA(c, mark(7));
    return KNOR_OK;
}

static knor_status enqueue_iteration(knor_ctx *c, cudaStream_t s, unsigned long long cond) {
    if (c->prec) return enqueue_prec(c, s, cond, nullptr);
    int32_t *fl = c->flags;
    if (c->ip_dense.acc_global) { // one slot, accumulated by atomics: start from zero
        KNOR_CUDA(c, cudaMemsetAsync(c->part_S, 0, sizeof(double) * (size_t)c->k * c->d, s));
        KNOR_CUDA(c, cudaMemsetAsync(c->part_cnt, 0, sizeof(long long) * (size_t)c->k, s));
    }
    KNOR_CUDA(c, scan_dense(c, s));
    if (!c->opts.no_prune) {
        KNOR_CUDA(c, scan_select(c, s));
        KNOR_CUDA(c, scan_mti(c, s));
    }
    KNOR_CUDA(c, scan_delta(c, s));
    KNOR_CUDA(c, launch_reduce(c->fp, fl + F_NSLOTS, fl + F_FRESH, s));
    FinParams f = c->fp;
    f.snapshot = 1;
    f.cond_handle = cond;
    KNOR_CUDA(c, launch_table(f, fl + F_MODE_DENSE, c->opts.no_prune ? 0 : 1, c->opts.full_recompute_every,
                              c->opts.no_prune ? 1 : 0, s));
    if (c->opts.debug_invariants && !c->opts.no_prune)
        KNOR_CUDA(c, launch_check_bounds(c->X, c->n, c->d, c->st, c->C32, c->F, c->stats, fl + F_RUN_ITER, s));
    if (c->opts.debug_invariants && c->opts.elkan)
        KNOR_CUDA(c, launch_elkan_check(c->dv, c->ip_mti, c->stats, fl + F_RUN_ITER, s));
    return KNOR_OK;
}

// One iteration launched kernel by kernel with events around each (profiling
// mode).  The host decides which scan runs with the same rule k_table writes
// into the device flag, so the launched scan is the one that does the work.
static knor_status profiled_iteration(knor_ctx *c) {
    cudaStream_t s = c->stream;
    int32_t *fl = c->flags;
    if (c->ev.empty()) {
        c->ev.resize(2 * KNOR_KERNEL_COUNT);
        for (auto &e : c->ev) KNOR_CUDA(c, cudaEventCreate(&e));
    }
    if (c->prec) {
        knor_status st = enqueue_prec(c, s, 0, c->ev.data());
        if (st != KNOR_OK) return st;
        KNOR_CUDA(c, cudaStreamSynchronize(s));
        const int kinds[] = {KNOR_KERNEL_DENSE, KNOR_KERNEL_RECHECK, KNOR_KERNEL_SUMS, KNOR_KERNEL_REDUCE,
                             KNOR_KERNEL_TABLE};
        const int evs[] = {0, 8, 10, 4, 6};
        for (int q = 0; q < 5; ++q) {
            float ms = 0.0f;
            KNOR_CUDA(c, cudaEventElapsedTime(&ms, c->ev[evs[q]], c->ev[evs[q] + 1]));
            c->prof.ms[kinds[q]] += ms;
            c->prof.launches[kinds[q]] += 1;
        }
        c->host_total_iter += 1;
        return KNOR_OK;
    }
    const int m = c->opts.full_recompute_every;
    const int tot = c->host_total_iter;
    const bool dense = c->opts.no_prune || tot == 0 || (m > 0 && (tot + 1) % m == 0);
    bool used[KNOR_KERNEL_COUNT] = {};
    if (c->ip_dense.acc_global) {
        KNOR_CUDA(c, cudaMemsetAsync(c->part_S, 0, sizeof(double) * (size_t)c->k * c->d, s));
        KNOR_CUDA(c, cudaMemsetAsync(c->part_cnt, 0, sizeof(long long) * (size_t)c->k, s));
    }
    auto timed = [&](int kind, cudaError_t (*fn)(knor_ctx *, cudaStream_t)) -> knor_status {
        KNOR_CUDA(c, cudaEventRecord(c->ev[2 * kind], s));
        KNOR_CUDA(c, fn(c, s));
        KNOR_CUDA(c, cudaEventRecord(c->ev[2 * kind + 1], s));
        used[kind] = true;
        return KNOR_OK;
    };
    knor_status ks = KNOR_OK;
    if (dense) {
        ks = timed(KNOR_KERNEL_DENSE, scan_dense);
        if (ks == KNOR_OK && c->dense_split) ks = timed(KNOR_KERNEL_DELTA, scan_delta);
    } else {
        if (c->mti_split && !c->opts.elkan) ks = timed(KNOR_KERNEL_SELECT, scan_select);
        if (ks == KNOR_OK) ks = timed(KNOR_KERNEL_MTI, scan_mti);
        if (ks == KNOR_OK && c->mti_split) ks = timed(KNOR_KERNEL_DELTA, scan_delta);
    }
    if (ks != KNOR_OK) return ks;
    KNOR_CUDA(c, cudaEventRecord(c->ev[4], s));
    KNOR_CUDA(c, launch_reduce(c->fp, fl + F_NSLOTS, fl + F_FRESH, s));
    KNOR_CUDA(c, cudaEventRecord(c->ev[5], s));
    FinParams f = c->fp;
    f.snapshot = 1;
    f.cond_handle = 0;
    KNOR_CUDA(c, cudaEventRecord(c->ev[6], s));
    KNOR_CUDA(c, launch_table(f, fl + F_MODE_DENSE, c->opts.no_prune ? 0 : 1, m, c->opts.no_prune ? 1 : 0, s));
    KNOR_CUDA(c, cudaEventRecord(c->ev[7], s));
    used[KNOR_KERNEL_REDUCE] = used[KNOR_KERNEL_TABLE] = true;
    if (c->opts.debug_invariants && !c->opts.no_prune)
        KNOR_CUDA(c, launch_check_bounds(c->X, c->n, c->d, c->st, c->C32, c->F, c->stats, fl + F_RUN_ITER, s));
    if (c->opts.debug_invariants && c->opts.elkan)
        KNOR_CUDA(c, launch_elkan_check(c->dv, c->ip_mti, c->stats, fl + F_RUN_ITER, s));
    KNOR_CUDA(c, cudaStreamSynchronize(s));
    for (int kk = 0; kk < KNOR_KERNEL_COUNT; ++kk) {
        if (!used[kk]) continue;
        float ms = 0.0f;
        KNOR_CUDA(c, cudaEventElapsedTime(&ms, c->ev[2 * kk], c->ev[2 * kk + 1]));
        c->prof.ms[kk] += ms;
        c->prof.launches[kk] += 1;
    }
    c->host_total_iter += 1;
    return KNOR_OK;
}

static knor_status build_graphs(knor_ctx *c) {
    // single iteration
    {
        cudaGraph_t g = nullptr;
        KNOR_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        knor_status st = enqueue_iteration(c, c->stream, 0);
        cudaGraph_t got = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &got);
        if (st != KNOR_OK) {
            if (got) cudaGraphDestroy(got);
            return st;
        }
        KNOR_CUDA(c, e);
        g = got;
        e = cudaGraphInstantiate(&c->iter_exec, g, 0);
        cudaGraphDestroy(g);
        KNOR_CUDA(c, e);
    }
    // whole run: WHILE node whose body is one iteration; k_table sets the
    // condition from the iteration's changed count and the run limit.
    {
        cudaGraph_t g = nullptr;
        KNOR_CUDA(c, cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) { cudaGraphDestroy(g); KNOR_CUDA(c, e); }
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        if (e != cudaSuccess) { cudaGraphDestroy(g); KNOR_CUDA(c, e); }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { cudaGraphDestroy(g); KNOR_CUDA(c, e); }
        knor_status st = enqueue_iteration(c, c->stream, (unsigned long long)h);
        cudaGraph_t got = nullptr;
        e = cudaStreamEndCapture(c->stream, &got);
        if (st != KNOR_OK) { cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) { cudaGraphDestroy(g); KNOR_CUDA(c, e); }
        e = cudaGraphInstantiate(&c->run_exec, g, 0);
        cudaGraphDestroy(g);
        KNOR_CUDA(c, e);
    }
    return KNOR_OK;
}

// C^0 is in c->C0: reset centroids, sums, bounds and tables to iteration 0.
static knor_status reset_run(knor_ctx *c) {
    cudaStream_t s = c->stream;
    const size_t kd = (size_t)c->k * c->d;
    KNOR_CUDA(c, cudaMemcpyAsync(c->C64, c->C0, kd * sizeof(double), cudaMemcpyDeviceToDevice, s));
    KNOR_CUDA(c, launch_round_c32(c->C0, c->C32, (int64_t)kd, s));
    KNOR_CUDA(c, cudaMemcpyAsync(c->C32n, c->C32, kd * sizeof(float), cudaMemcpyDeviceToDevice, s));
    KNOR_CUDA(c, cudaMemsetAsync(c->S, 0, kd * sizeof(double), s));
    KNOR_CUDA(c, cudaMemsetAsync(c->cnt, 0, (size_t)c->k * sizeof(long long), s));
    KNOR_CUDA(c, cudaMemsetAsync(c->cnt_next, 0, (size_t)c->k * sizeof(long long), s));
    KNOR_CUDA(c, cudaMemsetAsync(c->F, 0, (size_t)c->k * sizeof(float), s));
    KNOR_CUDA(c, cudaMemsetAsync(c->ctr, 0, sizeof(Counters), s));
    KNOR_CUDA(c, launch_init_state(c->st, c->n, s));
    int32_t fl[F_COUNT] = {0, 0, 1, 1, 1, 1, 0};
    KNOR_CUDA(c, cudaMemcpyAsync(c->flags, fl, sizeof(fl), cudaMemcpyHostToDevice, s));
    c->host_total_iter = 0;
    // tables for C^0 (drift 0, no record)
    FinParams f = c->fp;
    f.snapshot = 0;
    f.cond_handle = 0;
    KNOR_CUDA(c, launch_table(f, c->flags + F_MODE_DENSE, c->opts.no_prune ? 0 : 1, 0, 1, s));
    KNOR_CUDA(c, cudaStreamSynchronize(s));
    return KNOR_OK;
}

extern "C" {

const char *knor_version(void) { return "0.1.0"; }

const char *knor_last_error(const knor_ctx *ctx) {
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

void *knor_stream(const knor_ctx *ctx) { return ctx ? (void *)ctx->stream : nullptr; }

void knor_destroy(knor_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->dev);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
}

knor_status knor_create(const float *points, int64_t n, int32_t d, int32_t k, knor_init init, uint64_t seed,
                        const knor_opts *opts, knor_ctx **out) {
    g_create_err.clear();
    if (!out) { g_create_err = "knor_create: out is NULL"; return KNOR_ERR_ARG; }
    *out = nullptr;
    if (!points) { g_create_err = "knor_create: points is NULL"; return KNOR_ERR_ARG; }
    if (n < 1 || d < 1 || k < 1) { g_create_err = "knor_create: need n >= 1, d >= 1, k >= 1"; return KNOR_ERR_ARG; }
    if ((int64_t)k > n) { g_create_err = "knor_create: k > n"; return KNOR_ERR_ARG; }
    if ((double)n * (double)d > std::ldexp(1.0, 40)) { g_create_err = "knor_create: n*d above 2^40"; return KNOR_ERR_ARG; }
    if (n > (int64_t)1 << 31) { g_create_err = "knor_create: n above 2^31"; return KNOR_ERR_ARG; }
    if ((double)k * (double)d > (double)(1 << 28)) { g_create_err = "knor_create: k*d above 2^28"; return KNOR_ERR_ARG; }
    if (init != KNOR_INIT_FORGY && init != KNOR_INIT_EXPLICIT && init != KNOR_INIT_KMEANSPP) {
        g_create_err = "knor_create: bad init";
        return KNOR_ERR_ARG;
    }
    knor_opts o{};
    if (opts) o = *opts;
    if (o.precision != KNOR_PREC_FP32 && o.precision != KNOR_PREC_BF16 && o.precision != KNOR_PREC_FP16 &&
        o.precision != KNOR_PREC_FP8) {
        g_create_err = "knor_create: precision must be one of KNOR_PREC_FP32, _BF16, _FP16, _FP8";
        return KNOR_ERR_ARG;
    }
    const bool tc_form = o.precision != KNOR_PREC_FP32;
    if (tc_form && ((d != 64 && d != 128) || k > 8192 || (o.precision == KNOR_PREC_FP8 && d != 128))) {
        g_create_err = "knor_create: the tensor-core forms need d = 64 or 128 (FP8: 128) and k <= 8192";
        return KNOR_ERR_ARG;
    }
    if (o.full_recompute_every < 0) { g_create_err = "knor_create: full_recompute_every < 0"; return KNOR_ERR_ARG; }
    if (o.points_in_host && (tc_form || is_device_ptr(points) || (reinterpret_cast<uintptr_t>(points) & 15) != 0)) {
        g_create_err = "knor_create: points_in_host needs FP32 distances and a 16-byte aligned host buffer";
        return KNOR_ERR_ARG;
    }
    if (o.elkan && (o.no_prune || tc_form || o.full_recompute_every != 0)) {
        g_create_err = "knor_create: elkan needs pruning, FP32 distances and full_recompute_every = 0";
        return KNOR_ERR_ARG;
    }

    knor_ctx *c = new knor_ctx();
    c->n = n; c->d = d; c->k = k; c->opts = o; c->init = init; c->seed = seed;
    auto bail = [&](knor_status st) {
        g_create_err = c->err;
        free_all(c);
        delete c;
        return st;
    };
#define KC(call) do { knor_status s_ = (call); if (s_ != KNOR_OK) return bail(s_); } while (0)
#define KCU(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { c->err = std::string(#call) + ": " + cudaGetErrorString(e_); cudaGetLastError(); return bail(e_ == cudaErrorMemoryAllocation ? KNOR_ERR_OOM : KNOR_ERR_CUDA); } } while (0)
    KCU(cudaGetDevice(&c->dev));
    KCU(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev));
    KCU(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    const size_t nd = (size_t)n * d, kd = (size_t)k * d;
    if (o.points_in_host) {
        // read in place: pinned memory is mapped already; pageable memory is
        // registered (mapped) for the context's lifetime
        cudaPointerAttributes at{};
        const bool pinned = cudaPointerGetAttributes(&at, points) == cudaSuccess && at.type == cudaMemoryTypeHost;
        cudaGetLastError();
        if (!pinned) {
            KCU(cudaHostRegister(const_cast<float *>(points), nd * sizeof(float),
                                 cudaHostRegisterMapped));
            c->host_registered = const_cast<float *>(points);
        }
        void *dp = nullptr;
        KCU(cudaHostGetDevicePointer(&dp, const_cast<float *>(points), 0));
        c->X = static_cast<float *>(dp);
        c->X_on_host = true;
    } else {
        KC(dalloc(c, &c->X, nd));
        KCU(cudaMemcpyAsync(c->X, points, nd * sizeof(float),
                            is_device_ptr(points) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    }
    KC(dalloc(c, &c->d_bad, 1));
    KCU(cudaMemsetAsync(c->d_bad, 0, sizeof(unsigned long long), c->stream));
    KCU(launch_validate(c->X, (int64_t)nd, c->d_bad, c->stream));
    unsigned long long bad = 0;
    KCU(cudaMemcpyAsync(&bad, c->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
    KCU(cudaStreamSynchronize(c->stream));
    if (bad) {
        c->err = "knor_create: " + std::to_string(bad) + " coordinates are NaN, infinite or above 1e15 in magnitude";
        return bail(KNOR_ERR_ARG);
    }
    KC(dalloc(c, &c->st, (size_t)n));
    KC(dalloc(c, &c->C0, kd));
    KC(dalloc(c, &c->C64, kd));
    KC(dalloc(c, &c->S, kd));
    KC(dalloc(c, &c->C32, kd));
    KC(dalloc(c, &c->C32n, kd));
    KC(dalloc(c, &c->halfD, (size_t)k * k));
    KC(dalloc(c, &c->s, (size_t)k));
    KC(dalloc(c, &c->F, (size_t)k));
    KC(dalloc(c, &c->cnt, (size_t)k));
    KC(dalloc(c, &c->cnt_next, (size_t)k));
    KC(dalloc(c, &c->ctr, 1));
    KC(dalloc(c, &c->stats, kStatsCap));
    KC(dalloc(c, &c->flags, F_COUNT));
    KCU(cudaMallocHost((void **)&c->h_stats, sizeof(IterStats) * kStatsCap));

    // kernel configurations and persistent grids
    c->dv = supported_dv(d);
    int bd = 0, bm = 0;
    {
        // The split kernels (per-warp ranges, change lists, k_mti_delta)
        // where they fit: the MTI scan (unless KNOR_MTI_KERNEL = 1 selects the
        // one-kernel warp scan, for comparisons) and the dense scan (unless
        // full_recompute_every asks for sums rebuilt from every point).
        IterParams ps{};
        const int choice = o.elkan ? 0 : getenv_int("KNOR_MTI_KERNEL", 0);
        const size_t ssc = !tc_form ? plan_layout_scan(c, ps) : 0;
        int bsplit = 0, bsel = 0;
        if (ssc) {
            int bs = 0, bdl = 0;
            KCU(mti_scan_attr(c->dv, SP_WPB, ssc, &bsplit));
            // heavy points (Clause 2 would leave them M = k / 3 or more
            // candidates) from k = 8 on; KNOR_SEL_M (a tuning knob) sets M,
            // 0 turns the split off
            c->sel_M = std::max(0, getenv_int("KNOR_SEL_M", k >= 8 ? std::max(2, k / 3) : 0));
            c->smem_sel = plan_layout_sel(c, c->ip_sel);
            KCU(mti_sel_attr(SP_WPB, c->smem_sel, &bs));
            bsel = bs;
            KCU(mti_delta_attr(c->dv, (size_t)SP_WPB * ps.dl_split * ps.dl_warp_stride, ps.dl_split, &bdl));
            if (bs < 1 || bdl < 1) bsplit = 0;
        }
        c->mti_split = bsplit > 0 && choice == 0 && !o.no_prune;
        c->dense_split = bsplit > 0 && o.full_recompute_every == 0;
        if (o.elkan) {
            int be = 0;
            if (bsplit > 0) KCU(elkan_scan_attr(c->dv, ssc, &be));
            if (bsplit < 1 || be < bsplit) {
                c->err = "knor_create: elkan needs d in {8, 16, 32, 64}, k <= 110 and k*d <= 8192";
                return bail(KNOR_ERR_ARG);
            }
        }
        IterParams pw{}, pm{};
        int split_mult = bsplit;
        if (c->dense_split) {
            // the dense scan's own layout: centroids and drift (no k x k
            // table), then per warp DS_ROWS-row tiles, double-buffered
            c->ip_dense = ps;
            size_t off = 0;
            auto take = [&](size_t bytes) -> int32_t {
                const size_t o = off;
                off = (off + bytes + 15) & ~(size_t)15;
                return (int32_t)o;
            };
            c->ip_dense.off_cent = take((size_t)k * d * 4);
            c->ip_dense.off_F = take((size_t)k * 4);
            c->ip_dense.off_halfD = c->ip_dense.off_s = -1;
            c->ip_dense.sp_off_warp = take(0);
            c->ip_dense.sp_warp_stride = 2 * DS_ROWS * ps.sp_rs * 4;
            c->smem_dense = off + (size_t)SP_WPB * c->ip_dense.sp_warp_stride;
            KCU(dense_scan_attr(c->dv, c->smem_dense, &bd));
            if (bd < 1) c->dense_split = false;
            // where the dense scan fits twice as many CTAs per SM as the MTI
            // scan, the split grid takes a whole multiple of the MTI scan's
            // CTAs per SM: the dense scan gets the warps, the MTI kernels run
            // in whole waves
            else if (bsplit > 0 && bd >= 2 * bsplit) split_mult = bsplit * (bd / bsplit);
        }
        if (!c->dense_split) {
            const size_t sw = plan_layout_warp(c, false, pw);
            if (sw) { c->ip_dense = pw; c->smem_dense = sw; KCU(dense_w_attr(c->dv, sw, &bd)); }
            else { c->smem_dense = plan_layout(c, false, c->ip_dense); KCU(dense_attr(c->dv, c->smem_dense, &bd)); }
        }
        const size_t sm = c->mti_split ? 0 : plan_layout_warp(c, true, pm);
        if (c->mti_split) { c->ip_mti = ps; c->smem_mti = ssc; bm = bsplit; }
        else if (sm) { c->ip_mti = pm; c->smem_mti = sm; KCU(mti_w_attr(c->dv, sm, &bm)); }
        else { c->smem_mti = plan_layout(c, true, c->ip_mti); KCU(mti_attr(c->dv, c->smem_mti, &bm)); }
        c->grid_split = split_mult * c->num_sms;
        if (c->mti_split && bsel >= 2 * split_mult && getenv_int("KNOR_SEL_MULT", 2) >= 2) c->sel_mult = 2;
    }
    if (bd < 1 || bm < 1) { c->err = "knor_create: kernel does not fit on an SM"; return bail(KNOR_ERR_CUDA); }
    // (the split kernels all run on the split grid, in waves where fewer of
    // their CTAs fit on an SM)
    c->grid_dense = c->dense_split ? c->grid_split : bd * c->num_sms;
    c->grid_mti = c->mti_split ? c->grid_split : bm * c->num_sms;
    // Both scans use the same accumulation mode: per-CTA partial slots, or,
    // when k x d sums do not fit in shared memory, one slot updated by FP64
    // atomics.
    const int acc_global = (c->ip_dense.acc_global || c->ip_mti.acc_global || tc_form) ? 1 : 0;
    if (acc_global && (c->ip_dense.warp_kernels || c->ip_mti.warp_kernels)) {
        // the warp kernels always write per-CTA slots: use the CTA kernels for both
        c->ip_dense = IterParams{};
        c->ip_mti = IterParams{};
        c->mti_split = c->dense_split = false;
        c->smem_dense = plan_layout(c, false, c->ip_dense);
        c->smem_mti = plan_layout(c, true, c->ip_mti);
        KCU(dense_attr(c->dv, c->smem_dense, &bd));
        KCU(mti_attr(c->dv, c->smem_mti, &bm));
        c->grid_dense = bd * c->num_sms;
        c->grid_mti = bm * c->num_sms;
    }
    c->part_stride = acc_global ? 1 : std::max(c->grid_dense, c->grid_mti);
    KC(dalloc(c, &c->part_S, kd * c->part_stride));
    KC(dalloc(c, &c->part_cnt, (size_t)k * c->part_stride));
    fill_common(c, c->ip_dense);
    fill_common(c, c->ip_mti);
    if (c->ip_mti.warp_kernels == 1) {
        // per-warp TwoSum accumulators of k_mti_w (global, warp-private)
        KC(dalloc(c, &c->wacc, (size_t)c->grid_mti * WPC * 2 * kd));
        c->ip_mti.wacc = c->wacc;
    }
    if (c->mti_split || c->dense_split) {
        // per warp of the split grid: change lists with room for every point
        // of its range, and (MTI) batch records, one per 32 points of the
        // range plus one partial bucket per cluster and the unassigned one
        const int64_t nw = (int64_t)c->grid_split * SP_WPB;
        const int64_t units = (n + WPA - 1) / WPA;
        const int64_t range = ((units + nw - 1) / nw) * WPA;
        const int64_t cap = (range + 31) / 32 + k + 1;
        // k_mti_sel: two warps per scan warp where twice the split grid's
        // CTAs fit on an SM (its warps wait on shared memory: more of them
        // hide more), each over half the range, with a record list of its own
        const int64_t nws = nw * c->sel_mult;
        const int64_t range_s = ((units + nws - 1) / nws) * WPA;
        const int64_t cap_s = (range_s + 31) / 32 + k + 1;
        if (c->mti_split) {
            KC(dalloc(c, &c->rec, (size_t)(nws * cap_s * SP_REC)));
            KC(dalloc(c, &c->rec_cnt, (size_t)nws));
            if (c->sel_M > 0) {
                KC(dalloc(c, &c->theta, (size_t)k));
                c->ip_sel.theta = c->theta;
            }
        }
        KC(dalloc(c, &c->chg, (size_t)(nw * cap * 32)));
        KC(dalloc(c, &c->chg_cnt, (size_t)nw));
        fill_common(c, c->ip_sel);
        if (o.elkan) {
            // Elkan's lower bounds, n x k, cluster-major
            KC(dalloc(c, &c->lb, (size_t)n * k));
            const float ginv = (float)(1.0 - (d + 2) * std::ldexp(1.0, -24));
            const float ginv_dn = (double)ginv > 1.0 - (d + 2) * std::ldexp(1.0, -24) ? std::nextafter(ginv, 0.0f) : ginv;
            for (IterParams *q : {&c->ip_mti, &c->ip_dense}) {
                q->lb = c->lb;
                q->ginv_dn = ginv_dn;
            }
        }
        c->ip_delta = c->mti_split ? c->ip_mti : c->ip_dense;
        for (IterParams *q : {&c->ip_mti, &c->ip_sel, &c->ip_dense, &c->ip_delta}) {
            q->rec = c->rec;
            q->rec_cnt = c->rec_cnt;
            q->rec_cap = cap_s;
            q->sel_mult = c->sel_mult;
            q->chg_cap = cap * 32;
            q->chg = c->chg;
            q->chg_cnt = c->chg_cnt;
            q->dl_dense = c->dense_split ? 1 : 0;
            q->dl_mti = c->mti_split ? 1 : 0;
        }
    }
    c->ip_dense.part_stride = c->part_stride;
    c->ip_mti.part_stride = c->part_stride;
    c->ip_delta.part_stride = c->part_stride;
    c->ip_dense.acc_global = c->ip_mti.acc_global = acc_global;
    {
        const std::string w = "<" + std::to_string(c->dv) + ">";
        c->kname[KNOR_KERNEL_DENSE] =
            c->dense_split ? "k_dense_scan" + w : (c->ip_dense.warp_kernels ? "k_dense_w" : "k_dense") + w;
        if (c->mti_split && !o.elkan) c->kname[KNOR_KERNEL_SELECT] = "k_mti_sel";
        if (c->mti_split || c->dense_split) c->kname[KNOR_KERNEL_DELTA] = "k_mti_delta" + w;
        c->kname[KNOR_KERNEL_MTI] =
            (c->mti_split ? (o.elkan ? "k_elkan_scan" : "k_mti_scan") : c->ip_mti.warp_kernels ? "k_mti_w" : "k_mti") + w;
        c->kname[KNOR_KERNEL_REDUCE] = "k_reduce";
        c->kname[KNOR_KERNEL_TABLE] = "k_table";
    }
    FinParams &f = c->fp;
    f.part_S = c->part_S; f.part_cnt = c->part_cnt; f.part_stride = c->part_stride;
    f.k = k; f.d = d;
    f.S = c->S; f.cnt = c->cnt; f.cnt_next = c->cnt_next; f.C64 = c->C64; f.C32 = c->C32; f.C32n = c->C32n;
    f.halfD = c->halfD; f.s = c->s; f.F = c->F; f.cnt_out = c->cnt; f.ctr = c->ctr; f.stats = c->stats;
    f.run_iter = c->flags + F_RUN_ITER; f.total_iter = c->flags + F_TOTAL_ITER;
    f.max_iters_dev = c->flags + F_MAX_ITERS;
    f.theta = c->theta;
    f.th_M = c->sel_M;

    if (tc_form) {
        // The precision form scans every point each iteration (no MTI bounds):
        // its sums move by deltas through partial slot 0.
        c->prec = true;
        c->opts.no_prune = 1;
        c->fmt = o.precision == KNOR_PREC_FP16 ? PREC_FMT_FP16
                 : o.precision == KNOR_PREC_FP8 ? PREC_FMT_FP8
                                                : PREC_FMT_BF16;
        const size_t esize = c->fmt == PREC_FMT_FP8 ? 1 : 2;
        KC(dalloc(c, (uint8_t **)&c->Xb, nd * esize));
        KC(dalloc(c, (uint8_t **)&c->Cb, kd * esize));
        KC(dalloc(c, &c->xn, (size_t)n));
        KC(dalloc(c, &c->cn, (size_t)k));
        KC(dalloc(c, &c->pit, 1));
        KC(dalloc(c, &c->absmax, 1));
        KC(dalloc(c, &c->a_next, (size_t)n));
        KC(dalloc(c, &c->rlist, (size_t)n));
        KC(dalloc(c, &c->rcand, (size_t)n * PREC_CANDS));
        KC(dalloc(c, (uint8_t **)&c->Xc, nd * esize));
        KC(dalloc(c, &c->rm1, (size_t)n));
        KC(dalloc(c, &c->rxn, (size_t)n));
        KC(dalloc(c, &c->rcount, 1));
        int ex = 0;
        if (c->fmt == PREC_FMT_FP16) {
            // point scale 2^ex from the largest |x_j| (read back once)
            float am = 0.0f;
            KCU(prec_absmax(c->X, (int64_t)nd, c->absmax, c->stream));
            KCU(cudaMemcpyAsync(&am, c->absmax, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
            KCU(cudaStreamSynchronize(c->stream));
            ex = prec_point_scale_exp(c->fmt, am);
        }
        c->xdn = c->xn;
        c->rxdn = c->rxn;
        if (c->fmt == PREC_FMT_FP8) {
            // per-dimension scales sigma_j = 2^ceil(log2 max_i |x_ij|) (so
            // |x_ij / sigma_j| <= 1), the points' scale 2^7, and the norms of
            // x / sigma for the bound
            KC(dalloc(c, &c->xdn, (size_t)n));
            KC(dalloc(c, &c->rxdn, (size_t)n));
            KC(dalloc(c, &c->sigma, (size_t)2 * d));
            std::vector<float> mx((size_t)d), sg((size_t)2 * d);
            KCU(prec_dim_absmax(c->X, n, d, c->sigma, c->stream));
            KCU(cudaMemcpyAsync(mx.data(), c->sigma, sizeof(float) * d, cudaMemcpyDeviceToHost, c->stream));
            KCU(cudaStreamSynchronize(c->stream));
            for (int j = 0; j < d; ++j) {
                int e = 0;
                if (mx[(size_t)j] > 0.0f) {
                    const float m = std::frexp(mx[(size_t)j], &e); // mx = m 2^e, m in [0.5, 1)
                    if (m == 0.5f) e -= 1;                          // e = ceil(log2 mx)
                }
                e = std::max(-60, std::min(60, e));
                sg[(size_t)j] = std::ldexp(1.0f, e);          // sigma_j
                sg[(size_t)d + j] = std::ldexp(1.0f, -e);     // 1 / sigma_j
            }
            KCU(cudaMemcpyAsync(c->sigma, sg.data(), sizeof(float) * 2 * d, cudaMemcpyHostToDevice, c->stream));
            ex = prec_point_scale_exp(c->fmt, 1.0f);
        }
        c->sx = std::ldexp(1.0f, ex);
        KCU(prec_points(c->X, n, d, c->fmt, c->sx, c->sigma ? c->sigma + d : nullptr, c->Xb, c->xn, c->xdn,
                        c->stream));
        KC(encode_op_map(c, c->tmX, c->Xb, (uint64_t)d, (uint64_t)n, 128));
        KC(encode_op_map(c, c->tmC, c->Cb, (uint64_t)d, (uint64_t)k, 256));
        KC(encode_op_map(c, c->tmXc, c->Xc, (uint64_t)d, (uint64_t)n, 128));
        c->prec_smem = prec_smem_bytes(d, k, (int)esize);
        int smem_optin = 0;
        KCU(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
        if (c->prec_smem > (size_t)smem_optin) {
            c->err = "knor_create: the precision form's shared-memory tiles for this k do not fit one CTA";
            return bail(KNOR_ERR_ARG);
        }
        KCU(prec_assign_attr(c->prec_smem));
        const int64_t ntile = (n + 127) / 128;
        c->prec_grid = (int)std::min<int64_t>(c->num_sms, ntile);
        PrecParams &pp = c->pp;
        pp.n = n; pp.d = d; pp.k = k; pp.xn = c->xn; pp.cn = c->cn; pp.it = c->pit;
        pp.a_next = c->a_next; pp.rlist = c->rlist; pp.rcount = c->rcount; pp.rcand = c->rcand;
        pp.rm1 = c->rm1; pp.rxn = c->rxn; pp.mode = 0;
        pp.xdn = c->xdn; pp.rxdn = c->rxdn;
        prec_error_constants(c->fmt, d, c->sx, pp);
        pp.err = c->flags + F_ERR;
        c->pp2 = pp;
        c->pp2.mode = 1;
        c->kname[KNOR_KERNEL_DENSE] = "k_tc_assign";
        c->kname[KNOR_KERNEL_RECHECK] =
            "k_prec_gather + k_tc_assign (candidates) + k_recheck<" + std::to_string(c->dv) + ">";
        c->kname[KNOR_KERNEL_SUMS] = "k_delta_sums";
    }
    // C^0
    if (init == KNOR_INIT_FORGY || init == KNOR_INIT_KMEANSPP) {
        if (init == KNOR_INIT_FORGY) c->init_idx = forgy_indices(n, k, seed);
        else KCU(kmeanspp_indices(c->X, n, d, k, seed, c->dv, c->num_sms, c->stream, c->init_idx));
        KC(dalloc(c, &c->d_idx, (size_t)k));
        KCU(cudaMemcpyAsync(c->d_idx, c->init_idx.data(), sizeof(int64_t) * k, cudaMemcpyHostToDevice, c->stream));
        KCU(launch_gather_rows(c->X, d, c->d_idx, k, c->C0, c->stream));
        c->c0_set = true;
    } else {
        KCU(cudaMemsetAsync(c->C0, 0, kd * sizeof(double), c->stream));
    }
    KC(reset_run(c));
    KC(build_graphs(c));
    *out = c;
    return KNOR_OK;
#undef KC
#undef KCU
}

knor_status knor_set_init_centroids(knor_ctx *c, const double *c_kxd) {
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    if (!c_kxd) return fail(c, KNOR_ERR_ARG, "knor_set_init_centroids: NULL centroids");
    const size_t kd = (size_t)c->k * c->d;
    std::vector<double> h(kd);
    if (is_device_ptr(c_kxd)) KNOR_CUDA(c, cudaMemcpy(h.data(), c_kxd, kd * sizeof(double), cudaMemcpyDeviceToHost));
    else std::memcpy(h.data(), c_kxd, kd * sizeof(double));
    for (double v : h)
        if (!std::isfinite(v) || std::fabs(v) > 1e15)
            return fail(c, KNOR_ERR_ARG, "knor_set_init_centroids: coordinate not finite or above 1e15");
    KNOR_CUDA(c, cudaMemcpyAsync(c->C0, h.data(), kd * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->c0_set = true;
    return reset_run(c);
}

knor_status knor_reset(knor_ctx *c) {
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    return reset_run(c);
}

// A bounded device-side wait that gave up leaves F_ERR set.
static knor_status check_timeout(knor_ctx *c) {
    int32_t err = 0;
    KNOR_CUDA(c, cudaMemcpy(&err, c->flags + F_ERR, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) {
        cudaMemsetAsync(c->flags + F_ERR, 0, sizeof(int32_t), c->stream);
        cudaStreamSynchronize(c->stream);
        return fail(c, KNOR_ERR_TIMEOUT, "a device-side wait timed out (results of this iteration are invalid)");
    }
    return KNOR_OK;
}

static knor_status read_stats(knor_ctx *c, int count, knor_iter_stats *out) {
    knor_status st = check_timeout(c);
    if (st != KNOR_OK) return st;
    if (count <= 0 || !out) return KNOR_OK;
    KNOR_CUDA(c, cudaMemcpyAsync(c->h_stats, c->stats, sizeof(IterStats) * count, cudaMemcpyDeviceToHost, c->stream));
    KNOR_CUDA(c, cudaStreamSynchronize(c->stream));
    static_assert(sizeof(IterStats) == sizeof(knor_iter_stats), "stats layout");
    std::memcpy(out, c->h_stats, sizeof(IterStats) * count);
    return KNOR_OK;
}

knor_status knor_iterate(knor_ctx *c, knor_iter_stats *out) {
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    if (!c->c0_set) return fail(c, KNOR_ERR_STATE, "knor_iterate: explicit init centroids not set");
    KNOR_CUDA(c, cudaMemsetAsync(c->flags + F_RUN_ITER, 0, sizeof(int32_t), c->stream));
    if (c->profiling) {
        knor_status st = profiled_iteration(c);
        if (st != KNOR_OK) return st;
    } else {
        KNOR_CUDA(c, cudaGraphLaunch(c->iter_exec, c->stream));
        KNOR_CUDA(c, cudaStreamSynchronize(c->stream));
        c->host_total_iter += 1;
    }
    return read_stats(c, 1, out);
}

knor_status knor_run(knor_ctx *c, int32_t max_iters, int32_t *iters_done, knor_iter_stats *per_iter) {
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    if (iters_done) *iters_done = 0;
    if (max_iters < 0 || max_iters > kStatsCap)
        return fail(c, KNOR_ERR_ARG, "knor_run: max_iters must be in [0, 65536]");
    if (!c->c0_set) return fail(c, KNOR_ERR_STATE, "knor_run: explicit init centroids not set");
    if (max_iters == 0) return KNOR_OK;
    int32_t hv[3] = {0, 0, max_iters};
    KNOR_CUDA(c, cudaMemsetAsync(c->flags + F_RUN_ITER, 0, sizeof(int32_t), c->stream));
    if (c->profiling) {
        int32_t done = 0;
        for (int t = 0; t < max_iters; ++t) {
            knor_status st = profiled_iteration(c);
            if (st != KNOR_OK) return st;
            done = t + 1;
            IterStats r;
            KNOR_CUDA(c, cudaMemcpy(&r, c->stats + t, sizeof(r), cudaMemcpyDeviceToHost));
            if (r.changed == 0) break;
        }
        if (iters_done) *iters_done = done;
        return read_stats(c, done, per_iter);
    }
    KNOR_CUDA(c, cudaMemcpyAsync(c->flags + F_MAX_ITERS, &hv[2], sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    KNOR_CUDA(c, cudaGraphLaunch(c->run_exec, c->stream));
    int32_t done = 0;
    KNOR_CUDA(c, cudaMemcpyAsync(&done, c->flags + F_RUN_ITER, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    KNOR_CUDA(c, cudaStreamSynchronize(c->stream));
    c->host_total_iter += done;
    if (iters_done) *iters_done = done;
    return read_stats(c, done, per_iter);
}

knor_status knor_test_fail_alloc(int32_t after) {
    g_fail_alloc_after.store(after < 0 ? -1 : (int64_t)after);
    return KNOR_OK;
}

knor_status knor_test_raise_error_flag(knor_ctx *c) {
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    const int32_t one = 1;
    KNOR_CUDA(c, cudaMemcpyAsync(c->flags + F_ERR, &one, sizeof(one), cudaMemcpyHostToDevice, c->stream));
    KNOR_CUDA(c, cudaStreamSynchronize(c->stream));
    return KNOR_OK;
}

const char *knor_kernel_name(const knor_ctx *c, int32_t kernel) {
    if (!c || kernel < 0 || kernel >= KNOR_KERNEL_COUNT) return "";
    return c->kname[kernel].c_str();
}

knor_status knor_set_profiling(knor_ctx *c, int32_t on) {
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    c->profiling = on != 0;
    return KNOR_OK;
}

knor_status knor_get_profile(knor_ctx *c, knor_profile *out, int32_t reset_after) {
    if (!c || !out) return KNOR_ERR_ARG;
    c->err.clear();
    *out = c->prof;
    if (reset_after) c->prof = knor_profile{};
    return KNOR_OK;
}

knor_status knor_get_assignments(const knor_ctx *cc, int32_t *out_n) {
    knor_ctx *c = const_cast<knor_ctx *>(cc);
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    if (!out_n) return fail(c, KNOR_ERR_ARG, "knor_get_assignments: NULL output");
    if (is_device_ptr(out_n)) {
        KNOR_CUDA(c, launch_extract_assign(c->st, c->n, out_n, c->stream));
        KNOR_CUDA(c, cudaStreamSynchronize(c->stream));
        return KNOR_OK;
    }
    int32_t *tmp = nullptr;
    knor_status s = dalloc(c, &tmp, (size_t)c->n);
    if (s != KNOR_OK) return s;
    cudaError_t e = launch_extract_assign(c->st, c->n, tmp, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_n, tmp, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    KNOR_CUDA(c, e);
    return KNOR_OK;
}

static knor_status copy_out(knor_ctx *c, void *dst, const void *src, size_t bytes) {
    KNOR_CUDA(c, cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
    KNOR_CUDA(c, cudaStreamSynchronize(c->stream));
    return KNOR_OK;
}

knor_status knor_get_centroids(const knor_ctx *cc, double *out) {
    knor_ctx *c = const_cast<knor_ctx *>(cc);
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    if (!out) return fail(c, KNOR_ERR_ARG, "knor_get_centroids: NULL output");
    return copy_out(c, out, c->C64, sizeof(double) * (size_t)c->k * c->d);
}

knor_status knor_get_centroids_f32(const knor_ctx *cc, float *out) {
    knor_ctx *c = const_cast<knor_ctx *>(cc);
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    if (!out) return fail(c, KNOR_ERR_ARG, "knor_get_centroids_f32: NULL output");
    return copy_out(c, out, c->C32, sizeof(float) * (size_t)c->k * c->d);
}

knor_status knor_get_init_indices(const knor_ctx *c, int64_t *out_k) {
    if (!c) return KNOR_ERR_ARG;
    c->err.clear();
    if (!out_k) return fail(c, KNOR_ERR_ARG, "knor_get_init_indices: NULL output");
    if (c->init == KNOR_INIT_EXPLICIT) return fail(c, KNOR_ERR_STATE, "knor_get_init_indices: context uses explicit init");
    std::memcpy(out_k, c->init_idx.data(), sizeof(int64_t) * c->k);
    return KNOR_OK;
}

knor_status knor_get_iteration(const knor_ctx *cc, int32_t *out) {
    knor_ctx *c = const_cast<knor_ctx *>(cc);
    if (!c || !out) return KNOR_ERR_ARG;
    c->err.clear();
    KNOR_CUDA(c, cudaMemcpyAsync(out, c->flags + F_TOTAL_ITER, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    KNOR_CUDA(c, cudaStreamSynchronize(c->stream));
    return KNOR_OK;
}

// State image: header | C0 | C64 | S | cnt | C32 | F | halfD | s | st
static size_t state_size(const knor_ctx *c) {
    const size_t kd = (size_t)c->k * c->d, k = (size_t)c->k;
    return sizeof(StateHeader) + 3 * kd * sizeof(double) + k * sizeof(long long) + kd * sizeof(float) +
           k * sizeof(float) + k * k * sizeof(float) + k * sizeof(float) + (size_t)c->n * sizeof(PtState) +
           (c->lb ? (size_t)c->n * k * sizeof(float) : 0);
}

knor_status knor_get_state(const knor_ctx *cc, void *buf, size_t *size) {
    knor_ctx *c = const_cast<knor_ctx *>(cc);
    if (!c || !size) return KNOR_ERR_ARG;
    c->err.clear();
    const size_t need = state_size(c);
    if (!buf) { *size = need; return KNOR_OK; }
    if (*size < need) return fail(c, KNOR_ERR_ARG, "knor_get_state: buffer too small");
    int32_t fl[F_COUNT];
    KNOR_CUDA(c, cudaMemcpy(fl, c->flags, sizeof(fl), cudaMemcpyDeviceToHost));
    StateHeader h{kStateMagic, kStateVersion, c->n, c->d, c->k, c->opts.no_prune, c->opts.precision,
                  c->opts.full_recompute_every, fl[F_TOTAL_ITER], fl[F_MODE_DENSE], c->opts.elkan};
    char *p = static_cast<char *>(buf);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const size_t kd = (size_t)c->k * c->d, k = (size_t)c->k;
    struct Part { const void *src; size_t bytes; } parts[] = {
        {c->C0, kd * 8}, {c->C64, kd * 8}, {c->S, kd * 8}, {c->cnt, k * 8}, {c->C32, kd * 4}, {c->F, k * 4},
        {c->halfD, k * k * 4}, {c->s, k * 4}, {c->st, (size_t)c->n * sizeof(PtState)},
        {c->lb, c->lb ? (size_t)c->n * k * 4 : 0}};
    for (auto &pt : parts) {
        if (!pt.bytes) continue;
        KNOR_CUDA(c, cudaMemcpyAsync(p, pt.src, pt.bytes, cudaMemcpyDeviceToHost, c->stream));
        p += pt.bytes;
    }
    KNOR_CUDA(c, cudaStreamSynchronize(c->stream));
    *size = need;
    return KNOR_OK;
}

knor_status knor_set_state(knor_ctx *c, const void *buf, size_t size) {
    if (!c || !buf) return KNOR_ERR_ARG;
    c->err.clear();
    if (size != state_size(c)) return fail(c, KNOR_ERR_ARG, "knor_set_state: size does not match this context");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kStateMagic || h.version != kStateVersion || h.n != c->n || h.d != c->d || h.k != c->k ||
        h.no_prune != c->opts.no_prune || h.precision != c->opts.precision ||
        h.recompute != c->opts.full_recompute_every || h.pad != c->opts.elkan)
        return fail(c, KNOR_ERR_ARG, "knor_set_state: state is from a context with other sizes or options");
    const char *p = static_cast<const char *>(buf) + sizeof(h);
    const size_t kd = (size_t)c->k * c->d, k = (size_t)c->k;
    struct Part { void *dst; size_t bytes; } parts[] = {
        {c->C0, kd * 8}, {c->C64, kd * 8}, {c->S, kd * 8}, {c->cnt, k * 8}, {c->C32, kd * 4}, {c->F, k * 4},
        {c->halfD, k * k * 4}, {c->s, k * 4}, {c->st, (size_t)c->n * sizeof(PtState)},
        {c->lb, c->lb ? (size_t)c->n * k * 4 : 0}};
    for (auto &pt : parts) {
        if (!pt.bytes) continue;
        KNOR_CUDA(c, cudaMemcpyAsync(pt.dst, p, pt.bytes, cudaMemcpyHostToDevice, c->stream));
        p += pt.bytes;
    }
    KNOR_CUDA(c, launch_theta(c->fp, c->stream)); // k_mti_sel's thresholds from the restored table
    int32_t fl[F_COUNT] = {0, h.total_iter, 1, h.mode_dense, 1, 1, 0};
    c->host_total_iter = h.total_iter;
    KNOR_CUDA(c, cudaMemcpyAsync(c->flags, fl, sizeof(fl), cudaMemcpyHostToDevice, c->stream));
    KNOR_CUDA(c, cudaMemsetAsync(c->ctr, 0, sizeof(Counters), c->stream));
    KNOR_CUDA(c, cudaStreamSynchronize(c->stream));
    c->c0_set = true;
    return KNOR_OK;
}

} // extern "C"

// batch.cu -- the batched form: m independent k-means problems advanced
// together, one iteration of every active problem per step.
//
// All instances live in one set of concatenated device arrays (points,
// per-point state, centroids, sums, tables), addressed through a per-instance
// descriptor.  The points are cut into work units (instance, point range);
// the units are ordered longest-processing-time first (cost = points x k x d)
// and one persistent kernel drains them through an atomic counter -- the GPU
// counterpart of the paper's task queue with work stealing ("Parallel Lloyd's
// Algorithm", NUMA-aware task scheduling): a CTA that finishes early simply
// takes the next unit, and the costly units are handed out first so the tail
// is short.  That kernel full-scans (iteration 1, plain Lloyd, instances in
// dense mode); an MTI iteration runs sort-segmented over the whole batch
// instead: Clause 1 on every point appends the survivors to the segment of
// their cluster, and warps scan batches of 32 survivors of one cluster.
// Every point runs the same MTI test and pruned scan as in the single-problem
// scan (Clauses 1-3 with the rounding slack), so an instance gets exactly the
// assignments it would get alone from the same centroids; cluster sums move
// by the deltas of the points that changed cluster (FP64).  K5 (merge +
// finalize) and K1 (drift, half distances, s)
// are batched launches over all centroids of all active instances; a small
// bookkeeping kernel masks the instances that converged.  An iteration is one
// CUDA graph; a run is a graph with a device-side WHILE loop.
//
// The unit size per (d, k) bucket and the number of persistent CTAs per SM
// are chosen by a grid search over dry scans (no state written) at creation,
// cached per device and bucket for the process (and in a file when
// KNOR_AUTOTUNE_CACHE names one).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "knor_internal.cuh"
#include "knor.h"

namespace knor {

constexpr int BT = 256;            // threads of the scan CTA
constexpr int B_KMAX = 256;        // largest k of an instance
constexpr int B_PART_CAP = 2048;   // k x d up to which a unit sums in shared memory

struct BInst {
    int64_t n;      // points
    int64_t xoff;   // first coordinate in X
    int64_t poff;   // first point in the per-point arrays
    int64_t coff;   // first element of the k x d centroid arrays
    int64_t hoff;   // first entry of the k x k half-distance table
    int32_t d, k;
    int32_t koff;   // first entry of the per-centroid arrays
    int32_t pad;
    float g_up, onepk, tau, tiny; // FP32 distance bound and MTI slack for this d
};

struct BUnit {
    int32_t inst, pad;
    int64_t lo, hi; // points [lo, hi) of the instance
};

struct BCounters {
    unsigned long long changed, skipped, evals, empty;
    unsigned long long bytes;  // algorithmic bytes of the scan: 8 per point, + 4d + 8 per scanned point
    unsigned long long passed; // points Clause 1 cannot skip (counted in dense scans too)
    unsigned long long overflow; // points that found their cluster's segment full (never expected)
};

struct BParams {
    const BInst *inst;
    int32_t m;
    int32_t nunits;
    const BUnit *units;
    unsigned *qctr;
    const float *X;
    PtState *st;
    float *C32, *C32n;
    double *C64, *S, *D;
    long long *cnt, *Dcnt;
    float *halfD, *s, *F;     // halfD: per centroid a, 1/2 d(c_a, c) over c != a sorted ascending
    int32_t *order;           // ... and the centroid c of each entry (row a of k entries, +inf padded)
    int32_t *active;          // per instance: still iterating
    int32_t *dense;           // per instance: the next iteration scans every point
    int32_t *iters;           // per instance: iterations since reset
    long long *changed_last;  // per instance: changed count of its last iteration
    BCounters *bctr;          // per instance, this iteration
    const int32_t *cinst;     // per global centroid: its instance
    unsigned long long *work; // since reset: [0] point-iterations, [1] scan bytes
    IterStats *stats;
    int32_t *run_iter, *total_iter;
    const int32_t *max_iters_dev;
    unsigned long long cond_handle;
    int32_t mti, dry;
    int32_t kd_max, k_max;    // shared-memory layout of the scan
    int32_t total_k;
    // sort-segmented MTI scan: per centroid g the segment seg[sbase[g] ..
    // sbase[g] + cnt[g]) of the points assigned to it, of which acnt[g]
    // failed Clause 1 this iteration; bdesc: (g, first entry) per batch of
    // 32, grouped by the instance's width
    int32_t *seg;
    int64_t *sbase;
    unsigned *acnt;
    int2 *bdesc;
    unsigned *ctr2;           // [0] units of k_bclause1, [1 + q] batches of width class q,
                              // [5 + q] batches of class q handed out by k_bmti
    int64_t boff[4];          // first descriptor of width class q (d = 8, 16, 32, 64)
};

__host__ __device__ __forceinline__ int width_class(int d) { return d <= 8 ? 0 : (d <= 16 ? 1 : (d <= 32 ? 2 : 3)); }

// An instance whose iteration runs the sort-segmented MTI scan (its points
// all have a cluster; pruning is on and has been paying).
__device__ __forceinline__ bool seg_iter(const BParams &p, int i) {
    return p.mti && !p.dry && p.active[i] && !p.dense[i] && p.iters[i] > 0;
}

// ------------------------------------------------------------------- scan

// The new state of one scanned point and its delta sums.
template <int DV>
__device__ __forceinline__ void commit_point(const BInst &I, PtState *st, int64_t i, int a, int best, float bd,
                                             const unsigned long long (&x)[DV / 2], const float *F_s,
                                             double *part, long long *pcnt, double *D, long long *Dc,
                                             long long &changed) {
    PtState ns;
    ns.a = best;
    ns.ub = __fsub_ru(bound_up(bd, I.g_up, I.tiny), F_s[best]);
    st[i] = ns;
    if (best == a) return;
    ++changed;
    double *dst_new = part ? part + (size_t)best * DV : D + (size_t)best * DV;
    double *dst_old = a >= 0 ? (part ? part + (size_t)a * DV : D + (size_t)a * DV) : nullptr;
#pragma unroll
    for (int j = 0; j < DV / 2; ++j) {
        float x0, x1;
        unpack2(x[j], x0, x1);
        atomicAdd(dst_new + 2 * j, (double)x0);
        atomicAdd(dst_new + 2 * j + 1, (double)x1);
        if (dst_old) {
            atomicAdd(dst_old + 2 * j, -(double)x0);
            atomicAdd(dst_old + 2 * j + 1, -(double)x1);
        }
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(pcnt ? pcnt + best : Dc + best), 1ULL);
    if (a >= 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(pcnt ? pcnt + a : Dc + a), (unsigned long long)-1LL);
}

// Full scan of one point (iteration 1 and plain Lloyd): strict <, in index
// order, so the lowest index wins ties; NC consecutive centroids per step
// (independent chains, the same values as one at a time).
template <int DV>
__device__ __forceinline__ void full_scan(const unsigned long long (&x)[DV / 2], const float *cent, int k,
                                          int &best, float &bd) {
    constexpr int NC = DV <= 32 ? 4 : 2;
    bd = CUDART_INF_F;
    best = 0;
    int c = 0;
    for (; c + NC <= k; c += NC) {
        float r[NC];
        d2_regN<DV, NC>(x, cent + (size_t)c * DV, r);
#pragma unroll
        for (int q = 0; q < NC; ++q)
            if (r[q] < bd) { bd = r[q]; best = c + q; }
    }
    for (; c < k; ++c) {
        const float r = d2_reg<DV>(x, cent + (size_t)c * DV);
        if (r < bd) { bd = r; best = c; }
    }
}

// Full scan of a unit's points (iteration 1, plain Lloyd, and MTI
// instances in dense mode), one point per thread.
template <int DV>
__device__ __forceinline__ void scan_unit(const BParams &p, const BInst &I, int64_t lo, int64_t hi,
                                          const float *cent, const float *s_s, const float *F_s, double *part,
                                          long long *pcnt, long long &changed, long long &evals, long long &passed) {
    const int k = I.k;
    const float *X = p.X + I.xoff;
    PtState *st = p.st + I.poff;
    double *D = p.D + I.coff;
    long long *Dc = p.Dcnt + I.koff;
    for (int64_t i = lo + threadIdx.x; i < hi; i += BT) {
        const PtState ps = st[i];
        const int a = ps.a;
        // Clause 1 is evaluated (not used): how many points an MTI scan
        // would have to scan decides the instance's next mode
        if (p.mti) {
            bool pass = true;
            if (a >= 0) pass = !(__fmaf_ru(__fadd_ru(ps.ub, F_s[a]), I.onepk, I.tau) < s_s[a]);
            passed += pass ? 1 : 0;
        }
        unsigned long long x[DV / 2];
        ldg_x2<DV>(x, X + i * DV);
        int best;
        float bd;
        full_scan<DV>(x, cent, k, best, bd);
        evals += k;
        if (!p.dry) commit_point<DV>(I, st, i, a, best, bd, x, F_s, part, pcnt, D, Dc, changed);
    }
}

__device__ __forceinline__ long long block_sum(long long v, long long *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    long long t = 0;
    for (int w = 0; w < BT / 32; ++w) t += red[w];
    return t;
}

// Persistent: every CTA takes units from the LPT-ordered list until it is
// drained and full-scans the units of the instances that are not in a
// sort-segmented MTI iteration.  Per unit: stage the instance's centroids, s
// and F in shared memory, scan the unit's points (thread per point), merge
// the unit's delta sums into the instance's (FP64 atomics), add the unit's
// counters.
__global__ void __launch_bounds__(BT) k_bscan(const BParams p) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_unit;
    __shared__ long long red[BT / 32];
    float *cent = reinterpret_cast<float *>(sm);
    float *s_s = cent + p.kd_max;
    float *F_s = s_s + p.k_max;
    double *part = reinterpret_cast<double *>(F_s + p.k_max + ((p.kd_max + 2 * p.k_max) & 1));
    long long *pcnt = reinterpret_cast<long long *>(part + min(p.kd_max, B_PART_CAP));
    const int tid = threadIdx.x;
    while (true) {
        if (tid == 0) s_unit = (int)atomicAdd(p.qctr, 1u);
        __syncthreads();
        const int u = s_unit;
        __syncthreads();
        if (u >= p.nunits) break;
        const BUnit U = p.units[u];
        if (!p.active[U.inst] || seg_iter(p, U.inst)) continue;
        const BInst I = p.inst[U.inst];
        const int kd = I.k * I.d;
        const bool use_part = !p.dry && kd <= B_PART_CAP;
        for (int e = tid; e < kd; e += BT) cent[e] = p.C32[I.coff + e];
        for (int c = tid; c < I.k; c += BT) {
            s_s[c] = p.s[I.koff + c];
            F_s[c] = p.F[I.koff + c];
        }
        if (use_part) {
            for (int e = tid; e < kd; e += BT) part[e] = 0.0;
            for (int c = tid; c < I.k; c += BT) pcnt[c] = 0;
        }
        __syncthreads();
        long long ch = 0, ev = 0, pa = 0;
        double *pp = use_part ? part : nullptr;
        long long *pc = use_part ? pcnt : nullptr;
        switch (I.d) {
        case 8: scan_unit<8>(p, I, U.lo, U.hi, cent, s_s, F_s, pp, pc, ch, ev, pa); break;
        case 16: scan_unit<16>(p, I, U.lo, U.hi, cent, s_s, F_s, pp, pc, ch, ev, pa); break;
        case 32: scan_unit<32>(p, I, U.lo, U.hi, cent, s_s, F_s, pp, pc, ch, ev, pa); break;
        default: scan_unit<64>(p, I, U.lo, U.hi, cent, s_s, F_s, pp, pc, ch, ev, pa); break;
        }
        __syncthreads();
        if (use_part) {
            double *D = p.D + I.coff;
            long long *Dc = p.Dcnt + I.koff;
            for (int e = tid; e < kd; e += BT)
                if (part[e] != 0.0) atomicAdd(D + e, part[e]);
            for (int c = tid; c < I.k; c += BT)
                if (pcnt[c] != 0) atomicAdd(reinterpret_cast<unsigned long long *>(Dc + c), (unsigned long long)pcnt[c]);
        }
        ch = block_sum(ch, red);
        ev = block_sum(ev, red);
        pa = block_sum(pa, red);
        if (tid == 0 && !p.dry) {
            BCounters *b = p.bctr + U.inst;
            const long long np = U.hi - U.lo;
            if (ch) atomicAdd(&b->changed, (unsigned long long)ch);
            if (ev) atomicAdd(&b->evals, (unsigned long long)ev);
            if (pa) atomicAdd(&b->passed, (unsigned long long)pa);
            atomicAdd(&b->bytes, (unsigned long long)(np * (4LL * I.d + 16)));
        }
        __syncthreads();
    }
}

// ------------------------------------------------- sort-segmented MTI scan
//
// An MTI iteration of an instance runs in three launches over the whole
// batch.  k_bclause1 applies Clause 1 to every point and appends the points
// it cannot skip to the segment of their cluster; k_bbatches cuts every
// segment into batches of 32; k_bmti scans one batch per warp.  All points
// of a batch share their cluster a, so the warp walks the row 1/2 d(c_a, .)
// (sorted ascending) once -- the union of its lanes' Clause 2 survivor sets
// is the prefix below the largest bound -- and every centroid and table
// load is a broadcast.  Per point the arithmetic is that of the unit scan.

// Segment bases (exclusive prefix of the cluster counts within each
// instance) and zero active counts.  One CTA of BT >= k threads per instance.
__global__ void __launch_bounds__(BT) k_bseg(const BParams p) {
    __shared__ long long wsum[BT / 32];
    const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const BInst I = p.inst[i];
    const bool on = seg_iter(p, i);
    const long long v = (on && tid < I.k) ? p.cnt[I.koff + tid] : 0;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    long long base = 0;
    for (int ww = 0; ww < w; ++ww) base += wsum[ww];
    if (tid < I.k) {
        p.sbase[I.koff + tid] = I.poff + base + incl - v;
        p.acnt[I.koff + tid] = 0;
    }
}

// Clause 1 over the units of the segment instances.  Appends are
// aggregated per CTA: a round of BT x B_C1PA points counts its survivors per
// cluster in shared memory (each survivor gets its rank there), reserves one
// range per cluster present with a single global atomic, then writes.
constexpr int B_C1PA = 4;
__global__ void __launch_bounds__(BT) k_bclause1(const BParams p) {
    __shared__ int s_unit;
    __shared__ long long red[BT / 32];
    __shared__ unsigned hcnt[B_KMAX], hbase[B_KMAX];
    const int tid = threadIdx.x;
    for (int c = tid; c < B_KMAX; c += BT) hcnt[c] = 0;
    while (true) {
        if (tid == 0) s_unit = (int)atomicAdd(p.ctr2, 1u);
        __syncthreads();
        const int u = s_unit;
        __syncthreads();
        if (u >= p.nunits) break;
        const BUnit U = p.units[u];
        if (!seg_iter(p, U.inst)) continue;
        const BInst I = p.inst[U.inst];
        const PtState *st = p.st + I.poff;
        const float *s_g = p.s + I.koff, *F_g = p.F + I.koff;
        long long sk = 0, ov = 0;
        for (int64_t base = U.lo; base < U.hi; base += (int64_t)BT * B_C1PA) {
            int a[B_C1PA];
            unsigned rank[B_C1PA];
#pragma unroll
            for (int v = 0; v < B_C1PA; ++v) {
                const int64_t i = base + (int64_t)v * BT + tid;
                a[v] = -1;
                if (i < U.hi) {
                    const PtState ps = st[i];
                    // every point has a cluster here; a point without one
                    // (impossible) is reported, not scanned
                    if (ps.a < 0 || ps.a >= I.k) {
                        ++ov;
                    } else {
                        const float uu = __fadd_ru(ps.ub, __ldg(F_g + ps.a)); // u^t = ub + F^t(a)
                        if (!(__fmaf_ru(uu, I.onepk, I.tau) < __ldg(s_g + ps.a))) {
                            a[v] = ps.a;
                            rank[v] = atomicAdd(&hcnt[ps.a], 1u);
                        } else {
                            ++sk;
                        }
                    }
                }
            }
            __syncthreads();
            for (int c = tid; c < I.k; c += BT) {
                const unsigned h = hcnt[c];
                if (h) {
                    hbase[c] = atomicAdd(p.acnt + I.koff + c, h);
                    hcnt[c] = 0; // for the next round, past the barrier below
                }
            }
            __syncthreads();
#pragma unroll
            for (int v = 0; v < B_C1PA; ++v) {
                if (a[v] < 0) continue;
                const int g = I.koff + a[v];
                const unsigned pos = hbase[a[v]] + rank[v];
                // the segment of cluster a has room for the cnt[g] points
                // assigned to it (and stays inside the instance's range)
                const int64_t slot = p.sbase[g] + pos;
                if ((long long)pos < p.cnt[g] && slot < I.poff + I.n)
                    p.seg[slot] = (int32_t)(base + (int64_t)v * BT + tid);
                else
                    ++ov;
            }
        }
        sk = block_sum(sk, red);
        ov = block_sum(ov, red);
        if (tid == 0) {
            BCounters *b = p.bctr + U.inst;
            const long long np = U.hi - U.lo;
            if (sk) atomicAdd(&b->skipped, (unsigned long long)sk);
            if (ov) atomicAdd(&b->overflow, (unsigned long long)ov);
            atomicAdd(&b->passed, (unsigned long long)(np - sk));
            atomicAdd(&b->bytes, (unsigned long long)(8 * np + (np - sk) * (4LL * I.d + 8)));
        }
        __syncthreads();
    }
}

// Batches of 32 per non-empty segment: (g, first entry), in the region of
// the instance's width class.  One CTA of BT >= k threads per instance: its
// batches are contiguous and in cluster order, so that the warps of a CTA of
// k_bmti, which take consecutive batches, share the instance's centroids and
// table rows in L1.
__global__ void __launch_bounds__(BT) k_bbatches(const BParams p) {
    __shared__ int wsum[BT / 32];
    __shared__ unsigned s_base;
    const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (!seg_iter(p, i)) return;
    const BInst I = p.inst[i];
    const int g = I.koff + tid;
    int nb = 0;
    if (tid < I.k) {
        const long long na = min((long long)p.acnt[g], min(p.cnt[g], (long long)(I.poff + I.n - p.sbase[g])));
        nb = (int)((na + 31) / 32);
    }
    int incl = nb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int ww = 0; ww < BT / 32; ++ww) {
        before += ww < w ? wsum[ww] : 0;
        total += wsum[ww];
    }
    const int q = width_class(I.d);
    if (tid == 0) s_base = total ? atomicAdd(p.ctr2 + 1 + q, (unsigned)total) : 0u;
    __syncthreads();
    int2 *out = p.bdesc + p.boff[q] + s_base + before + incl - nb;
    for (int j = 0; j < nb; ++j) out[j] = make_int2(g, 32 * j);
}

// One batch: up to 32 points of the segment of centroid g (instance I,
// cluster a = g - I.koff), entries [first, first + 32).
template <int DV>
__device__ __forceinline__ void seg_batch(const BParams &p, const BInst &I, int inst, int g, int first,
                                          const float *cent) {
    const int lane = threadIdx.x & 31;
    const int k = I.k, a = g - I.koff;
    const long long na = min((long long)p.acnt[g], min(p.cnt[g], (long long)(I.poff + I.n - p.sbase[g])));
    const int nb = (int)min((long long)32, na - first);
    PtState *st = p.st + I.poff;
    int64_t i = 0;
    unsigned long long x[DV / 2];
    float bd = CUDART_INF_F, tst = 0.0f;
    int best = a;
    unsigned ev = 0;
    if (lane < nb) {
        i = p.seg[p.sbase[g] + first + lane];
        ldg_x2_stream<DV>(x, p.X + I.xoff + i * DV);
        // Clause 3: tighten u to (a bound on) the exact d(v, c_a)
        bd = d2_reg<DV>(x, cent + (size_t)a * DV);
        ev = 1;
        tst = __fmaf_ru(bound_up(bd, I.g_up, I.tiny), I.onepk, I.tau);
    } else {
#pragma unroll
        for (int j = 0; j < DV / 2; ++j) x[j] = 0ULL;
    }
    // Clause 2 along the sorted row: each lane's survivors are the prefix
    // of entries not above its bound; the warp stops after the longest
    // (the argmin with lowest-index ties does not depend on the order).
    // Four entries per step, scored side by side; a lane adopts an entry
    // only if it is one of its own survivors.
    const float tmax = __uint_as_float(__reduce_max_sync(FULL_MASK, __float_as_uint(tst) & 0x7fffffffu));
    const float *hs = p.halfD + I.hoff + (size_t)a * k;
    const int32_t *od = p.order + I.hoff + (size_t)a * k;
    float h[4];
    int c[4];
    auto fetch = [&](int j, float (&hh)[4], int (&cc)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool in = j + q < k - 1;
            hh[q] = in ? __ldg(hs + j + q) : CUDART_INF_F;
            cc[q] = in ? __ldg(od + j + q) : a;
        }
    };
    fetch(0, h, c);
    for (int j = 0; j < k - 1; j += 4) {
        if (tmax < h[0]) break;
        float hn[4];
        int cn[4];
        fetch(j + 4, hn, cn); // the next step's entries, in flight during this one
        float r[4];
        d2_reg4<DV>(x, cent + (size_t)c[0] * DV, cent + (size_t)c[1] * DV, cent + (size_t)c[2] * DV,
                    cent + (size_t)c[3] * DV, r);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (lane < nb && !(tst < h[q])) {
                ++ev;
                if (r[q] < bd || (r[q] == bd && c[q] < best)) { bd = r[q]; best = c[q]; }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) { h[q] = hn[q]; c[q] = cn[q]; }
    }
    long long ch = 0;
    if (lane < nb)
        commit_point<DV>(I, st, i, a, best, bd, x, p.F + I.koff, nullptr, nullptr, p.D + I.coff,
                         p.Dcnt + I.koff, ch);
    unsigned chu = (unsigned)ch;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_xor_sync(FULL_MASK, ev, o);
        chu += __shfl_xor_sync(FULL_MASK, chu, o);
    }
    if (lane == 0) {
        BCounters *b = p.bctr + inst;
        atomicAdd(&b->evals, (unsigned long long)ev);
        if (chu) atomicAdd(&b->changed, (unsigned long long)chu);
    }
}

// Persistent, one launch per width class.  A CTA takes B_CHUNK consecutive
// batches at a time (one atomic), its warps every (BTM / 32)-th of them, so
// the batches of one instance and neighbouring clusters run on one SM; the
// centroids of the chunk's first instance are staged in shared memory (a
// batch of another instance in the same chunk reads them from global).
constexpr int B_CHUNK = 64;
constexpr int BTM = 128; // threads of a k_bmti CTA
template <int DV>
__global__ void __launch_bounds__(BTM, DV >= 64 ? 3 : (DV >= 32 ? 4 : 5)) k_bmti(const BParams p) {
    constexpr int q = DV <= 8 ? 0 : (DV <= 16 ? 1 : (DV <= 32 ? 2 : 3));
    extern __shared__ __align__(16) float cs[];
    __shared__ unsigned s_chunk;
    const unsigned nb = p.ctr2[1 + q];
    const int2 *desc = p.bdesc + p.boff[q];
    const int w = threadIdx.x >> 5;
    int staged = -1;
    while (true) {
        if (threadIdx.x == 0) s_chunk = atomicAdd(p.ctr2 + 5 + q, (unsigned)B_CHUNK);
        __syncthreads();
        const unsigned c0 = s_chunk;
        if (c0 >= nb) break;
        const unsigned c1 = min(nb, c0 + B_CHUNK);
        const int i0 = p.cinst[desc[c0].x];
        if (i0 != staged) {
            const BInst I0 = p.inst[i0];
            const float4 *src = reinterpret_cast<const float4 *>(p.C32 + I0.coff);
            float4 *dst = reinterpret_cast<float4 *>(cs);
            for (int e = threadIdx.x; e < I0.k * DV / 4; e += BTM) dst[e] = src[e];
            staged = i0;
        }
        __syncthreads();
        for (unsigned b = c0 + w; b < c1; b += BTM / 32) {
            const int2 dsc = desc[b];
            const int inst = p.cinst[dsc.x];
            const BInst I = p.inst[inst];
            // two call sites, so that the staged path reads shared memory directly
            if (inst == staged) seg_batch<DV>(p, I, inst, dsc.x, dsc.y, cs);
            else seg_batch<DV>(p, I, inst, dsc.x, dsc.y, p.C32 + I.coff);
        }
        __syncthreads(); // the staged centroids stay until every warp is done
    }
}

// ------------------------------------------------ merge, bookkeeping, table

// K5 per centroid of every active instance: S += the iteration's deltas,
// c = S / count in FP64 (an empty cluster keeps its centroid, its sum reset
// to exactly 0), the FP32 scan copy of the result.
__global__ void k_breduce(const BParams p) {
    const int g = blockIdx.x;
    const int i = p.cinst[g];
    if (!p.active[i]) return;
    const BInst I = p.inst[i];
    const int c = g - I.koff;
    const int j = threadIdx.x;
    const long long cn = p.cnt[g] + p.Dcnt[g];
    if (j < I.d) {
        const int64_t e = I.coff + (int64_t)c * I.d + j;
        double Sn = p.S[e] + p.D[e];
        double cv = p.C64[e];
        if (cn > 0) cv = Sn / (double)cn;
        else Sn = 0.0;
        p.S[e] = Sn;
        p.C64[e] = cv;
        p.C32n[e] = __double2float_rn(cv);
        p.D[e] = 0.0;
    }
    __syncthreads();
    if (j == 0) {
        p.cnt[g] = cn;
        p.Dcnt[g] = 0;
        if (cn == 0) atomicAdd(&p.bctr[i].empty, 1ULL);
    }
}

// After the merge: per instance, count the iteration, mask it once no point
// changed; the run's record (sums over the instances active in it) and the
// device-side loop condition.  One CTA.
__global__ void k_bstep(const BParams p, int32_t snapshot) {
    __shared__ unsigned long long red[5][32];
    __shared__ int any_s;
    unsigned long long ch = 0, sk = 0, ev = 0, em = 0, pts = 0, by = 0, ov = 0;
    int any = 0;
    if (threadIdx.x == 0) any_s = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < p.m; i += blockDim.x) {
        const BCounters b = p.bctr[i];
        if (p.active[i]) {
            p.iters[i] += 1;
            p.changed_last[i] = (long long)b.changed;
            ch += b.changed;
            sk += b.skipped;
            ev += b.evals;
            em += b.empty;
            ov += b.overflow;
            pts += (unsigned long long)p.inst[i].n;
            by += b.bytes;
            if (b.changed == 0) p.active[i] = 0;
            // next mode: after an MTI iteration in which Clause 1 let most
            // points through and Clause 2 pruned little (at least 70 % of
            // their k distances evaluated), scan every point once -- an MTI
            // scan then costs more than the plain one; after a dense
            // iteration, MTI again (its counters tell whether pruning pays)
            const unsigned long long nk = (unsigned long long)p.inst[i].k;
            p.dense[i] = (p.mti && !p.dense[i] && 2 * b.passed > (unsigned long long)p.inst[i].n &&
                          10 * b.evals >= 7 * b.passed * nk)
                             ? 1
                             : 0;
        }
        any |= p.active[i];
        p.bctr[i] = BCounters{0, 0, 0, 0, 0, 0, 0};
    }
    if (any) atomicOr(&any_s, 1);
    if (snapshot) {
        if (pts) atomicAdd(&p.work[0], pts);
        if (by) atomicAdd(&p.work[1], by);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ch += __shfl_xor_sync(FULL_MASK, ch, o);
        sk += __shfl_xor_sync(FULL_MASK, sk, o);
        ev += __shfl_xor_sync(FULL_MASK, ev, o);
        em += __shfl_xor_sync(FULL_MASK, em, o);
        ov += __shfl_xor_sync(FULL_MASK, ov, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][w] = ch; red[1][w] = sk; red[2][w] = ev; red[3][w] = em; red[4][w] = ov; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    ch = sk = ev = em = ov = 0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
        ch += red[0][ww]; sk += red[1][ww]; ev += red[2][ww]; em += red[3][ww]; ov += red[4][ww];
    }
    if (!snapshot) return;
    const int it = *p.run_iter;
    const int total = *p.total_iter + 1;
    IterStats r;
    r.changed = (long long)ch;
    r.clause1_skipped = (long long)sk;
    r.dist_evals = (long long)ev;
    r.rechecked = 0;
    r.empty = (int32_t)em;
    r.iteration = total;
    r.violations = (long long)ov; // points that found their segment full (never expected)
    p.stats[it] = r;
    *p.run_iter = it + 1;
    *p.total_iter = total;
    if (p.cond_handle) {
        const unsigned go = (any_s && it + 1 < *p.max_iters_dev) ? 1u : 0u;
        cudaGraphSetConditional((cudaGraphConditionalHandle)p.cond_handle, go);
    }
}

// K1 per centroid a of every active instance, from the FP32 scan copies,
// in FP32 with directed rounding on the library's FP32 distance d~^2 (for
// which d~^2 <= d^2 g + tiny and d^2 <= d~^2 g + tiny, g = 1/(1 - (d+2)
// 2^-24)): the drift f(a) <= sqrt(d~^2 g + tiny) rounded up and added
// (rounded up) to F(a); 1/2 d(c_a, c) >= 1/2 sqrt((d~^2 - tiny) / g)
// rounded down; s(a) their minimum over c != a; then the new scan copy
// replaces the old one.  (The single-problem table computes the same bounds
// in FP64; these are a little looser but need no FP64 units, which matters
// with up to 256 x 256 pairs per instance.)
__global__ void k_btable(const BParams p, int32_t need_table) {
    const int g = blockIdx.x;
    const int i = p.cinst[g];
    if (!p.active[i]) return;
    const BInst I = p.inst[i];
    const int a = g - I.koff, k = I.k, d = I.d, tid = threadIdx.x;
    const float *Cn = p.C32n + I.coff;
    float *Co = p.C32 + I.coff;
    __shared__ float hv[B_KMAX];
    __shared__ int cv[B_KMAX];
    if (need_table) {
        if (tid == 0) {
            const float d2 = d2_gen(Cn + (size_t)a * d, Co + (size_t)a * d, d);
            p.F[g] = __fadd_ru(p.F[g], bound_up(d2, I.g_up, I.tiny));
        }
        // 1/2 d(c_a, c) for c != a, then the row sorted ascending (bitonic
        // over the first P entries, P the power of two >= k - 1; the rest
        // is +inf padding) with its centroid indices; s(a) is the first entry
        int P = 1;
        while (P < k - 1) P <<= 1;
        for (int j = tid; j < max(P, k); j += blockDim.x) { // every entry written out below
            float h = CUDART_INF_F;
            int c = a;
            if (j < k - 1) {
                c = j < a ? j : j + 1;
                const float d2 = d2_gen(Cn + (size_t)a * d, Cn + (size_t)c * d, d);
                const float lo2 = fmaxf(__fdiv_rd(__fsub_rd(d2, I.tiny), I.g_up), 0.0f);
                h = __fmul_rd(0.5f, __fsqrt_rd(lo2));
            }
            hv[j] = h;
            cv[j] = c;
        }
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                __syncthreads();
                for (int t = tid; t < P / 2; t += blockDim.x) {
                    const int lo = 2 * t - (t & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const float x = hv[lo], y = hv[hi];
                    if ((x > y) == up) {
                        hv[lo] = y;
                        hv[hi] = x;
                        const int ci = cv[lo];
                        cv[lo] = cv[hi];
                        cv[hi] = ci;
                    }
                }
            }
        }
        __syncthreads();
        float *hrow = p.halfD + I.hoff + (size_t)a * k;
        int32_t *orow = p.order + I.hoff + (size_t)a * k;
        for (int j = tid; j < k; j += blockDim.x) {
            hrow[j] = hv[j];
            orow[j] = cv[j];
        }
        if (tid == 0) p.s[g] = hv[0];
        __syncthreads();
    }
    for (int j = tid; j < d; j += blockDim.x) Co[(size_t)a * d + j] = Cn[(size_t)a * d + j];
}

__global__ void k_binit_state(PtState *st, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        st[i] = PtState{CUDART_INF_F, -1};
}

__global__ void k_bround(const double *C64, float *C32, float *C32n, int64_t total) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const float v = __double2float_rn(C64[e]);
        C32[e] = v;
        C32n[e] = v;
    }
}

__global__ void k_bgather(const float *X, int32_t d, const int64_t *idx, int32_t k, double *C0) {
    const int64_t total = (int64_t)k * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        C0[e] = (double)X[idx[e / d] * d + e % d];
}

__global__ void k_bextract(const PtState *st, int64_t n, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = st[i].a;
}

static int gridfor(int64_t count, int threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((count + threads - 1) / threads, 4096));
}

} // namespace knor

using namespace knor;

// ------------------------------------------------------------------ host

enum BFlag { BF_RUN_ITER = 0, BF_TOTAL_ITER, BF_MAX_ITERS, BF_COUNT };

struct knor_batch {
    int dev = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int32_t m = 0;
    knor_opts opts{};
    uint64_t seed = 0;
    std::vector<BInst> h_inst;
    std::vector<std::vector<int64_t>> init_idx;
    std::vector<int32_t> unit_pts;  // tuned unit size per instance
    int64_t total_n = 0, total_x = 0, total_c = 0, total_h = 0;
    int32_t total_k = 0, kd_max = 0, k_max = 0;
    float *X = nullptr, *C32 = nullptr, *C32n = nullptr, *halfD = nullptr, *s = nullptr, *F = nullptr;
    int32_t *order = nullptr;
    PtState *st = nullptr;
    double *C0 = nullptr, *C64 = nullptr, *S = nullptr, *D = nullptr;
    long long *cnt = nullptr, *Dcnt = nullptr, *changed_last = nullptr;
    BInst *inst = nullptr;
    BUnit *units = nullptr;
    int32_t nunits = 0;
    unsigned *qctr = nullptr, *ctr2 = nullptr, *acnt = nullptr;
    int32_t *seg = nullptr;
    int64_t *sbase = nullptr;
    int2 *bdesc = nullptr;
    int grid_c1 = 0, grid_mti[4] = {};
    size_t smem_mti[4] = {};
    int64_t boff[4] = {};
    int32_t *active = nullptr, *iters = nullptr, *cinst = nullptr, *flags = nullptr, *dense = nullptr;
    BCounters *bctr = nullptr;
    unsigned long long *work = nullptr;
    IterStats *stats = nullptr;
    int64_t *d_idx = nullptr;
    size_t smem = 0;
    int grid = 0, bps = 1;
    cudaGraphExec_t iter_exec = nullptr, run_exec = nullptr;
    bool profiling = false;
    cudaEvent_t ev[6] = {};
    int64_t prof_n[KNOR_KERNEL_COUNT] = {};
    double prof_ms[KNOR_KERNEL_COUNT] = {};
    std::string tuning;
};

namespace {

constexpr int kBStatsCap = 65536;

knor_status bfail(knor_batch *b, knor_status st, const std::string &msg) {
    b->err = msg;
    return st;
}

#define BCUDA(b, call)                                                                                \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            cudaGetLastError();                                                                       \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? KNOR_ERR_OOM : KNOR_ERR_CUDA,           \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                         \
        }                                                                                             \
    } while (0)

template <class T>
knor_status balloc(knor_batch *b, T **p, size_t count) {
    BCUDA(b, cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T)));
    return KNOR_OK;
}

void bfree_all(knor_batch *b) {
    void *bufs[] = {b->X,    b->C32,   b->C32n, b->halfD, b->s,      b->F,     b->st,     b->C0,
                    b->C64,  b->S,     b->D,    b->cnt,   b->Dcnt,   b->changed_last, b->inst, b->units,
                    b->qctr, b->active, b->iters, b->cinst, b->flags, b->bctr,  b->stats,  b->d_idx, b->work, b->dense, b->order,
                    b->ctr2, b->acnt, b->seg, b->sbase, b->bdesc};
    for (void *p : bufs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->iter_exec) cudaGraphExecDestroy(b->iter_exec);
    if (b->run_exec) cudaGraphExecDestroy(b->run_exec);
    if (b->stream) cudaStreamDestroy(b->stream);
}

BParams params_of(const knor_batch *b, int dry, unsigned long long cond, const BUnit *units, int32_t nunits) {
    BParams p{};
    p.inst = b->inst;
    p.m = b->m;
    p.nunits = nunits;
    p.units = units;
    p.qctr = b->qctr;
    p.X = b->X;
    p.st = b->st;
    p.C32 = b->C32;
    p.C32n = b->C32n;
    p.C64 = b->C64;
    p.S = b->S;
    p.D = b->D;
    p.cnt = b->cnt;
    p.Dcnt = b->Dcnt;
    p.halfD = b->halfD;
    p.order = b->order;
    p.s = b->s;
    p.F = b->F;
    p.active = b->active;
    p.dense = b->dense;
    p.iters = b->iters;
    p.changed_last = b->changed_last;
    p.bctr = b->bctr;
    p.cinst = b->cinst;
    p.work = b->work;
    p.stats = b->stats;
    p.run_iter = b->flags + BF_RUN_ITER;
    p.total_iter = b->flags + BF_TOTAL_ITER;
    p.max_iters_dev = b->flags + BF_MAX_ITERS;
    p.cond_handle = cond;
    p.mti = b->opts.no_prune ? 0 : 1;
    p.dry = dry;
    p.kd_max = b->kd_max;
    p.k_max = b->k_max;
    p.total_k = b->total_k;
    p.seg = b->seg;
    p.sbase = b->sbase;
    p.acnt = b->acnt;
    p.bdesc = b->bdesc;
    p.ctr2 = b->ctr2;
    for (int q = 0; q < 4; ++q) p.boff[q] = b->boff[q];
    return p;
}

// Work units: each instance cut into pieces of its bucket's unit size, all
// pieces ordered by cost (points x k x d) descending, ties by instance and
// position (a fixed order).
std::vector<BUnit> make_units(const knor_batch *b, const std::vector<int32_t> &unit_pts,
                              const std::vector<int> *only = nullptr) {
    std::vector<BUnit> u;
    std::vector<double> cost;
    for (int32_t i = 0; i < b->m; ++i) {
        if (only && std::find(only->begin(), only->end(), i) == only->end()) continue;
        const BInst &I = b->h_inst[i];
        const int64_t step = std::max<int64_t>(1, unit_pts[i]);
        for (int64_t lo = 0; lo < I.n; lo += step) {
            BUnit x{};
            x.inst = i;
            x.lo = lo;
            x.hi = std::min<int64_t>(I.n, lo + step);
            u.push_back(x);
        }
    }
    std::vector<size_t> ord(u.size());
    std::iota(ord.begin(), ord.end(), 0);
    auto cost_of = [&](const BUnit &x) {
        const BInst &I = b->h_inst[x.inst];
        return (double)(x.hi - x.lo) * I.k * I.d;
    };
    std::stable_sort(ord.begin(), ord.end(), [&](size_t p, size_t q) { return cost_of(u[p]) > cost_of(u[q]); });
    std::vector<BUnit> out;
    out.reserve(u.size());
    for (size_t q : ord) out.push_back(u[q]);
    return out;
}

knor_status enqueue_iter(knor_batch *b, cudaStream_t s, unsigned long long cond, cudaEvent_t *ev) {
    const BParams p = params_of(b, 0, cond, b->units, b->nunits);
    auto mark = [&](int i) -> cudaError_t { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
    BCUDA(b, cudaMemsetAsync(b->qctr, 0, sizeof(unsigned), s));
    BCUDA(b, cudaMemsetAsync(b->ctr2, 0, 9 * sizeof(unsigned), s));
    BCUDA(b, mark(0));
    k_bscan<<<b->grid, BT, b->smem, s>>>(p);
    BCUDA(b, cudaGetLastError());
    if (p.mti) {
        k_bseg<<<b->m, BT, 0, s>>>(p);
        BCUDA(b, cudaGetLastError());
        k_bclause1<<<b->grid_c1, BT, 0, s>>>(p);
        BCUDA(b, cudaGetLastError());
        k_bbatches<<<b->m, BT, 0, s>>>(p);
        BCUDA(b, cudaGetLastError());
        if (b->grid_mti[0]) k_bmti<8><<<b->grid_mti[0], BTM, b->smem_mti[0], s>>>(p);
        if (b->grid_mti[1]) k_bmti<16><<<b->grid_mti[1], BTM, b->smem_mti[1], s>>>(p);
        if (b->grid_mti[2]) k_bmti<32><<<b->grid_mti[2], BTM, b->smem_mti[2], s>>>(p);
        if (b->grid_mti[3]) k_bmti<64><<<b->grid_mti[3], BTM, b->smem_mti[3], s>>>(p);
        BCUDA(b, cudaGetLastError());
    }
    BCUDA(b, mark(1));
    k_breduce<<<b->total_k, 64, 0, s>>>(p);
    BCUDA(b, cudaGetLastError());
    BCUDA(b, mark(2));
    k_bstep<<<1, 512, 0, s>>>(p, 1);
    BCUDA(b, cudaGetLastError());
    k_btable<<<b->total_k, 128, 0, s>>>(p, b->opts.no_prune ? 0 : 1);
    BCUDA(b, cudaGetLastError());
    BCUDA(b, mark(3));
    return KNOR_OK;
}

knor_status build_graphs(knor_batch *b) {
    {
        BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        knor_status st = enqueue_iter(b, b->stream, 0, nullptr);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (st != KNOR_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        BCUDA(b, e);
        e = cudaGraphInstantiate(&b->iter_exec, g, 0);
        cudaGraphDestroy(g);
        BCUDA(b, e);
    }
    {
        cudaGraph_t g = nullptr;
        BCUDA(b, cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) { cudaGraphDestroy(g); BCUDA(b, e); }
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        if (e != cudaSuccess) { cudaGraphDestroy(g); BCUDA(b, e); }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(b->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { cudaGraphDestroy(g); BCUDA(b, e); }
        knor_status st = enqueue_iter(b, b->stream, (unsigned long long)h, nullptr);
        cudaGraph_t got = nullptr;
        e = cudaStreamEndCapture(b->stream, &got);
        if (st != KNOR_OK) { cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) { cudaGraphDestroy(g); BCUDA(b, e); }
        e = cudaGraphInstantiate(&b->run_exec, g, 0);
        cudaGraphDestroy(g);
        BCUDA(b, e);
    }
    return KNOR_OK;
}

// Back to C^0 (b->C0): centroids, sums, counts, drift, bounds, tables.
knor_status breset(knor_batch *b) {
    cudaStream_t s = b->stream;
    const size_t tc = (size_t)b->total_c, tk = (size_t)b->total_k;
    BCUDA(b, cudaMemcpyAsync(b->C64, b->C0, tc * sizeof(double), cudaMemcpyDeviceToDevice, s));
    k_bround<<<gridfor((int64_t)tc, 256), 256, 0, s>>>(b->C0, b->C32, b->C32n, (int64_t)tc);
    BCUDA(b, cudaGetLastError());
    BCUDA(b, cudaMemsetAsync(b->S, 0, tc * sizeof(double), s));
    BCUDA(b, cudaMemsetAsync(b->D, 0, tc * sizeof(double), s));
    BCUDA(b, cudaMemsetAsync(b->cnt, 0, tk * sizeof(long long), s));
    BCUDA(b, cudaMemsetAsync(b->Dcnt, 0, tk * sizeof(long long), s));
    BCUDA(b, cudaMemsetAsync(b->F, 0, tk * sizeof(float), s));
    BCUDA(b, cudaMemsetAsync(b->bctr, 0, (size_t)b->m * sizeof(BCounters), s));
    BCUDA(b, cudaMemsetAsync(b->work, 0, 2 * sizeof(unsigned long long), s));
    BCUDA(b, cudaMemsetAsync(b->iters, 0, (size_t)b->m * sizeof(int32_t), s));
    BCUDA(b, cudaMemsetAsync(b->dense, 0, (size_t)b->m * sizeof(int32_t), s));
    BCUDA(b, cudaMemsetAsync(b->changed_last, 0, (size_t)b->m * sizeof(long long), s));
    std::vector<int32_t> ones((size_t)b->m, 1);
    BCUDA(b, cudaMemcpyAsync(b->active, ones.data(), ones.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_binit_state<<<gridfor(b->total_n, 256), 256, 0, s>>>(b->st, b->total_n);
    BCUDA(b, cudaGetLastError());
    int32_t fl[BF_COUNT] = {0, 0, 1};
    BCUDA(b, cudaMemcpyAsync(b->flags, fl, sizeof(fl), cudaMemcpyHostToDevice, s));
    // tables for C^0 (drift 0, no record)
    const BParams p = params_of(b, 0, 0, b->units, b->nunits);
    k_btable<<<b->total_k, 128, 0, s>>>(p, b->opts.no_prune ? 0 : 1);
    BCUDA(b, cudaGetLastError());
    BCUDA(b, cudaStreamSynchronize(s));
    return KNOR_OK;
}

// ---------------------------------------------------------------- autotune

std::mutex g_tune_mu;
std::map<std::string, int32_t> g_tune; // key -> unit size
bool g_tune_loaded = false;

std::string tune_key(const cudaDeviceProp &pr, int d, int kb, bool mti) {
    char buf[320];
    std::snprintf(buf, sizeof(buf), "%s|sm%d|%d.%d|d%d|kb%d|%s", pr.name, pr.multiProcessorCount, pr.major,
                  pr.minor, d, kb, mti ? "mti" : "plain");
    return buf;
}

void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("KNOR_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        char *sep = std::strrchr(line, '=');
        if (!sep) continue;
        *sep = 0;
        g_tune[line] = std::atoi(sep + 1);
    }
    std::fclose(f);
}

void tune_store(const std::string &key, int32_t v) {
    g_tune[key] = v;
    const char *path = std::getenv("KNOR_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s=%d\n", key.c_str(), v);
    std::fclose(f);
}

int k_bucket(int k) { return k <= 32 ? 0 : (k <= 96 ? 1 : 2); }

// Times one dry scan (nothing written) over the given units.
knor_status time_dry(knor_batch *b, const std::vector<BUnit> &u, int grid, float *ms) {
    BUnit *du = nullptr;
    BCUDA(b, cudaMalloc(&du, std::max<size_t>(u.size(), 1) * sizeof(BUnit)));
    cudaError_t e = cudaMemcpyAsync(du, u.data(), u.size() * sizeof(BUnit), cudaMemcpyHostToDevice, b->stream);
    const BParams p = params_of(b, 1, 0, du, (int32_t)u.size());
    float best = 1e30f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaMemsetAsync(b->qctr, 0, sizeof(unsigned), b->stream);
        if (e != cudaSuccess) break;
        e = cudaEventRecord(b->ev[0], b->stream);
        if (e != cudaSuccess) break;
        k_bscan<<<grid, BT, b->smem, b->stream>>>(p);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        e = cudaEventRecord(b->ev[1], b->stream);
        if (e != cudaSuccess) break;
        e = cudaEventSynchronize(b->ev[1]);
        if (e != cudaSuccess) break;
        float t = 0.0f;
        e = cudaEventElapsedTime(&t, b->ev[0], b->ev[1]);
        best = std::min(best, t);
    }
    cudaFree(du);
    BCUDA(b, e);
    *ms = best;
    return KNOR_OK;
}

// Grid search: per (d, k) bucket the unit size in {1024, 4096, 16384,
// 65536} points, timed on a sample of that bucket's instances (at most
// 8M points) in their iteration-1 state; then the persistent CTAs per SM.
knor_status autotune(knor_batch *b) {
    cudaDeviceProp pr{};
    BCUDA(b, cudaGetDeviceProperties(&pr, b->dev));
    int maxbps = 1;
    BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxbps, k_bscan, BT, b->smem));
    maxbps = std::max(1, maxbps);
    const bool enabled = !(std::getenv("KNOR_AUTOTUNE") && std::string(std::getenv("KNOR_AUTOTUNE")) == "0");
    const int32_t cands[4] = {1024, 4096, 16384, 65536};
    const bool mti = !b->opts.no_prune;
    std::map<std::pair<int, int>, std::vector<int>> buckets;
    for (int32_t i = 0; i < b->m; ++i)
        buckets[{b->h_inst[i].d, k_bucket(b->h_inst[i].k)}].push_back(i);
    b->unit_pts.assign((size_t)b->m, 8192);
    std::string desc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
    }
    b->grid = b->num_sms * maxbps;
    for (auto &kv : buckets) {
        const std::string key = tune_key(pr, kv.first.first, kv.first.second, mti);
        int32_t chosen = 8192;
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) { chosen = it->second; cached = true; }
        }
        if (!cached && enabled) {
            // sample: the bucket's instances, largest first, up to 8M points
            std::vector<int> sample = kv.second;
            std::sort(sample.begin(), sample.end(), [&](int p, int q) { return b->h_inst[p].n > b->h_inst[q].n; });
            std::vector<int> take;
            int64_t pts = 0;
            for (int i : sample) {
                if (pts >= (8 << 20)) break;
                take.push_back(i);
                pts += b->h_inst[i].n;
            }
            float best = 1e30f;
            for (int32_t c : cands) {
                std::vector<int32_t> up((size_t)b->m, c);
                const std::vector<BUnit> u = make_units(b, up, &take);
                float ms = 0.0f;
                knor_status st = time_dry(b, u, b->grid, &ms);
                if (st != KNOR_OK) return st;
                if (ms < best) { best = ms; chosen = c; }
            }
            std::lock_guard<std::mutex> lk(g_tune_mu);
            tune_store(key, chosen);
        }
        for (int i : kv.second) b->unit_pts[(size_t)i] = chosen;
        char buf[96];
        std::snprintf(buf, sizeof(buf), "%sd%d/kb%d:%d", desc.empty() ? "" : " ", kv.first.first, kv.first.second,
                      chosen);
        desc += buf;
    }
    // persistent CTAs per SM, on the whole unit list
    const std::vector<BUnit> all = make_units(b, b->unit_pts);
    int best_bps = maxbps;
    if (enabled && maxbps > 1) {
        float best = 1e30f;
        for (int q = 1; q <= maxbps; ++q) {
            float ms = 0.0f;
            knor_status st = time_dry(b, all, b->num_sms * q, &ms);
            if (st != KNOR_OK) return st;
            if (ms < best) { best = ms; best_bps = q; }
        }
    }
    b->bps = best_bps;
    b->grid = b->num_sms * best_bps;
    char buf[128];
    std::snprintf(buf, sizeof(buf), "; %d CTAs/SM x %d SMs; %zu units", best_bps, b->num_sms, all.size());
    b->tuning = "unit points per (d, k bucket): " + desc + buf + (enabled ? "" : " (autotune off)");
    return KNOR_OK;
}

knor_status read_bstats(knor_batch *b, int32_t count, knor_iter_stats *out) {
    if (!out || count <= 0) return KNOR_OK;
    std::vector<IterStats> h((size_t)count);
    BCUDA(b, cudaMemcpy(h.data(), b->stats, sizeof(IterStats) * count, cudaMemcpyDeviceToHost));
    for (int32_t t = 0; t < count; ++t) {
        knor_iter_stats &o = out[t];
        o.changed = h[t].changed;
        o.clause1_skipped = h[t].clause1_skipped;
        o.dist_evals = h[t].dist_evals;
        o.rechecked = h[t].rechecked;
        o.empty = h[t].empty;
        o.iteration = h[t].iteration;
        o.violations = h[t].violations;
    }
    return KNOR_OK;
}

knor_status profiled_iter(knor_batch *b) {
    knor_status st = enqueue_iter(b, b->stream, 0, b->ev);
    if (st != KNOR_OK) return st;
    BCUDA(b, cudaStreamSynchronize(b->stream));
    float t = 0.0f;
    BCUDA(b, cudaEventElapsedTime(&t, b->ev[0], b->ev[1]));
    b->prof_n[KNOR_KERNEL_MTI] += 1;
    b->prof_ms[KNOR_KERNEL_MTI] += t;
    BCUDA(b, cudaEventElapsedTime(&t, b->ev[1], b->ev[2]));
    b->prof_n[KNOR_KERNEL_REDUCE] += 1;
    b->prof_ms[KNOR_KERNEL_REDUCE] += t;
    BCUDA(b, cudaEventElapsedTime(&t, b->ev[2], b->ev[3]));
    b->prof_n[KNOR_KERNEL_TABLE] += 1;
    b->prof_ms[KNOR_KERNEL_TABLE] += t;
    return KNOR_OK;
}

knor_status check_instance(const knor_batch *b, int32_t i) {
    if (i < 0 || i >= b->m) return KNOR_ERR_ARG;
    return KNOR_OK;
}

} // namespace

extern "C" {

knor_status knor_batch_create(int32_t m, const float *const *points, const int64_t *n, const int32_t *d,
                              const int32_t *k, uint64_t seed, const knor_opts *opts, knor_batch **out) {
    if (!out) return KNOR_ERR_ARG;
    *out = nullptr;
    set_global_error("");
    if (m < 1 || !points || !n || !d || !k) {
        set_global_error("knor_batch_create: need m >= 1 and non-NULL points, n, d, k");
        return KNOR_ERR_ARG;
    }
    knor_opts o{};
    if (opts) o = *opts;
    if (o.precision != KNOR_PREC_FP32 || o.full_recompute_every != 0 || o.elkan != 0) {
        set_global_error("knor_batch_create: the batched form supports FP32 distances, delta sums and MTI only");
        return KNOR_ERR_ARG;
    }
    for (int32_t i = 0; i < m; ++i) {
        if (!points[i] || n[i] < 1 || k[i] < 1 || k[i] > n[i] || k[i] > B_KMAX ||
            (d[i] != 8 && d[i] != 16 && d[i] != 32 && d[i] != 64)) {
            set_global_error(("knor_batch_create: instance " + std::to_string(i) +
                              ": need 1 <= k <= min(n, 256), d in {8, 16, 32, 64} and non-NULL points").c_str());
            return KNOR_ERR_ARG;
        }
    }
    knor_batch *b = new knor_batch();
    b->m = m;
    b->opts = o;
    b->seed = seed;
    auto bail = [&](knor_status st) {
        set_global_error(b->err.c_str());
        bfree_all(b);
        delete b;
        return st;
    };
#define BC(call) do { knor_status s_ = (call); if (s_ != KNOR_OK) return bail(s_); } while (0)
#define BCU(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { b->err = std::string(#call) + ": " + cudaGetErrorString(e_); cudaGetLastError(); return bail(e_ == cudaErrorMemoryAllocation ? KNOR_ERR_OOM : KNOR_ERR_CUDA); } } while (0)
    BCU(cudaGetDevice(&b->dev));
    BCU(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->dev));
    BCU(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    for (auto &e : b->ev) BCU(cudaEventCreate(&e));
    // layout
    b->h_inst.resize((size_t)m);
    std::vector<int32_t> cinst;
    const double u = std::ldexp(1.0, -24);
    for (int32_t i = 0; i < m; ++i) {
        BInst &I = b->h_inst[(size_t)i];
        I.n = n[i];
        I.d = d[i];
        I.k = k[i];
        I.xoff = b->total_x;
        I.poff = b->total_n;
        I.coff = b->total_c;
        I.hoff = b->total_h;
        I.koff = b->total_k;
        const double g = (I.d + 2) * u / (1.0 - (I.d + 2) * u);
        I.g_up = f32_up(1.0 / (1.0 - (I.d + 2) * u));
        I.onepk = f32_up(1.0 + g);
        I.tau = std::ldexp(1.0f, -40);
        I.tiny = (float)std::ldexp((double)I.d, -149);
        b->total_x += I.n * I.d;
        b->total_n += I.n;
        b->total_c += (int64_t)I.k * I.d;
        b->total_h += (int64_t)I.k * I.k;
        b->total_k += I.k;
        b->kd_max = std::max(b->kd_max, I.k * I.d);
        b->k_max = std::max(b->k_max, I.k);
        for (int c = 0; c < I.k; ++c) cinst.push_back(i);
    }
    const size_t tc = (size_t)b->total_c, tk = (size_t)b->total_k;
    BC(balloc(b, &b->X, (size_t)b->total_x));
    BC(balloc(b, &b->st, (size_t)b->total_n));
    BC(balloc(b, &b->C0, tc));
    BC(balloc(b, &b->C64, tc));
    BC(balloc(b, &b->S, tc));
    BC(balloc(b, &b->D, tc));
    BC(balloc(b, &b->C32, tc));
    BC(balloc(b, &b->C32n, tc));
    BC(balloc(b, &b->halfD, (size_t)b->total_h));
    BC(balloc(b, &b->order, (size_t)b->total_h));
    BC(balloc(b, &b->s, tk));
    BC(balloc(b, &b->F, tk));
    BC(balloc(b, &b->cnt, tk));
    BC(balloc(b, &b->Dcnt, tk));
    BC(balloc(b, &b->cinst, tk));
    BC(balloc(b, &b->inst, (size_t)m));
    BC(balloc(b, &b->active, (size_t)m));
    BC(balloc(b, &b->dense, (size_t)m));
    BC(balloc(b, &b->iters, (size_t)m));
    BC(balloc(b, &b->changed_last, (size_t)m));
    BC(balloc(b, &b->bctr, (size_t)m));
    BC(balloc(b, &b->work, 2));
    BC(balloc(b, &b->qctr, 1));
    BC(balloc(b, &b->ctr2, 9));
    BC(balloc(b, &b->acnt, tk));
    BC(balloc(b, &b->sbase, tk));
    if (!b->opts.no_prune) {
        // descriptor regions per width class: an instance's segments need
        // at most n / 32 + k batches
        int64_t cap[4] = {0, 0, 0, 0};
        for (const BInst &I : b->h_inst) cap[width_class(I.d)] += I.n / 32 + I.k + 1;
        int64_t off = 0;
        for (int q = 0; q < 4; ++q) { b->boff[q] = off; off += cap[q]; }
        BC(balloc(b, &b->seg, (size_t)b->total_n));
        BC(balloc(b, &b->bdesc, (size_t)off));
    }
    BC(balloc(b, &b->flags, BF_COUNT));
    BC(balloc(b, &b->stats, kBStatsCap));
    BC(balloc(b, &b->d_idx, (size_t)b->k_max));
    BCU(cudaMemcpyAsync(b->inst, b->h_inst.data(), sizeof(BInst) * (size_t)m, cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->cinst, cinst.data(), sizeof(int32_t) * tk, cudaMemcpyHostToDevice, b->stream));
    // points (host or device), validated
    unsigned long long *bad = nullptr;
    BC(balloc(b, &bad, 1));
    BCU(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), b->stream));
    for (int32_t i = 0; i < m; ++i) {
        const BInst &I = b->h_inst[(size_t)i];
        const size_t bytes = sizeof(float) * (size_t)I.n * I.d;
        BCU(cudaMemcpyAsync(b->X + I.xoff, points[i], bytes, cudaMemcpyDefault, b->stream));
    }
    BCU(launch_validate(b->X, b->total_x, bad, b->stream));
    unsigned long long nbad = 0;
    BCU(cudaMemcpyAsync(&nbad, bad, sizeof(nbad), cudaMemcpyDeviceToHost, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    cudaFree(bad);
    if (nbad) {
        b->err = "knor_batch_create: " + std::to_string(nbad) + " coordinates are NaN, infinite or above 1e15";
        return bail(KNOR_ERR_ARG);
    }
    // C^0: Forgy per instance, seed + instance
    b->init_idx.resize((size_t)m);
    for (int32_t i = 0; i < m; ++i) {
        const BInst &I = b->h_inst[(size_t)i];
        b->init_idx[(size_t)i] = forgy_indices(I.n, I.k, seed + (uint64_t)i);
        BCU(cudaMemcpyAsync(b->d_idx, b->init_idx[(size_t)i].data(), sizeof(int64_t) * I.k, cudaMemcpyHostToDevice,
                            b->stream));
        k_bgather<<<gridfor((int64_t)I.k * I.d, 256), 256, 0, b->stream>>>(b->X + I.xoff, I.d, b->d_idx, I.k,
                                                                             b->C0 + I.coff);
        BCU(cudaGetLastError());
        BCU(cudaStreamSynchronize(b->stream)); // d_idx is reused
    }
    // scan launch shape
    b->smem = sizeof(float) * ((size_t)b->kd_max + 2 * b->k_max + 1) +
              sizeof(double) * (size_t)std::min(b->kd_max, B_PART_CAP) + sizeof(long long) * b->k_max + 16;
    BCU(cudaFuncSetAttribute(k_bscan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    {
        int q1 = 1, qm[4] = {1, 1, 1, 1};
        BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q1, k_bclause1, BT, 0));
        // k_bmti stages k x d centroids of the largest k of its width class
        int kmax_w[4] = {0, 0, 0, 0};
        for (const BInst &I : b->h_inst) kmax_w[width_class(I.d)] = std::max(kmax_w[width_class(I.d)], I.k);
        const int widths[4] = {8, 16, 32, 64};
        for (int q = 0; q < 4; ++q) b->smem_mti[q] = sizeof(float) * (size_t)std::max(1, kmax_w[q]) * widths[q];
        BCU(cudaFuncSetAttribute(k_bmti<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_mti[0]));
        BCU(cudaFuncSetAttribute(k_bmti<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_mti[1]));
        BCU(cudaFuncSetAttribute(k_bmti<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_mti[2]));
        BCU(cudaFuncSetAttribute(k_bmti<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_mti[3]));
        BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&qm[0], k_bmti<8>, BTM, b->smem_mti[0]));
        BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&qm[1], k_bmti<16>, BTM, b->smem_mti[1]));
        BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&qm[2], k_bmti<32>, BTM, b->smem_mti[2]));
        BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&qm[3], k_bmti<64>, BTM, b->smem_mti[3]));
        b->grid_c1 = b->num_sms * std::max(1, q1);
        // a width class without instances gets no launch
        bool has[4] = {false, false, false, false};
        for (const BInst &I : b->h_inst) has[width_class(I.d)] = true;
        for (int q = 0; q < 4; ++q) b->grid_mti[q] = has[q] ? b->num_sms * std::max(1, qm[q]) : 0;
    }
    BC(breset(b));
    BC(autotune(b));
    const std::vector<BUnit> units = make_units(b, b->unit_pts);
    b->nunits = (int32_t)units.size();
    BC(balloc(b, &b->units, units.size()));
    BCU(cudaMemcpyAsync(b->units, units.data(), sizeof(BUnit) * units.size(), cudaMemcpyHostToDevice, b->stream));
    BC(breset(b));
    BC(build_graphs(b));
    *out = b;
    return KNOR_OK;
#undef BC
#undef BCU
}

void knor_batch_destroy(knor_batch *b) {
    if (!b) return;
    cudaSetDevice(b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    bfree_all(b);
    delete b;
}

const char *knor_batch_last_error(const knor_batch *b) { return b ? b->err.c_str() : ""; }
void *knor_batch_stream(const knor_batch *b) { return b ? (void *)b->stream : nullptr; }
const char *knor_batch_describe(const knor_batch *b) { return b ? b->tuning.c_str() : ""; }

knor_status knor_batch_reset(knor_batch *b) {
    if (!b) return KNOR_ERR_ARG;
    b->err.clear();
    return breset(b);
}

knor_status knor_batch_set_init_centroids(knor_batch *b, int32_t instance, const double *c_kxd) {
    if (!b) return KNOR_ERR_ARG;
    b->err.clear();
    if (check_instance(b, instance) != KNOR_OK || !c_kxd)
        return bfail(b, KNOR_ERR_ARG, "knor_batch_set_init_centroids: bad instance or NULL centroids");
    const BInst &I = b->h_inst[(size_t)instance];
    const size_t kd = (size_t)I.k * I.d;
    std::vector<double> h(kd);
    BCUDA(b, cudaMemcpy(h.data(), c_kxd, kd * sizeof(double), cudaMemcpyDefault));
    for (double v : h)
        if (!std::isfinite(v) || std::fabs(v) > 1e15)
            return bfail(b, KNOR_ERR_ARG, "knor_batch_set_init_centroids: coordinate not finite or above 1e15");
    BCUDA(b, cudaMemcpy(b->C0 + I.coff, h.data(), kd * sizeof(double), cudaMemcpyHostToDevice));
    return breset(b);
}

knor_status knor_batch_iterate(knor_batch *b, knor_iter_stats *out) {
    if (!b) return KNOR_ERR_ARG;
    b->err.clear();
    BCUDA(b, cudaMemsetAsync(b->flags + BF_RUN_ITER, 0, sizeof(int32_t), b->stream));
    if (b->profiling) {
        knor_status st = profiled_iter(b);
        if (st != KNOR_OK) return st;
    } else {
        BCUDA(b, cudaGraphLaunch(b->iter_exec, b->stream));
        BCUDA(b, cudaStreamSynchronize(b->stream));
    }
    return read_bstats(b, 1, out);
}

knor_status knor_batch_run(knor_batch *b, int32_t max_iters, int32_t *iters_done, knor_iter_stats *per_iter) {
    if (!b) return KNOR_ERR_ARG;
    b->err.clear();
    if (iters_done) *iters_done = 0;
    if (max_iters < 0 || max_iters > kBStatsCap) return bfail(b, KNOR_ERR_ARG, "knor_batch_run: max_iters out of range");
    if (max_iters == 0) return KNOR_OK;
    BCUDA(b, cudaMemsetAsync(b->flags + BF_RUN_ITER, 0, sizeof(int32_t), b->stream));
    int32_t done = 0;
    if (b->profiling) {
        for (int t = 0; t < max_iters; ++t) {
            knor_status st = profiled_iter(b);
            if (st != KNOR_OK) return st;
            done = t + 1;
            int32_t any = 0;
            std::vector<int32_t> act((size_t)b->m);
            BCUDA(b, cudaMemcpy(act.data(), b->active, sizeof(int32_t) * act.size(), cudaMemcpyDeviceToHost));
            for (int32_t v : act) any |= v;
            if (!any) break;
        }
    } else {
        BCUDA(b, cudaMemcpyAsync(b->flags + BF_MAX_ITERS, &max_iters, sizeof(int32_t), cudaMemcpyHostToDevice,
                                 b->stream));
        BCUDA(b, cudaGraphLaunch(b->run_exec, b->stream));
        BCUDA(b, cudaMemcpyAsync(&done, b->flags + BF_RUN_ITER, sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream));
        BCUDA(b, cudaStreamSynchronize(b->stream));
    }
    if (iters_done) *iters_done = done;
    return read_bstats(b, done, per_iter);
}

knor_status knor_batch_get_assignments(const knor_batch *bc, int32_t instance, int32_t *out_n) {
    knor_batch *b = const_cast<knor_batch *>(bc);
    if (!b) return KNOR_ERR_ARG;
    b->err.clear();
    if (check_instance(b, instance) != KNOR_OK || !out_n)
        return bfail(b, KNOR_ERR_ARG, "knor_batch_get_assignments: bad instance or NULL output");
    const BInst &I = b->h_inst[(size_t)instance];
    int32_t *tmp = nullptr;
    BCUDA(b, cudaMallocAsync(&tmp, sizeof(int32_t) * (size_t)I.n, b->stream));
    k_bextract<<<gridfor(I.n, 256), 256, 0, b->stream>>>(b->st + I.poff, I.n, tmp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_n, tmp, sizeof(int32_t) * (size_t)I.n, cudaMemcpyDefault, b->stream);
    cudaFreeAsync(tmp, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    BCUDA(b, e);
    return KNOR_OK;
}

knor_status knor_batch_get_centroids(const knor_batch *bc, int32_t instance, double *out_kxd) {
    knor_batch *b = const_cast<knor_batch *>(bc);
    if (!b) return KNOR_ERR_ARG;
    b->err.clear();
    if (check_instance(b, instance) != KNOR_OK || !out_kxd)
        return bfail(b, KNOR_ERR_ARG, "knor_batch_get_centroids: bad instance or NULL output");
    const BInst &I = b->h_inst[(size_t)instance];
    BCUDA(b, cudaMemcpyAsync(out_kxd, b->C64 + I.coff, sizeof(double) * (size_t)I.k * I.d, cudaMemcpyDefault,
                             b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    return KNOR_OK;
}

knor_status knor_batch_get_centroids_f32(const knor_batch *bc, int32_t instance, float *out_kxd) {
    knor_batch *b = const_cast<knor_batch *>(bc);
    if (!b) return KNOR_ERR_ARG;
    b->err.clear();
    if (check_instance(b, instance) != KNOR_OK || !out_kxd)
        return bfail(b, KNOR_ERR_ARG, "knor_batch_get_centroids_f32: bad instance or NULL output");
    const BInst &I = b->h_inst[(size_t)instance];
    BCUDA(b, cudaMemcpyAsync(out_kxd, b->C32 + I.coff, sizeof(float) * (size_t)I.k * I.d, cudaMemcpyDefault,
                             b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    return KNOR_OK;
}

knor_status knor_batch_get_init_indices(const knor_batch *b, int32_t instance, int64_t *out_k) {
    if (!b || check_instance(b, instance) != KNOR_OK || !out_k) return KNOR_ERR_ARG;
    const std::vector<int64_t> &v = b->init_idx[(size_t)instance];
    std::memcpy(out_k, v.data(), sizeof(int64_t) * v.size());
    return KNOR_OK;
}

knor_status knor_batch_get_instance(const knor_batch *bc, int32_t instance, knor_batch_instance *out) {
    knor_batch *b = const_cast<knor_batch *>(bc);
    if (!b) return KNOR_ERR_ARG;
    b->err.clear();
    if (check_instance(b, instance) != KNOR_OK || !out)
        return bfail(b, KNOR_ERR_ARG, "knor_batch_get_instance: bad instance or NULL output");
    int32_t it = 0, act = 0;
    long long ch = 0;
    BCUDA(b, cudaMemcpy(&it, b->iters + instance, sizeof(it), cudaMemcpyDeviceToHost));
    BCUDA(b, cudaMemcpy(&act, b->active + instance, sizeof(act), cudaMemcpyDeviceToHost));
    BCUDA(b, cudaMemcpy(&ch, b->changed_last + instance, sizeof(ch), cudaMemcpyDeviceToHost));
    const BInst &I = b->h_inst[(size_t)instance];
    out->n = I.n;
    out->d = I.d;
    out->k = I.k;
    out->iterations = it;
    out->converged = (it > 0 && ch == 0) ? 1 : 0;
    out->changed_last = ch;
    return KNOR_OK;
}

knor_status knor_batch_get_work(const knor_batch *bc, int64_t *point_iterations, int64_t *scan_bytes) {
    knor_batch *b = const_cast<knor_batch *>(bc);
    if (!b) return KNOR_ERR_ARG;
    b->err.clear();
    unsigned long long w[2] = {0, 0};
    BCUDA(b, cudaMemcpyAsync(w, b->work, sizeof(w), cudaMemcpyDeviceToHost, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    if (point_iterations) *point_iterations = (int64_t)w[0];
    if (scan_bytes) *scan_bytes = (int64_t)w[1];
    return KNOR_OK;
}

knor_status knor_batch_set_profiling(knor_batch *b, int32_t on) {
    if (!b) return KNOR_ERR_ARG;
    b->profiling = on != 0;
    return KNOR_OK;
}

knor_status knor_batch_get_profile(knor_batch *b, knor_profile *out, int32_t reset_after) {
    if (!b || !out) return KNOR_ERR_ARG;
    for (int q = 0; q < KNOR_KERNEL_COUNT; ++q) {
        out->launches[q] = b->prof_n[q];
        out->ms[q] = b->prof_ms[q];
        if (reset_after) { b->prof_n[q] = 0; b->prof_ms[q] = 0.0; }
    }
    return KNOR_OK;
}

const char *knor_batch_kernel_name(const knor_batch *b, int32_t kernel) {
    if (!b) return "";
    switch (kernel) {
    case KNOR_KERNEL_MTI: return "k_bscan + k_bclause1 + k_bmti";
    case KNOR_KERNEL_REDUCE: return "k_breduce";
    case KNOR_KERNEL_TABLE: return "k_bstep + k_btable";
    default: return "";
    }
}

} // extern "C"

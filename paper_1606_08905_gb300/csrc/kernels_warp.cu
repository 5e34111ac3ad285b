// kernels_warp.cu -- warp-autonomous point kernels of libknor.so.
//
// Same arithmetic as k_dense / k_mti (kernels.cu): the FP32 direct-form
// distance d2_reg, lowest-index ties, bounds rounded toward safety, TwoSum
// cluster sums.  The difference is the schedule: every warp streams its own
// tiles (cp.async, double-buffered), keeps its own cluster-sum accumulators
// and never waits at a CTA barrier until the final merge.  Cluster sums are
// formed per group of lanes that chose the same cluster (ballot), with lanes
// walking the dimensions, so each (cluster, dim) accumulator of a warp is
// updated in a fixed order; the CTA adds its warps' accumulators in warp
// order.  The sums are therefore deterministic.
#include "device_common.cuh"
#include "knor_internal.cuh"

namespace knor {

constexpr int WT = WPC * 32; // threads per CTA

// Adds (sign = +1) or subtracts (sign = -1) the rows of the lanes with
// has = true into the warp's accumulators, cluster cl of each lane.  Rows are
// read from `rowsrc(p, j)` (member lane p, dimension j).
template <int DV, class RowFn>
__device__ __forceinline__ void warp_group_accumulate(RowFn rowsrc, int cl, bool has, float sign, float *acc_hi,
                                                      float *acc_lo, int *cnt) {
    const int lane = threadIdx.x & 31;
    unsigned rem = __ballot_sync(FULL_MASK, has);
    while (rem) {
        const int leader = __ffs(rem) - 1;
        const int c = __shfl_sync(FULL_MASK, cl, leader);
        const unsigned grp = __ballot_sync(FULL_MASK, has && cl == c);
        rem &= ~grp;
        if constexpr (DV <= 32) {
            constexpr int G = 32 / DV; // members summed side by side
            const int sub = lane / DV, j = lane % DV;
            float h = 0.0f, l = 0.0f;
            unsigned m = grp;
            int idx = 0;
            while (m) {
                const int pl = __ffs(m) - 1;
                m &= m - 1;
                if (idx % G == sub) two_sum_reg(h, l, rowsrc(pl, j) * sign);
                ++idx;
            }
#pragma unroll
            for (int o = DV; o < 32; o <<= 1) {
                const float h2 = __shfl_xor_sync(FULL_MASK, h, o);
                const float l2 = __shfl_xor_sync(FULL_MASK, l, o);
                two_sum_merge(h, l, h2, l2);
            }
            if (sub == 0) {
                float H = acc_hi[c * DV + j], L = acc_lo[c * DV + j];
                two_sum_merge(H, L, h, l);
                acc_hi[c * DV + j] = H;
                acc_lo[c * DV + j] = L;
            }
        } else {
            constexpr int R = DV / 32;
            float h[R], l[R];
#pragma unroll
            for (int r = 0; r < R; ++r) { h[r] = 0.0f; l[r] = 0.0f; }
            unsigned m = grp;
            while (m) {
                const int pl = __ffs(m) - 1;
                m &= m - 1;
#pragma unroll
                for (int r = 0; r < R; ++r) two_sum_reg(h[r], l[r], rowsrc(pl, lane + 32 * r) * sign);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = c * DV + lane + 32 * r;
                float H = acc_hi[e], L = acc_lo[e];
                two_sum_merge(H, L, h[r], l[r]);
                acc_hi[e] = H;
                acc_lo[e] = L;
            }
        }
        if (lane == 0) cnt[c] += (sign > 0.0f ? 1 : -1) * __popc(grp);
    }
}

// Warp w's accumulators: shared memory, or its slot of p.wacc.
__device__ __forceinline__ float *warp_acc_hi(const IterParams &p, unsigned char *sm, int w) {
    if (p.wacc) return p.wacc + ((size_t)blockIdx.x * WPC + w) * 2 * (size_t)p.k * p.d;
    return reinterpret_cast<float *>(sm + p.w_base + w * p.w_stride + p.w_acc_hi);
}
__device__ __forceinline__ float *warp_acc_lo(const IterParams &p, unsigned char *sm, int w) {
    if (p.wacc) return p.wacc + ((size_t)blockIdx.x * WPC + w) * 2 * (size_t)p.k * p.d + (size_t)p.k * p.d;
    return reinterpret_cast<float *>(sm + p.w_base + w * p.w_stride + p.w_acc_lo);
}

// The CTA's partial slot: its warps' accumulators added in warp order.
__device__ __forceinline__ void flush_warp_partials(const IterParams &p, unsigned char *sm) {
    const int kd = p.k * p.d;
    for (int e = threadIdx.x; e < kd; e += WT) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < WPC; ++w) {
            s += (double)warp_acc_hi(p, sm, w)[e];
            s += (double)warp_acc_lo(p, sm, w)[e];
        }
        p.part_S[(size_t)e * p.part_stride + blockIdx.x] = s;
    }
    for (int c = threadIdx.x; c < p.k; c += WT) {
        long long s = 0;
#pragma unroll
        for (int w = 0; w < WPC; ++w)
            s += reinterpret_cast<const int *>(sm + p.w_base + w * p.w_stride + p.w_cnt)[c];
        p.part_cnt[(size_t)c * p.part_stride + blockIdx.x] = s;
    }
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Stages the CTA-shared tables into shared memory.  The warp kernels are
// only chosen when the centroids, the k x k table and s, F fit, so these
// pointers always address shared memory (plain shared loads, no generic
// address resolution in the inner loops).
struct Shared {
    const float *cent, *halfD, *s, *F;
};
__device__ __forceinline__ Shared stage_shared(const IterParams &p, unsigned char *sm, bool need_table) {
    const int kd = p.k * p.d;
    float *cs = reinterpret_cast<float *>(sm + p.off_cent);
    for (int e = threadIdx.x; e < kd; e += WT) cs[e] = p.C32[e];
    float *hs = reinterpret_cast<float *>(sm + p.off_halfD);
    if (need_table)
        for (int e = threadIdx.x; e < p.k * p.k; e += WT) hs[e] = p.halfD[e];
    float *a1 = reinterpret_cast<float *>(sm + p.off_s);
    float *a2 = reinterpret_cast<float *>(sm + p.off_F);
    for (int c = threadIdx.x; c < p.k; c += WT) { a1[c] = p.s[c]; a2[c] = p.F[c]; }
    return Shared{cs, hs, a1, a2};
}

// ------------------------------------------------------------ dense scan

template <int DV>
__global__ void __launch_bounds__(WT) k_dense_w(const IterParams p, const int32_t *mode_dense, int32_t *nslots,
                                                int32_t *fresh) {
    if (*mode_dense == 0) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int k = p.k;
    constexpr int CH = DV / 4;
    unsigned char *wr = sm + p.w_base + w * p.w_stride;
    float *acc_hi = reinterpret_cast<float *>(wr + p.w_acc_hi);
    float *acc_lo = reinterpret_cast<float *>(wr + p.w_acc_lo);
    int *cnt = reinterpret_cast<int *>(wr + p.w_cnt);
    float *tile = reinterpret_cast<float *>(wr + p.w_tile);
    const int dpad = p.dpad;
    if (blockIdx.x == 0 && tid == 0) { *nslots = (int)gridDim.x; *fresh = 1; }
    for (int e = lane; e < k * DV; e += 32) { acc_hi[e] = 0.0f; acc_lo[e] = 0.0f; }
    for (int c = lane; c < k; c += 32) cnt[c] = 0;
    const Shared sh = stage_shared(p, sm, false);
    __syncthreads();
    int64_t lo, hi;
    block_range(p.n, 1, lo, hi);
    const int64_t ntile = (hi - lo + 31) / 32;

    auto load_tile = [&](int stage, int64_t t) {
        const int64_t base = lo + t * 32;
        const int rows = (int)min((int64_t)32, hi - base);
        float *dst = tile + stage * 32 * dpad;
        const float *src = p.X + base * DV;
        for (int f = lane; f < rows * CH; f += 32) {
            const int r = f / CH, ch = f % CH;
            cp_async16(dst + r * dpad + ch * 4, src + (size_t)r * DV + ch * 4);
        }
        cp_async_commit();
    };

    long long my_changed = 0;
    int stage = 0;
    if (w < ntile) load_tile(0, w);
    for (int64_t t = w; t < ntile; t += WPC) {
        if (t + WPC < ntile) {
            load_tile(stage ^ 1, t + WPC);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        const float *tl = tile + stage * 32 * dpad;
        const int64_t base = lo + t * 32;
        const int rows = (int)min((int64_t)32, hi - base);
        const bool valid = lane < rows;
        int best = -1;
        if (valid) {
            unsigned long long x2[DV / 2];
            load_x2<DV>(x2, tl + lane * dpad);
            float bd = CUDART_INF_F;
            best = 0;
            int c = 0;
            constexpr int NC = DV <= 32 ? 4 : 2;
            for (; c + NC <= k; c += NC) {
                float r[NC];
                d2_regN<DV, NC>(x2, sh.cent + (size_t)c * DV, r);
#pragma unroll
                for (int q = 0; q < NC; ++q)
                    if (r[q] < bd) { bd = r[q]; best = c + q; }
            }
            for (; c < k; ++c) {
                const float r = d2_reg<DV>(x2, sh.cent + (size_t)c * DV);
                if (r < bd) { bd = r; best = c; }
            }
            const int64_t i = base + lane;
            const PtState old = p.st[i];
            my_changed += (old.a != best);
            PtState ns;
            ns.a = best;
            ns.ub = p.mti ? __fsub_ru(bound_up(bd, p.g_up, p.tiny), sh.F[best]) : 0.0f;
            p.st[i] = ns;
        }
        warp_group_accumulate<DV>([&](int pl, int j) { return tl[pl * dpad + j]; }, best, valid, 1.0f,
                                  acc_hi, acc_lo, cnt);
        __syncwarp();
        stage ^= 1;
    }
    const long long ch = warp_sum_ll(my_changed);
    if (lane == 0) {
        atomicAdd(&p.ctr->changed, (unsigned long long)ch);
    }
    __syncthreads();
    flush_warp_partials(p, sm);
    if (tid == 0) atomicAdd(&p.ctr->evals, (unsigned long long)((hi - lo) * (int64_t)k));
}

// --------------------------------------------------------------- MTI scan

// Per warp: the packed state of its chunks streams into shared memory with
// cp.async (WSTAGES chunks in flight); the points that Clause 1 cannot skip
// go, in point order, to the bucket of their cluster; every bucket that
// reaches 32 points is scanned one point per lane (Clause 3 tightening,
// Clause 2 per centroid), and the warp's partial buckets after its last
// chunk.  The rows that changed cluster move between the warp's sums (read
// back from global memory, where the scan has just loaded them).  Bucket
// order depends only on the point order, so the sums stay deterministic.
// d <= 32: 5 resident CTAs x 4 warps per SM (registers capped at 96, no
// spills); wider points keep their registers
template <int DV>
__global__ void __launch_bounds__(WT, DV <= 32 ? 5 : 1) k_mti_w(const IterParams p, const int32_t *mode_dense,
                                                                int32_t *nslots, int32_t *fresh) {
    if (*mode_dense != 0) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int k = p.k;
    unsigned char *wr = sm + p.w_base + w * p.w_stride;
    float *acc_hi = warp_acc_hi(p, sm, w);
    float *acc_lo = warp_acc_lo(p, sm, w);
    int *cnt = reinterpret_cast<int *>(wr + p.w_cnt);
    // per-cluster buckets: bucket c (c < k: points assigned to cluster c;
    // c = k: unassigned points) is a ring of WBCAP local indices
    int *bk = reinterpret_cast<int *>(wr + p.w_bucket);
    int *bhead = bk + (k + 1) * WBCAP;
    int *bcnt = bhead + (k + 1);
    PtState *stbuf = reinterpret_cast<PtState *>(wr + p.w_state);
    if (blockIdx.x == 0 && tid == 0) { *nslots = (int)gridDim.x; *fresh = 0; }
    for (int e = lane; e < k * DV; e += 32) { acc_hi[e] = 0.0f; acc_lo[e] = 0.0f; }
    for (int c = lane; c < k; c += 32) cnt[c] = 0;
    for (int c = lane; c <= k; c += 32) { bhead[c] = 0; bcnt[c] = 0; }
    const Shared sh = stage_shared(p, sm, true);
    __syncthreads();
    int64_t lo, hi;
    block_range(p.n, WPA, lo, hi);
    const int64_t nchunk = (hi - lo + WCH - 1) / WCH;

    auto prefetch = [&](int stage, int64_t m) {
        if (m < nchunk) {
            const int64_t i0 = lo + m * WCH + (int64_t)lane * WPA;
            if (i0 + WPA <= hi) {
                const char *src = reinterpret_cast<const char *>(p.st + i0);
                char *dst = reinterpret_cast<char *>(stbuf + stage * WCH + lane * WPA);
#pragma unroll
                for (int v = 0; v < WPA * 8 / 16; ++v) cp_async16(dst + 16 * v, src + 16 * v);
            }
        }
        cp_async_commit();
    };

    // per-lane counts: a lane sees at most n / (32 x warps) points, each
    // with at most k evaluations, far below 2^32 for any resident n
    unsigned my_skipped = 0, my_evals = 0, my_changed = 0;

    // Phases B and C on the first nb (<= 32) points of bucket cb: every
    // lane of the batch shares a = cb, hence the row of the k x k table, and
    // the candidate sets of Clause 2 are nested (all centroids c with
    // 1/2 d(c_a, c) below the point's bound), so the walk over the union of
    // the lanes' masks leaves few lanes idle.
    auto run_batch = [&](int cb, int nb) {
        const int a = cb == k ? -1 : cb;
        const int *ring = bk + cb * WBCAP;
        const int h0 = bhead[cb];
        int best = -1;
        int64_t i = 0;
        bool changed = false;
        unsigned long long xk[DV / 2];
        float bd = CUDART_INF_F, tst = 0.0f;
        if (lane < nb) {
            i = lo + ring[(h0 + lane) & (WBCAP - 1)];
            // rows of >= 8 floats start on 32-byte boundaries (cudaMalloc base)
            if constexpr (DV % 8 == 0) ldg_x2_w32<DV>(xk, p.X + i * DV);
            else ldg_x2<DV>(xk, p.X + i * DV);
            if (a < 0) {
                best = 0;
                for (int c = 0; c < k; ++c) {
                    const float r = d2_reg<DV>(xk, sh.cent + (size_t)c * DV);
                    if (r < bd) { bd = r; best = c; }
                }
                my_evals += k;
            } else {
                // Clause 3: tighten u to (a bound on) the exact d(v, c_a)
                bd = d2_reg<DV>(xk, sh.cent + (size_t)a * DV);
                best = a;
                ++my_evals;
            }
            tst = __fmaf_ru(bound_up(bd, p.g_up, p.tiny), p.onepk, p.tau);
        }
        // Clause 2: every centroid c != a with u >= 1/2 d(c_a, c) survives.
        // The lanes share the row 1/2 d(c_a, .), so the union of their
        // survivors is the survivor set of the largest bound: lane b tests
        // centroid cw + b against it, and the warp walks the union in index
        // order, each lane scoring its own survivors.
        if (a >= 0) {
            const float *hrow = sh.halfD + (size_t)a * k;
            // tst >= 0 (sign bit cleared for -0): its bit pattern orders like the value
            const float tmax = __uint_as_float(__reduce_max_sync(FULL_MASK, __float_as_uint(tst) & 0x7fffffffu));
            for (int cw = 0; cw < k; cw += 32) {
                const int cl = cw + lane;
                unsigned uni = __ballot_sync(FULL_MASK, cl < k && cl != a && !(tmax < hrow[min(cl, k - 1)]));
                while (uni) {
                    const int b = __ffs(uni) - 1;
                    uni &= uni - 1;
                    const int c = cw + b;
                    if (lane < nb && !(tst < hrow[c])) {
                        const float r = d2_reg<DV>(xk, sh.cent + (size_t)c * DV);
                        ++my_evals;
                        if (r < bd || (r == bd && c < best)) { bd = r; best = c; }
                    }
                }
            }
        }
        if (lane < nb) {
            PtState ns;
            ns.a = best;
            ns.ub = __fsub_ru(bound_up(bd, p.g_up, p.tiny), sh.F[best]);
            p.st[i] = ns;
            changed = best != a;
            my_changed += changed ? 1 : 0;
        }
        // member pl's row, by its bucket entry (no shuffles: the member loop
        // of warp_group_accumulate is lane-divergent)
        const float *X = p.X;
        auto row = [&](int pl, int j) { return __ldg(X + (lo + ring[(h0 + pl) & (WBCAP - 1)]) * DV + j); };
        warp_group_accumulate<DV>(row, best, changed, 1.0f, acc_hi, acc_lo, cnt);
        warp_group_accumulate<DV>(row, a, changed && a >= 0, -1.0f, acc_hi, acc_lo, cnt);
        __syncwarp();
        if (lane == 0) {
            bhead[cb] = (h0 + nb) & (WBCAP - 1);
            bcnt[cb] -= nb;
        }
        __syncwarp();
    };

#pragma unroll
    for (int s = 0; s < WSTAGES - 1; ++s) prefetch(s, w + (int64_t)s * WPC);
    int stage = 0;
    for (int64_t m = w; m < nchunk; m += WPC) {
        prefetch((stage + WSTAGES - 1) % WSTAGES, m + (int64_t)(WSTAGES - 1) * WPC);
        cp_async_wait<WSTAGES - 1>();
        __syncwarp();
        // ---- phase A: Clause 1 on WPA consecutive points per lane
        const int64_t i0 = lo + m * WCH + (int64_t)lane * WPA;
        PtState ps[WPA];
        if (i0 + WPA <= hi) {
            const int4 *src = reinterpret_cast<const int4 *>(stbuf + stage * WCH + lane * WPA);
#pragma unroll
            for (int v = 0; v < WPA / 2; ++v) {
                const int4 q = src[v];
                ps[2 * v].ub = __int_as_float(q.x);
                ps[2 * v].a = q.y;
                ps[2 * v + 1].ub = __int_as_float(q.z);
                ps[2 * v + 1].a = q.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < WPA; ++u) {
                if (i0 + u < hi) ps[u] = p.st[i0 + u];
                else { ps[u].ub = 0.0f; ps[u].a = -2; }
            }
        }
        unsigned amask = 0;
        int nvalid = 0;
#pragma unroll
        for (int u = 0; u < WPA; ++u) {
            const int a = ps[u].a;
            if (a == -2) continue;
            ++nvalid;
            bool act = true;
            if (a >= 0) {
                const float uu = __fadd_ru(ps[u].ub, sh.F[a]); // u^t = ub + F^t(a)
                act = !(__fmaf_ru(uu, p.onepk, p.tau) < sh.s[a]);
            }
            amask |= (act ? 1u : 0u) << u;
        }
        const int na = __popc(amask);
        my_skipped += nvalid - na;
        int incl = na;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(FULL_MASK, incl, 31);
        // the points that pass Clause 1, in point order, staged in the state
        // buffer just read (its next prefetch comes after this chunk)
        int2 *stg = reinterpret_cast<int2 *>(stbuf + stage * WCH);
        __syncwarp();
        int pos = incl - na;
#pragma unroll
        for (int u = 0; u < WPA; ++u) {
            if ((amask >> u) & 1u) {
                stg[pos] = make_int2((int)(i0 + u - lo), ps[u].a);
                ++pos;
            }
        }
        __syncwarp();
        stage = (stage + 1) % WSTAGES;

        // ---- append to the buckets 32 at a time; a bucket that reaches 32
        // points runs as one batch
        for (int base = 0; base < total; base += 32) {
            const int e = base + lane;
            const bool valid = e < total;
            const int2 ent = valid ? stg[e] : make_int2(0, 0);
            const int key = valid ? (ent.y < 0 ? k : ent.y) : -1 - lane;
            const unsigned grp = __match_any_sync(FULL_MASK, key);
            const int rank = __popc(grp & ((1u << lane) - 1u));
            int now = 0;
            if (valid) {
                const int c0 = bcnt[key];
                bk[key * WBCAP + ((bhead[key] + c0 + rank) & (WBCAP - 1))] = ent.x;
                now = c0 + __popc(grp);
            }
            __syncwarp();
            if (valid && rank == 0) bcnt[key] = now;
            __syncwarp();
            unsigned full = __ballot_sync(FULL_MASK, valid && rank == 0 && now >= 32);
            while (full) {
                const int leader = __ffs(full) - 1;
                full &= full - 1;
                run_batch(__shfl_sync(FULL_MASK, key, leader), 32);
            }
        }
        __syncwarp();
    }
    // the warp's partial buckets
    for (int cb = 0; cb <= k; ++cb) {
        const int left = bcnt[cb];
        if (left > 0) run_batch(cb, left);
    }
    cp_async_wait<0>();
    const long long t1 = warp_sum_ll((long long)my_changed);
    const long long t2 = warp_sum_ll((long long)my_skipped);
    const long long t3 = warp_sum_ll((long long)my_evals);
    if (lane == 0) {
        atomicAdd(&p.ctr->changed, (unsigned long long)t1);
        atomicAdd(&p.ctr->skipped, (unsigned long long)t2);
        atomicAdd(&p.ctr->evals, (unsigned long long)t3);
    }
    __syncthreads();
    flush_warp_partials(p, sm);
}

// ------------------------------------------------------------- launchers

#define KNOR_DVW_SWITCH(dv, FN, ...)                     \
    switch (dv) {                                        \
    case 4: return FN<4>(__VA_ARGS__);                   \
    case 8: return FN<8>(__VA_ARGS__);                   \
    case 16: return FN<16>(__VA_ARGS__);                 \
    case 32: return FN<32>(__VA_ARGS__);                 \
    case 64: return FN<64>(__VA_ARGS__);                 \
    case 128: return FN<128>(__VA_ARGS__);               \
    default: return cudaErrorInvalidValue;               \
    }

template <int DV>
static cudaError_t dense_w_attr_t(size_t smem, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_w<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_dense_w<DV>, WT, smem);
}
template <int DV>
static cudaError_t mti_w_attr_t(size_t smem, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_mti_w<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_mti_w<DV>, WT, smem);
}
template <int DV>
static cudaError_t dense_w_launch_t(const IterParams &p, int grid, size_t smem, cudaStream_t s, const int32_t *md,
                                    int32_t *ns, int32_t *fr) {
    k_dense_w<DV><<<grid, WT, smem, s>>>(p, md, ns, fr);
    return cudaGetLastError();
}
template <int DV>
static cudaError_t mti_w_launch_t(const IterParams &p, int grid, size_t smem, cudaStream_t s, const int32_t *md,
                                  int32_t *ns, int32_t *fr) {
    k_mti_w<DV><<<grid, WT, smem, s>>>(p, md, ns, fr);
    return cudaGetLastError();
}

cudaError_t dense_w_attr(int dv, size_t smem, int *bps) { KNOR_DVW_SWITCH(dv, dense_w_attr_t, smem, bps) }
cudaError_t mti_w_attr(int dv, size_t smem, int *bps) { KNOR_DVW_SWITCH(dv, mti_w_attr_t, smem, bps) }
cudaError_t launch_dense_w(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                           const int32_t *md, int32_t *ns, int32_t *fr) {
    KNOR_DVW_SWITCH(dv, dense_w_launch_t, p, grid, smem, s, md, ns, fr)
}
cudaError_t launch_mti_w(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                         const int32_t *md, int32_t *ns, int32_t *fr) {
    KNOR_DVW_SWITCH(dv, mti_w_launch_t, p, grid, smem, s, md, ns, fr)
}

} // namespace knor

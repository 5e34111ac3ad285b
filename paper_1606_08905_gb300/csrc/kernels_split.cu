// kernels_split.cu -- the MTI iteration's point work as two kernels.
//
// k_mti_sel   Clause 1 ("Minimal Triangle Inequality (MTI) Pruning") on the
//             packed state of every point.  Each warp owns a contiguous range
//             of points, streams its state, and puts the points that Clause 1
//             cannot skip into buckets in shared memory (32 local indices
//             each): one per cluster for its light points, and one shared
//             "mixed" bucket for the heavy points and the unassigned ones.
//             A point is heavy when its bound reaches the M-th smallest
//             1/2 d(c_a, c) of its cluster, so that Clause 2 would leave it
//             M or more candidates: one such point in a batch makes the
//             union the scan walks for all 32 lanes large, so heavy points
//             are batched apart and scored against every centroid.  A bucket
//             that fills is written out at once as one batch record
//             (cluster or k for mixed, count, 32 point indices) to the
//             warp's own list, and the partial buckets follow at the end.
//             Nothing but the 8-byte state of a point is read here.
// k_mti_scan  Clauses 3 and 2 on the records: warp w scans list w in order.
//             While it scores one batch, the rows of its next two batches
//             are on their way into the warp's two shared-memory slots
//             (cp.async), so the row gathers overlap the arithmetic.  The
//             points of a batch share their cluster a, hence the row of the
//             k x k table, and their Clause-2 candidate sets are nested, so
//             the warp walks one union; the points of a mixed batch score
//             every centroid.  New state; the points that changed
//             cluster go to the warp's change list (point, new and old
//             cluster).
// k_dense_scan  the full scan (plain Lloyd, the first MTI iteration) over the
//             same warp ranges, appending its changed points to the same lists.
// k_elkan_scan  Elkan's algorithm (MTI plus per-centroid lower bounds), the
//             ablation the paper leaves out, on the same ranges and lists.
// k_mti_delta Phase II by deltas: the rows of the change lists are added to
//             their new clusters and subtracted from their old ones (TwoSum
//             pairs in shared memory), each list split over a few warps.
//
// Record and change lists are a pure function of the state, and each is
// processed by one warp in order, so the sums (each CTA adds its warps'
// accumulators in warp order) do not depend on timing.
#include "device_common.cuh"
#include "knor_internal.cuh"

namespace knor {
namespace {

constexpr int SPW = SP_WPB; // warps per CTA of both kernels
constexpr int SPT = SPW * 32;

// Contiguous point range of global warp gw of nw, boundaries on multiples of
// WPA (so that state chunks start 32-byte aligned).
__device__ __forceinline__ void warp_range(int64_t n, int gw, int nw, int64_t &lo, int64_t &hi) {
    const int64_t units = (n + WPA - 1) / WPA;
    lo = min(n, units * gw / nw * WPA);
    hi = min(n, units * (gw + 1) / nw * WPA);
}

__device__ __forceinline__ long long sp_warp_sum(long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

} // namespace

// ---------------------------------------------------------------- Clause 1

__global__ void __launch_bounds__(SPT) k_mti_sel(const IterParams p, const int32_t *mode_dense) {
    if (*mode_dense != 0) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int k = p.k;
    float *s_s = reinterpret_cast<float *>(sm + p.off_s);
    float *F_s = reinterpret_cast<float *>(sm + p.off_F);
    float *th_s = reinterpret_cast<float *>(sm + p.off_th); // heavy thresholds (+inf: no split)
    for (int c = tid; c < k; c += SPT) {
        s_s[c] = p.s[c];
        F_s[c] = p.F[c];
        th_s[c] = p.theta != nullptr ? p.theta[c] : CUDART_INF_F;
    }
    unsigned char *wr = sm + p.w_base + w * p.w_stride;
    // buckets of 32 local indices: cluster a for its light points, k for
    // the heavy and the unassigned ones
    int *bk = reinterpret_cast<int *>(wr + p.w_bucket);
    int *bcnt = bk + (k + 1) * 32;
    PtState *stbuf = reinterpret_cast<PtState *>(wr + p.w_state);
    for (int c = lane; c <= k; c += 32) bcnt[c] = 0;
    __syncthreads();
    const int gw = blockIdx.x * SPW + w, nw = gridDim.x * SPW;
    int64_t lo, hi;
    warp_range(p.n, gw, nw, lo, hi);
    // offsets within the range are 32-bit (n <= 2^31)
    const int len = (int)(hi - lo);
    const int nchunk = (len + WCH - 1) / WCH;
    const PtState *st_lo = p.st + lo;
    int32_t *rec = p.rec + (size_t)gw * p.rec_cap * SP_REC;
    int nrec = 0;

    auto prefetch = [&](int stage, int m) {
        if (m < nchunk) {
            const int o0 = m * WCH + lane * WPA;
            if (o0 + WPA <= len) {
                const char *src = reinterpret_cast<const char *>(st_lo + o0);
                char *dst = reinterpret_cast<char *>(stbuf + stage * WCH + lane * WPA);
#pragma unroll
                for (int v = 0; v < WPA * 8 / 16; ++v) cp_async16(dst + 16 * v, src + 16 * v);
            }
        }
        cp_async_commit();
    };
    // Writes the nb (<= 32) points of bucket cb as the next record (the
    // caller then resets the bucket's count).
    auto emit = [&](int cb, int nb) {
        int32_t *r = rec + (size_t)nrec * SP_REC;
        if (lane < nb) r[4 + lane] = (int32_t)(lo + bk[cb * 32 + lane]);
        if (lane == 0) {
            r[0] = cb;
            r[1] = nb;
        }
        __syncwarp(); // every lane has read the bucket before it is refilled
        ++nrec;
    };

    unsigned my_skipped = 0;
#pragma unroll
    for (int s = 0; s < WSTAGES - 1; ++s) prefetch(s, s);
    int stage = 0;
    for (int m = 0; m < nchunk; ++m) {
        prefetch((stage + WSTAGES - 1) % WSTAGES, m + WSTAGES - 1);
        cp_async_wait<WSTAGES - 1>();
        __syncwarp();
        const int o0 = m * WCH + lane * WPA; // this lane's first point, from lo
        PtState ps[WPA];
        if (o0 + WPA <= len) {
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
                if (o0 + u < len) ps[u] = st_lo[o0 + u];
                else { ps[u].ub = 0.0f; ps[u].a = -2; }
            }
        }
        unsigned amask = 0;
        int nvalid = 0;
        int bkey[WPA]; // bucket of each point
#pragma unroll
        for (int u = 0; u < WPA; ++u) {
            // branch-free: a = -2 past the range, -1 unassigned, else a cluster
            const int a = ps[u].a;
            const int ac = max(a, 0);
            const float uu = __fadd_ru(ps[u].ub, F_s[ac]); // u^t = ub + F^t(a)
            const float t = __fmaf_ru(uu, p.onepk, p.tau);
            const bool valid = a != -2, assigned = a >= 0;
            const bool act = valid && !(assigned && t < s_s[ac]);
            bkey[u] = (assigned && t < th_s[ac]) ? a : k; // th = +inf without the heavy split
            nvalid += valid ? 1 : 0;
            amask |= (act ? 1u : 0u) << u;
        }
        my_skipped += nvalid - __popc(amask);
        // this lane's first place among the chunk's survivors, and their
        // number: one ballot per point slot (independent, short latency)
        int pos = 0, total = 0;
#pragma unroll
        for (int u = 0; u < WPA; ++u) {
            const unsigned b = __ballot_sync(FULL_MASK, (amask >> u) & 1u);
            pos += __popc(b & ((1u << lane) - 1u));
            total += __popc(b);
        }
        // survivors in point order, staged in the state buffer just read
        int2 *stg = reinterpret_cast<int2 *>(stbuf + stage * WCH);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < WPA; ++u) {
            if ((amask >> u) & 1u) {
                stg[pos] = make_int2(o0 + u, bkey[u]);
                ++pos;
            }
        }
        __syncwarp();
        stage = (stage + 1) % WSTAGES;
        for (int base = 0; base < total; base += 32) {
            const int e = base + lane;
            const bool valid = e < total;
            const int2 ent = valid ? stg[e] : make_int2(0, 0);
            const int key = valid ? ent.y : -1 - lane;
            const unsigned grp = __match_any_sync(FULL_MASK, key);
            const int rank = __popc(grp & ((1u << lane) - 1u));
            // the entries that fit go in; a bucket that fills is emitted at
            // once and the rest of its group starts it afresh (point order is
            // kept: first in, first out)
            const int c0 = valid ? bcnt[key] : 0;
            const int now = c0 + __popc(grp);
            if (valid && c0 + rank < 32) bk[key * 32 + c0 + rank] = ent.x;
            __syncwarp();
            unsigned fullm = __ballot_sync(FULL_MASK, valid && rank == 0 && now >= 32);
            while (fullm) {
                const int leader = __ffs(fullm) - 1;
                fullm &= fullm - 1;
                emit(__shfl_sync(FULL_MASK, key, leader), 32);
            }
            if (valid && c0 + rank >= 32) bk[key * 32 + c0 + rank - 32] = ent.x;
            if (valid && rank == 0) bcnt[key] = now >= 32 ? now - 32 : now;
            __syncwarp();
        }
        __syncwarp();
    }
    for (int cb = 0; cb <= k; ++cb) {
        const int left = bcnt[cb];
        if (left > 0) emit(cb, left);
    }
    cp_async_wait<0>();
    const long long t = sp_warp_sum((long long)my_skipped);
    if (lane == 0) {
        p.rec_cnt[gw] = nrec;
        atomicAdd(&p.ctr->skipped, (unsigned long long)t);
    }
}

// ------------------------------------------------------------ Clauses 2-3

namespace {

// Adds the staged rows of the lanes with has = true, in lane order, to their
// new clusters and subtracts them from their old ones (cl: new << 16 | old,
// old 0xFFFF for none), one row at a time with the lanes walking the
// dimensions: every (cluster, dimension) accumulator takes its rows in a
// fixed order.  Member counts move by shared-memory integer atomics.
template <int DV>
__device__ __forceinline__ void sp_accumulate_rows(const float *rb, int rs, int cl, bool has, float *acc_hi,
                                                   float *acc_lo, int *cnt) {
    const int lane = threadIdx.x & 31;
    const int cnew = (int)((unsigned)cl >> 16), cold = cl & 0xFFFF;
    if (has) {
        atomicAdd(&cnt[cnew], 1);
        if (cold != 0xFFFF) atomicAdd(&cnt[cold], -1);
    }
    for (unsigned m = __ballot_sync(FULL_MASK, has); m; m &= m - 1) {
        const int pl = __ffs(m) - 1;
        const int c = __shfl_sync(FULL_MASK, cl, pl);
        const int cn = (int)((unsigned)c >> 16), co = c & 0xFFFF;
#pragma unroll
        for (int j = lane; j < (DV < 32 ? 32 : DV); j += 32) {
            if (DV >= 32 || j < DV) {
                const float x = rb[pl * rs + j];
                two_sum_acc(&acc_hi[cn * DV + j], &acc_lo[cn * DV + j], x);
                if (co != 0xFFFF) two_sum_acc(&acc_hi[co * DV + j], &acc_lo[co * DV + j], -x);
            }
        }
    }
}

} // namespace

// DV <= 32: up to 5 CTAs (20 warps) per SM; DV = 64: the row slots limit it.
template <int DV>
__global__ void __launch_bounds__(SPT, DV <= 32 ? 5 : 2) k_mti_scan(const IterParams p, const int32_t *mode_dense,
                                                                    int32_t *nslots, int32_t *fresh) {
    if (*mode_dense != 0) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int k = p.k;
    const int rs = p.sp_rs;
    float *cent = reinterpret_cast<float *>(sm + p.off_cent);
    float *halfD = reinterpret_cast<float *>(sm + p.off_halfD);
    float *F_s = reinterpret_cast<float *>(sm + p.off_F);
    for (int e = tid; e < k * DV; e += SPT) cent[e] = p.C32[e];
    for (int e = tid; e < k * k; e += SPT) halfD[e] = p.halfD[e];
    for (int c = tid; c < k; c += SPT) F_s[c] = p.F[c];
    const int gw = blockIdx.x * SPW + w;
    float *slots = reinterpret_cast<float *>(sm + p.sp_off_warp + w * p.sp_warp_stride); // 2 x 32 rows
    int2 *chg = p.chg + (size_t)gw * p.chg_cap; // (point, new << 16 | old) of the points that changed
    int nchg = 0;
    __syncthreads();

    // this warp's record lists (sel_mult of them, back to back in memory)
    const int32_t *rec = p.rec + (size_t)gw * p.sel_mult * p.rec_cap * SP_REC;
    const int n0 = p.rec_cnt[gw * p.sel_mult];
    const int nrec = n0 + (p.sel_mult == 2 ? p.rec_cnt[gw * 2 + 1] : 0);
    // Record j's header and this lane's point index.
    auto meta = [&](int j, int &cb, int &nb, int &idx) {
        if (j < nrec) {
            const int32_t *r = rec + (size_t)(j < n0 ? j : j - n0 + (int)p.rec_cap) * SP_REC;
            const int2 h = *reinterpret_cast<const int2 *>(r);
            cb = h.x;
            nb = h.y;
            idx = r[4 + lane]; // (slots past nb hold stale values, never used)
        } else {
            cb = 0;
            nb = 0;
            idx = 0;
        }
    };
    // The rows of a record into slot `slot`: piece f (16 bytes) of the batch
    // is row f / (DV/4), so one warp instruction copies whole rows side by
    // side; then the copies are committed as one group.
    auto fetch = [&](int slot, int nb, int idx) {
        constexpr int CH = DV / 4;
        float *dst = slots + (size_t)slot * 32 * rs;
        // lane l copies piece l % CH of rows l / CH, l / CH + 32 / CH, ...
        const int part = lane % CH;
#pragma unroll
        for (int base = 0; base < 32 * CH; base += 32) {
            const int r = (base + lane) / CH;
            const int ir = __shfl_sync(FULL_MASK, idx, r);
            if (r < nb) cp_async16(dst + r * rs + part * 4, p.X + (int64_t)ir * DV + part * 4);
        }
        cp_async_commit();
    };

    unsigned my_evals = 0, my_changed = 0;
    // Two batches in flight: the rows of batch j + 2 go into the slot of
    // batch j as soon as batch j's rows are in registers.
    // The cluster of a lane's point in a mixed record (k: heavy points of any
    // cluster and unassigned ones, -1), read from the state when the rows of
    // the record are requested, two batches ahead.
    auto own_cluster = [&](int cb, int nb, int idx) { return cb == k && lane < nb ? p.st[idx].a : -1; };
    int cb0, nb0, ix0, cb1, nb1, ix1, cb2, nb2, ix2;
    meta(0, cb0, nb0, ix0);
    fetch(0, nb0, ix0);
    int al0 = own_cluster(cb0, nb0, ix0);
    meta(1, cb1, nb1, ix1);
    fetch(1, nb1, ix1);
    int al1 = own_cluster(cb1, nb1, ix1);
    meta(2, cb2, nb2, ix2);
    for (int j = 0; j < nrec; ++j) {
        cp_async_wait<1>();
        __syncwarp();
        const float *rb = slots + (size_t)(j & 1) * 32 * rs;
        const bool mixed = cb0 == k;
        const int a = mixed ? al0 : cb0; // this lane's cluster (-1: none yet)
        const int nb = nb0;
        int best = -1;
        unsigned long long xk[DV / 2];
        float bd = CUDART_INF_F, tst = 0.0f;
        if (lane < nb) {
#pragma unroll
            for (int jj = 0; jj < DV; jj += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(rb + lane * rs + jj);
                xk[jj / 2] = pack2(v.x, v.y);
                xk[jj / 2 + 1] = pack2(v.z, v.w);
            }
        }
        __syncwarp(); // every lane has its row: the slot takes batch j + 2
        fetch(j & 1, nb2, ix2);
        const int al2 = own_cluster(cb2, nb2, ix2);
        int cb3, nb3, ix3;
        meta(j + 3, cb3, nb3, ix3);
        if (lane < nb) {
            if (mixed) {
                // every centroid, in index order (the argmin with ties to the
                // lower index); for a heavy point the evaluations counted are
                // the ones Clauses 3 and 2 leave, as in a cluster's batch
                const float *hl = halfD + (size_t)max(a, 0) * k;
                float tl = 0.0f;
                if (a >= 0) {
                    tl = __fmaf_ru(bound_up(d2_reg<DV>(xk, cent + (size_t)a * DV), p.g_up, p.tiny), p.onepk, p.tau);
                    ++my_evals;
                } else {
                    my_evals += k;
                }
                best = 0;
                int c = 0;
                for (; c + 4 <= k; c += 4) {
                    float r[4];
                    d2_reg4<DV>(xk, cent + (size_t)c * DV, cent + (size_t)(c + 1) * DV, cent + (size_t)(c + 2) * DV,
                                cent + (size_t)(c + 3) * DV, r);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (r[q] < bd) { bd = r[q]; best = c + q; }
                        my_evals += (a >= 0 && c + q != a && !(tl < hl[c + q])) ? 1u : 0u;
                    }
                }
                for (; c < k; ++c) {
                    const float r = d2_reg<DV>(xk, cent + (size_t)c * DV);
                    if (r < bd) { bd = r; best = c; }
                    my_evals += (a >= 0 && c != a && !(tl < hl[c])) ? 1u : 0u;
                }
            } else {
                // Clause 3: tighten u to (a bound on) the exact d(v, c_a)
                bd = d2_reg<DV>(xk, cent + (size_t)a * DV);
                best = a;
                ++my_evals;
            }
            tst = __fmaf_ru(bound_up(bd, p.g_up, p.tiny), p.onepk, p.tau);
        }
        // Clause 2: every centroid c != a with u >= 1/2 d(c_a, c) survives.
        // The union of the lanes' survivor sets is the set of the largest
        // bound: lane b tests centroid cw + b against it and the warp walks
        // the union in index order.  Every lane scores every centroid of the
        // union: one that its own bound prunes is strictly farther than c_a
        // in computed FP32 values, so it cannot change the argmin (only the
        // lanes it survives count it as an evaluation).
        if (!mixed) {
            const float *hrow = halfD + (size_t)a * k;
            // tst >= 0 (sign bit cleared for -0): its bit pattern orders like the value
            const float tmax = __uint_as_float(__reduce_max_sync(FULL_MASK, __float_as_uint(tst) & 0x7fffffffu));
            for (int cw = 0; cw < k; cw += 32) {
                const int cl = cw + lane;
                unsigned uni = __ballot_sync(FULL_MASK, cl < k && cl != a && !(tmax < hrow[min(cl, k - 1)]));
                // four or two members per step (independent chains), in index order
                while (__popc(uni) >= 4) {
                    int cc[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        cc[q] = cw + __ffs(uni) - 1;
                        uni &= uni - 1;
                    }
                    if (lane < nb) {
                        float r[4];
                        d2_reg4<DV>(xk, cent + (size_t)cc[0] * DV, cent + (size_t)cc[1] * DV,
                                    cent + (size_t)cc[2] * DV, cent + (size_t)cc[3] * DV, r);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            my_evals += tst < hrow[cc[q]] ? 0u : 1u;
                            if (r[q] < bd || (r[q] == bd && cc[q] < best)) { bd = r[q]; best = cc[q]; }
                        }
                    }
                }
                while (uni) {
                    const int c = cw + __ffs(uni) - 1;
                    uni &= uni - 1;
                    if (uni) {
                        const int c2 = cw + __ffs(uni) - 1;
                        uni &= uni - 1;
                        if (lane < nb) {
                            float r, r2;
                            d2_reg2<DV>(xk, cent + (size_t)c * DV, cent + (size_t)c2 * DV, r, r2);
                            my_evals += (tst < hrow[c] ? 0u : 1u) + (tst < hrow[c2] ? 0u : 1u);
                            if (r < bd || (r == bd && c < best)) { bd = r; best = c; }
                            if (r2 < bd || (r2 == bd && c2 < best)) { bd = r2; best = c2; }
                        }
                    } else if (lane < nb) {
                        const float r = d2_reg<DV>(xk, cent + (size_t)c * DV);
                        my_evals += tst < hrow[c] ? 0u : 1u;
                        if (r < bd || (r == bd && c < best)) { bd = r; best = c; }
                    }
                }
            }
        }
        bool changed = false;
        if (lane < nb) {
            PtState ns;
            ns.a = best;
            ns.ub = __fsub_ru(bound_up(bd, p.g_up, p.tiny), F_s[best]);
            p.st[ix0] = ns;
            changed = best != a;
        }
        // the points that changed cluster, in batch order, for k_mti_delta
        // (an unassigned point has old cluster 0xFFFF: nothing to subtract)
        const unsigned cm = __ballot_sync(FULL_MASK, changed);
        if (changed)
            chg[nchg + __popc(cm & ((1u << lane) - 1u))] =
                make_int2(ix0, (int)(((unsigned)best << 16) | ((unsigned)a & 0xFFFFu)));
        nchg += __popc(cm);
        my_changed += __popc(cm);
        cb0 = cb1; nb0 = nb1; ix0 = ix1; al0 = al1;
        cb1 = cb2; nb1 = nb2; ix1 = ix2; al1 = al2;
        cb2 = cb3; nb2 = nb3; ix2 = ix3;
    }
    cp_async_wait<0>();
    const long long t2 = sp_warp_sum((long long)my_evals);
    if (lane == 0) {
        p.chg_cnt[gw] = nchg;
        atomicAdd(&p.ctr->changed, (unsigned long long)my_changed);
        atomicAdd(&p.ctr->evals, (unsigned long long)t2);
    }
}

// --------------------------------------------------------------- dense scan

// Every point scans every centroid (plain Lloyd, the first MTI iteration):
// warp w takes the same range as k_mti_sel's warp w, DS_P x 32 rows per tile
// (double-buffered with cp.async), DS_P points per lane (lane l has rows l,
// l + 32, ...), so each centroid read from shared memory serves DS_P
// distances, two centroids per step; writes the new state and appends the
// points that changed cluster to change list w, in point order, for
// k_mti_delta.
constexpr int DS_P = KNOR_DS_P;

template <int DV>
__global__ void __launch_bounds__(SPT) k_dense_scan(const IterParams p, const int32_t *mode_dense) {
    if (*mode_dense == 0) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int k = p.k;
    const int rs = p.sp_rs;
    constexpr int TR = 32 * DS_P; // rows per tile
    float *cent = reinterpret_cast<float *>(sm + p.off_cent);
    float *F_s = reinterpret_cast<float *>(sm + p.off_F);
    for (int e = tid; e < k * DV; e += SPT) cent[e] = p.C32[e];
    for (int c = tid; c < k; c += SPT) F_s[c] = p.F[c];
    float *tiles = reinterpret_cast<float *>(sm + p.sp_off_warp + w * p.sp_warp_stride); // 2 x TR rows
    __syncthreads();
    const int gw = blockIdx.x * SPW + w, nw = gridDim.x * SPW;
    int64_t lo, hi;
    warp_range(p.n, gw, nw, lo, hi);
    const int64_t ntile = (hi - lo + TR - 1) / TR;
    int2 *chg = p.chg + (size_t)gw * p.chg_cap;
    int nchg = 0;
    auto load_tile = [&](int slot, int64_t t) {
        if (t < ntile) {
            constexpr int CH = DV / 4;
            const int64_t base = lo + t * TR;
            const int rows = (int)min((int64_t)TR, hi - base);
            float *dst = tiles + (size_t)slot * TR * rs;
            const float *src = p.X + base * DV;
            for (int f = lane; f < rows * CH; f += 32) cp_async16(dst + (f / CH) * rs + (f % CH) * 4, src + (size_t)f * 4);
        }
        cp_async_commit();
    };
    unsigned my_changed = 0;
    load_tile(0, 0);
    for (int64_t t = 0; t < ntile; ++t) {
        load_tile((int)((t + 1) & 1), t + 1);
        cp_async_wait<1>();
        __syncwarp();
        const int64_t base = lo + t * TR;
        const int rows = (int)min((int64_t)TR, hi - base);
        const float *tl = tiles + (size_t)(t & 1) * TR * rs;
        // rows past the end compute on row 0 of the tile and are dropped
        unsigned long long x2[DS_P][DV / 2];
        float bd[DS_P];
        int best[DS_P], olda[DS_P];
#pragma unroll
        for (int q = 0; q < DS_P; ++q) {
            const int r = q * 32 + lane;
            // the old assignment is loaded here, so its latency hides under the scan
            olda[q] = r < rows ? p.st[base + r].a : -1;
            load_x2<DV>(x2[q], tl + (r < rows ? r : 0) * rs);
            bd[q] = CUDART_INF_F;
            best[q] = 0;
        }
        // Elkan's lower bounds, when kept: every distance of a full scan sets one
        auto keep = [&](int q, int c, float r) {
            const int rr = q * 32 + lane;
            if (p.lb != nullptr && rr < rows)
                p.lb[(size_t)c * p.n + base + rr] = __fadd_rd(bound_down(r, p.ginv_dn, p.tiny), F_s[c]);
        };
        int c = 0;
        for (; c + 2 <= k; c += 2) {
#pragma unroll
            for (int q = 0; q < DS_P; ++q) {
                float r0, r1;
                d2_reg2<DV>(x2[q], cent + (size_t)c * DV, cent + (size_t)(c + 1) * DV, r0, r1);
                if (r0 < bd[q]) { bd[q] = r0; best[q] = c; }
                if (r1 < bd[q]) { bd[q] = r1; best[q] = c + 1; }
                keep(q, c, r0);
                keep(q, c + 1, r1);
            }
        }
        for (; c < k; ++c) {
#pragma unroll
            for (int q = 0; q < DS_P; ++q) {
                const float r = d2_reg<DV>(x2[q], cent + (size_t)c * DV);
                if (r < bd[q]) { bd[q] = r; best[q] = c; }
                keep(q, c, r);
            }
        }
#pragma unroll
        for (int q = 0; q < DS_P; ++q) {
            const int r = q * 32 + lane;
            const int64_t i = base + r;
            bool changed = false;
            if (r < rows) {
                PtState ns;
                ns.a = best[q];
                ns.ub = p.mti ? __fsub_ru(bound_up(bd[q], p.g_up, p.tiny), F_s[best[q]]) : 0.0f;
                p.st[i] = ns;
                changed = olda[q] != best[q];
            }
            const unsigned cm = __ballot_sync(FULL_MASK, changed);
            if (changed)
                chg[nchg + __popc(cm & ((1u << lane) - 1u))] =
                    make_int2((int)i, (int)(((unsigned)best[q] << 16) | ((unsigned)olda[q] & 0xFFFFu)));
            nchg += __popc(cm);
            my_changed += __popc(cm);
        }
        __syncwarp(); // the tile's slot is refilled two steps on
    }
    cp_async_wait<0>();
    if (lane == 0) {
        p.chg_cnt[gw] = nchg;
        atomicAdd(&p.ctr->changed, (unsigned long long)my_changed);
        atomicAdd(&p.ctr->evals, (unsigned long long)((hi - lo) * (int64_t)k));
    }
}

// ------------------------------------------------------------ Elkan's scan

// Elkan's algorithm as an ablation of MTI: the same Clause 1 on the same
// upper bound, then for every other centroid c the fourth test besides
// Clause 2 -- c is ruled out when u is below max(1/2 d(c_a, c), l(x, c)),
// with l(x, c) = lb[c][x] - F(c) rounded down -- tightening u (Clause 3) the
// first time a centroid survives; every computed distance refreshes its
// lower bound.  One point per lane, 32-point tiles of warp w's range (the
// split grid's ranges), so the lower-bound loads of a warp are coalesced;
// the points that changed cluster go to change list w for k_mti_delta.
template <int DV>
__global__ void __launch_bounds__(SPT) k_elkan_scan(const IterParams p, const int32_t *mode_dense) {
    if (*mode_dense != 0) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int k = p.k;
    float *cent = reinterpret_cast<float *>(sm + p.off_cent);
    float *halfD = reinterpret_cast<float *>(sm + p.off_halfD);
    float *s_s = reinterpret_cast<float *>(sm + p.off_s);
    float *F_s = reinterpret_cast<float *>(sm + p.off_F);
    for (int e = tid; e < k * DV; e += SPT) cent[e] = p.C32[e];
    for (int e = tid; e < k * k; e += SPT) halfD[e] = p.halfD[e];
    for (int c = tid; c < k; c += SPT) { s_s[c] = p.s[c]; F_s[c] = p.F[c]; }
    __syncthreads();
    const int gw = blockIdx.x * SPW + w, nw = gridDim.x * SPW;
    int64_t lo, hi;
    warp_range(p.n, gw, nw, lo, hi);
    int2 *chg = p.chg + (size_t)gw * p.chg_cap;
    int nchg = 0;
    unsigned my_skipped = 0, my_evals = 0, my_changed = 0;
    for (int64_t base = lo; base < hi; base += 32) {
        const int64_t i = base + lane;
        bool changed = false;
        int a = -1, best = -1;
        if (i < hi) {
            const PtState ps = p.st[i];
            a = ps.a;
            bool active = true;
            float u = 0.0f, tst = 0.0f;
            if (a >= 0) {
                u = __fadd_ru(ps.ub, F_s[a]); // u^t = ub + F^t(a)
                tst = __fmaf_ru(u, p.onepk, p.tau);
                active = !(tst < s_s[a]); // Clause 1
            }
            if (!active) {
                ++my_skipped;
            } else {
                unsigned long long xk[DV / 2];
                if constexpr (DV % 8 == 0) ldg_x2_w32<DV>(xk, p.X + i * DV);
                else ldg_x2<DV>(xk, p.X + i * DV);
                float bd = CUDART_INF_F;
                bool tight = false;
                if (a < 0) { // no assignment yet: every distance, every bound
                    best = 0;
                    for (int c = 0; c < k; ++c) {
                        const float r = d2_reg<DV>(xk, cent + (size_t)c * DV);
                        p.lb[(size_t)c * p.n + i] = __fadd_rd(bound_down(r, p.ginv_dn, p.tiny), F_s[c]);
                        if (r < bd) { bd = r; best = c; }
                    }
                    my_evals += k;
                    tight = true;
                } else {
                    best = a;
                    for (int c = 0; c < k; ++c) {
                        if (c == a) continue;
                        const float l = __fsub_rd(p.lb[(size_t)c * p.n + i], F_s[c]);
                        const float thr = fmaxf(halfD[(size_t)a * k + c], l);
                        if (tst < thr) continue; // Clause 2 or the fourth test
                        if (!tight) {
                            // Clause 3: tighten u to (a bound on) the exact d(v, c_a)
                            bd = d2_reg<DV>(xk, cent + (size_t)a * DV);
                            ++my_evals;
                            p.lb[(size_t)a * p.n + i] = __fadd_rd(bound_down(bd, p.ginv_dn, p.tiny), F_s[a]);
                            tst = __fmaf_ru(bound_up(bd, p.g_up, p.tiny), p.onepk, p.tau);
                            tight = true;
                            if (tst < thr) continue;
                        }
                        const float r = d2_reg<DV>(xk, cent + (size_t)c * DV);
                        ++my_evals;
                        p.lb[(size_t)c * p.n + i] = __fadd_rd(bound_down(r, p.ginv_dn, p.tiny), F_s[c]);
                        if (r < bd || (r == bd && c < best)) { bd = r; best = c; }
                    }
                }
                if (tight) { // otherwise u stays as it was (no write)
                    PtState ns;
                    ns.a = best;
                    ns.ub = __fsub_ru(bound_up(bd, p.g_up, p.tiny), F_s[best]);
                    p.st[i] = ns;
                }
                changed = best != a;
            }
        }
        const unsigned cm = __ballot_sync(FULL_MASK, changed);
        if (changed)
            chg[nchg + __popc(cm & ((1u << lane) - 1u))] =
                make_int2((int)i, (int)(((unsigned)best << 16) | ((unsigned)a & 0xFFFFu)));
        nchg += __popc(cm);
        my_changed += __popc(cm);
    }
    const long long t1 = sp_warp_sum((long long)my_skipped);
    const long long t2 = sp_warp_sum((long long)my_evals);
    if (lane == 0) {
        p.chg_cnt[gw] = nchg;
        atomicAdd(&p.ctr->changed, (unsigned long long)my_changed);
        atomicAdd(&p.ctr->skipped, (unsigned long long)t1);
        atomicAdd(&p.ctr->evals, (unsigned long long)t2);
    }
}

// Debug check of Elkan's lower bounds after an iteration: a bound above an
// upper bound on the exact distance (from the FP32 distance and its error
// bound) is counted as a violation of the run's current record.
template <int DV>
__global__ void k_elkan_check(const IterParams p, IterStats *stats, const int32_t *run_iter) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    unsigned long long xk[DV / 2];
    ldg_x2<DV>(xk, p.X + i * DV);
    unsigned bad = 0;
    for (int c = 0; c < p.k; ++c) {
        const float r = d2_reg<DV>(xk, p.C32 + (size_t)c * DV);
        const float l = __fsub_rd(p.lb[(size_t)c * p.n + i], p.F[c]);
        if (l > bound_up(r, p.g_up, p.tiny)) ++bad;
    }
    if (bad) atomicAdd(reinterpret_cast<unsigned long long *>(&stats[*run_iter - 1].violations), bad);
}

// ------------------------------------------------------------ delta sums

// Adds (NEG: subtracts) row xrow to cluster cl's TwoSum accumulators (hi, lo
// pairs side by side, so that one 8-byte access moves both and a lane group
// of 16 spans all 32 banks), lane jl of the row's lane group taking
// dimensions jl, jl + 32, ...
template <int DV, bool NEG>
__device__ __forceinline__ void dl_add(float2 *acc, int cl, const float *xrow, int jl) {
    constexpr int GW = DV < 32 ? DV : 32;
#pragma unroll
    for (int r = 0; r < DV / GW; ++r) {
        const int o = cl * DV + jl + GW * r;
        const float x = xrow[jl + GW * r];
        float2 v = acc[o];
        two_sum_reg(v.x, v.y, NEG ? -x : x);
        acc[o] = v;
    }
}

// Phase II by deltas: CTA b takes the change lists of scan CTA b, each
// split into p.dl_split consecutive parts with one warp per part (warp w:
// list w / dl_split, part w % dl_split).  A warp takes its entries 32 at a
// time; the rows of the next 32 are copied into the warp's second row slot
// (cp.async, 16-byte pieces) while it adds the current ones.  A row takes
// GW = min(d, 32) lanes, so P = 32 / GW rows go at once (lane group g has
// row sP + g in step s): each row is added to its new cluster and then
// subtracted from its old one in the warp's TwoSum accumulators (shared
// memory).  Rows of one step that meet in a cluster go one group after the
// other, so every (cluster, dimension) accumulator takes its rows in list
// order, adds before subtractions within a step.  The CTA adds its warps'
// accumulators in warp order into its partial slot.  Order and grouping
// depend only on the lists and the fixed split: deterministic.
template <int DV>
__global__ void __launch_bounds__(512) k_mti_delta(const IterParams p, const int32_t *mode_dense, int32_t *nslots,
                                                    int32_t *fresh) {
    if (*mode_dense != 0 ? !p.dl_dense : !p.dl_mti) return; // this iteration's scan summed for itself
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int nthr = blockDim.x;
    const int k = p.k;
    constexpr int GW = DV < 32 ? DV : 32; // lanes per row
    constexpr int P = 32 / GW;            // rows per step
    constexpr int CH = DV / 4;            // 16-byte pieces per row
    constexpr unsigned GMASK = (1u << P) - 1u;
    const int g = lane / GW, jl = lane % GW;
    if (blockIdx.x == 0 && tid == 0) { *nslots = (int)gridDim.x; *fresh = 0; }
    unsigned char *wr = sm + (size_t)w * p.dl_warp_stride;
    float2 *acc = reinterpret_cast<float2 *>(wr); // k x DV (hi, lo) pairs
    int *cnt = reinterpret_cast<int *>(acc + (size_t)k * DV);
    float *slots = reinterpret_cast<float *>(wr + p.dl_off_rows); // 2 x 32 rows of DV floats
    for (int e = lane; e < k * DV; e += 32) acc[e] = make_float2(0.0f, 0.0f);
    for (int c = lane; c < k; c += 32) cnt[c] = 0;
    __syncwarp();
    const int list = blockIdx.x * SPW + w / p.dl_split, part = w % p.dl_split;
    const int2 *chg = p.chg + (size_t)list * p.chg_cap;
    const int nchg = p.chg_cnt[list];
    const int e0 = (int)((int64_t)nchg * part / p.dl_split), e1 = (int)((int64_t)nchg * (part + 1) / p.dl_split);
    auto entry = [&](int g0) { return g0 + lane < e1 ? chg[g0 + lane] : make_int2(0, 0); };
    // the rows of entries g0 .. g0 + 31 (those below e1) into slot `slot`
    auto fetch = [&](int slot, int g0, int idx) {
        const int nb = max(0, min(32, e1 - g0));
        float *dst = slots + (size_t)slot * 32 * DV;
#pragma unroll
        for (int base = 0; base < 32 * CH; base += 32) {
            const int f = base + lane;
            const int ir = __shfl_sync(FULL_MASK, idx, f / CH);
            if (f < nb * CH) cp_async16(dst + (size_t)f * 4, p.X + (int64_t)ir * DV + (f % CH) * 4);
        }
        cp_async_commit();
    };
    int2 cur = entry(e0), nxt = entry(e0 + 32);
    fetch(0, e0, cur.x);
    int slot = 0;
    for (int g0 = e0; g0 < e1; g0 += 32) {
        const int2 nn = entry(g0 + 64);
        fetch(slot ^ 1, g0 + 32, nxt.x); // (nothing when g0 + 32 >= e1)
        const int nb = min(32, e1 - g0);
        const bool mine = lane < nb; // this lane's entry (entry `lane` of the batch) exists
        const int cn_l = (int)((unsigned)cur.y >> 16), co_l = cur.y & 0xFFFF;
        if (mine) {
            atomicAdd(&cnt[cn_l], 1);
            if (co_l != 0xFFFF) atomicAdd(&cnt[co_l], -1);
        }
        const bool any_old = __any_sync(FULL_MASK, mine && co_l != 0xFFFF);
        // entries whose step (entry / P) has another entry of the same new
        // (old) cluster: those steps go one group after the other
        unsigned clash_n = 0, clash_o = 0;
        if constexpr (P > 1) {
            const int st = lane / P;
            const unsigned mn = __match_any_sync(FULL_MASK, mine ? (st << 16 | cn_l) : -1 - lane);
            clash_n = __ballot_sync(FULL_MASK, __popc(mn) > 1);
            if (any_old) {
                const bool ho = mine && co_l != 0xFFFF;
                const unsigned mo = __match_any_sync(FULL_MASK, ho ? (st << 16 | co_l) : -1 - lane);
                clash_o = __ballot_sync(FULL_MASK, __popc(mo) > 1);
            }
        }
        cp_async_wait<1>();
        __syncwarp();
        const float *rb = slots + (size_t)slot * 32 * DV;
        if (nb == 32 && !any_old && clash_n == 0) {
            // a full batch of additions without clashes (the dense step's)
#pragma unroll
            for (int s0 = 0; s0 < 32; s0 += P) {
                const int q = s0 + g;
                const int c = __shfl_sync(FULL_MASK, cur.y, q);
                dl_add<DV, false>(acc, (int)((unsigned)c >> 16), rb + (size_t)q * DV, jl);
                if constexpr (P > 1) __syncwarp();
            }
        } else {
            for (int s0 = 0; s0 < nb; s0 += P) {
                const int q = s0 + g; // this lane group's entry
                const int c = __shfl_sync(FULL_MASK, cur.y, q);
                const bool hn = q < nb;
                const float *xrow = rb + (size_t)q * DV;
                const int cn = (int)((unsigned)c >> 16), co = c & 0xFFFF;
                if (P == 1 || ((clash_n >> s0) & GMASK) == 0) {
                    if (hn) dl_add<DV, false>(acc, cn, xrow, jl);
                } else {
                    for (int gg = 0; gg < P; ++gg) {
                        if (hn && g == gg) dl_add<DV, false>(acc, cn, xrow, jl);
                        __syncwarp();
                    }
                }
                if constexpr (P > 1) __syncwarp(); // later groups see these sums
                if (any_old) {
                    const bool ho = hn && co != 0xFFFF;
                    if (P == 1 || ((clash_o >> s0) & GMASK) == 0) {
                        if (ho) dl_add<DV, true>(acc, co, xrow, jl);
                    } else {
                        for (int gg = 0; gg < P; ++gg) {
                            if (ho && g == gg) dl_add<DV, true>(acc, co, xrow, jl);
                            __syncwarp();
                        }
                    }
                    if constexpr (P > 1) __syncwarp();
                }
            }
        }
        __syncwarp(); // every lane is done with the slot before it is refilled
        cur = nxt;
        nxt = nn;
        slot ^= 1;
    }
    cp_async_wait<0>();
    __syncthreads();
    const int kd = k * DV, nw = nthr >> 5;
    for (int e = tid; e < kd; e += nthr) {
        double sum = 0.0;
        for (int q = 0; q < nw; ++q) {
            const float2 a = reinterpret_cast<const float2 *>(sm + (size_t)q * p.dl_warp_stride)[e];
            sum += (double)a.x;
            sum += (double)a.y;
        }
        p.part_S[(size_t)e * p.part_stride + blockIdx.x] = sum;
    }
    for (int c = tid; c < k; c += nthr) {
        long long sum = 0;
        for (int q = 0; q < nw; ++q) sum += reinterpret_cast<const int *>(sm + (size_t)q * p.dl_warp_stride + (size_t)2 * kd * 4)[c];
        p.part_cnt[(size_t)c * p.part_stride + blockIdx.x] = sum;
    }
}

// ------------------------------------------------------------- launchers

cudaError_t mti_sel_attr(int wpb, size_t smem, int *bps) {
    if (wpb != SPW) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_mti_sel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_mti_sel, SPT, smem);
}
cudaError_t launch_mti_sel(const IterParams &p, int grid, size_t smem, cudaStream_t s, const int32_t *md) {
    k_mti_sel<<<grid, SPT, smem, s>>>(p, md);
    return cudaGetLastError();
}

template <int DV>
static cudaError_t mti_scan_attr_t(size_t smem, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_mti_scan<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_mti_scan<DV>, SPT, smem);
}
template <int DV>
static cudaError_t mti_scan_launch_t(const IterParams &p, int grid, size_t smem, cudaStream_t s, const int32_t *md,
                                     int32_t *ns, int32_t *fr) {
    k_mti_scan<DV><<<grid, SPT, smem, s>>>(p, md, ns, fr);
    return cudaGetLastError();
}

#define KNOR_DVSP_SWITCH(dv, FN, ...)                    \
    switch (dv) {                                        \
    case 8: return FN<8>(__VA_ARGS__);                   \
    case 16: return FN<16>(__VA_ARGS__);                 \
    case 32: return FN<32>(__VA_ARGS__);                 \
    case 64: return FN<64>(__VA_ARGS__);                 \
    default: return cudaErrorInvalidValue;               \
    }

template <int DV>
static cudaError_t mti_delta_attr_t(size_t smem, int split, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_mti_delta<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_mti_delta<DV>, SPT * split, smem);
}
template <int DV>
static cudaError_t mti_delta_launch_t(const IterParams &p, int grid, size_t smem, cudaStream_t s,
                                      const int32_t *md, int32_t *ns, int32_t *fr) {
    k_mti_delta<DV><<<grid, SPT * p.dl_split, smem, s>>>(p, md, ns, fr);
    return cudaGetLastError();
}

template <int DV>
static cudaError_t dense_scan_attr_t(size_t smem, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_scan<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_dense_scan<DV>, SPT, smem);
}
template <int DV>
static cudaError_t dense_scan_launch_t(const IterParams &p, int grid, size_t smem, cudaStream_t s,
                                       const int32_t *md) {
    k_dense_scan<DV><<<grid, SPT, smem, s>>>(p, md);
    return cudaGetLastError();
}
cudaError_t dense_scan_attr(int dv, size_t smem, int *bps) { KNOR_DVSP_SWITCH(dv, dense_scan_attr_t, smem, bps) }
cudaError_t launch_dense_scan(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                              const int32_t *md) {
    KNOR_DVSP_SWITCH(dv, dense_scan_launch_t, p, grid, smem, s, md)
}

template <int DV>
static cudaError_t elkan_scan_attr_t(size_t smem, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_elkan_scan<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_elkan_scan<DV>, SPT, smem);
}
template <int DV>
static cudaError_t elkan_scan_launch_t(const IterParams &p, int grid, size_t smem, cudaStream_t s,
                                       const int32_t *md) {
    k_elkan_scan<DV><<<grid, SPT, smem, s>>>(p, md);
    return cudaGetLastError();
}
template <int DV>
static cudaError_t elkan_check_launch_t(const IterParams &p, IterStats *stats, const int32_t *run_iter,
                                        cudaStream_t s) {
    k_elkan_check<DV><<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(p, stats, run_iter);
    return cudaGetLastError();
}
cudaError_t elkan_scan_attr(int dv, size_t smem, int *bps) { KNOR_DVSP_SWITCH(dv, elkan_scan_attr_t, smem, bps) }
cudaError_t launch_elkan_scan(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                              const int32_t *md) {
    KNOR_DVSP_SWITCH(dv, elkan_scan_launch_t, p, grid, smem, s, md)
}
cudaError_t launch_elkan_check(int dv, const IterParams &p, IterStats *stats, const int32_t *run_iter,
                               cudaStream_t s) {
    KNOR_DVSP_SWITCH(dv, elkan_check_launch_t, p, stats, run_iter, s)
}

cudaError_t mti_delta_attr(int dv, size_t smem, int split, int *bps) {
    KNOR_DVSP_SWITCH(dv, mti_delta_attr_t, smem, split, bps)
}
cudaError_t launch_mti_delta(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                             const int32_t *md, int32_t *ns, int32_t *fr) {
    KNOR_DVSP_SWITCH(dv, mti_delta_launch_t, p, grid, smem, s, md, ns, fr)
}

cudaError_t mti_scan_attr(int dv, int wpb, size_t smem, int *bps) {
    if (wpb != SPW) return cudaErrorInvalidValue;
    KNOR_DVSP_SWITCH(dv, mti_scan_attr_t, smem, bps)
}
cudaError_t launch_mti_scan(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s, const int32_t *md,
                            int32_t *ns, int32_t *fr) {
    KNOR_DVSP_SWITCH(dv, mti_scan_launch_t, p, grid, smem, s, md, ns, fr)
}

} // namespace knor

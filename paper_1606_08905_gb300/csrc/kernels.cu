// kernels.cu -- sm_103a kernels of libknor.so: Lloyd's k-means with MTI pruning.
//
// One iteration ("Parallel Lloyd's Algorithm", Algorithm 1, with the Clauses
// of "Minimal Triangle Inequality (MTI) Pruning") runs as
//   k_dense | k_mti   Phase I (nearest centroid per point) fused with the
//                     per-CTA cluster sums of Phase II (||Lloyd's per-thread
//                     centroids become per-CTA partials)
//   k_reduce          mergePtStructs: ordered FP64 reduction of the partials,
//                     new FP64 centroids and their FP32 scan copy
//   k_table           drift f(c) = d(c^t, c^{t-1}), the k x k table of
//                     1/2 d(c_a, c) and s(c) = 1/2 min_{c' != c} d(c, c')
//                     for the next iteration; iteration counters
// Distances are FP32 in the direct form sum_i (x_i - c_i)^2, accumulated in
// index order with one rounding per fma, so the dense and the pruned scan
// produce identical values; every MTI bound is rounded toward safety.
#include "knor_internal.cuh"
#include "device_common.cuh"

namespace knor {

constexpr int W = NT / 32;          // warps per CTA

__device__ __forceinline__ long long block_sum_ll(long long v, long long *scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < W; ++i) t += scratch[i];
    return t; // valid in thread 0
}

// Phase II for one tile of rows: add each row to its new cluster (tb) and,
// for MTI deltas, subtract it from its old one (ta).  Cluster c is owned by
// warp c % W, whose lanes walk the dimensions, so every (cluster, dim)
// accumulator is updated by one lane in a fixed order: the sums are
// deterministic.  Rows come from the shared tile (templated widths) or from
// global memory (generic width).
template <int DV>
__device__ __forceinline__ void accumulate(const IterParams &p, int nb, const int *tb, const int *ta,
                                           const int *ti, const float *tl, int64_t lo, float *acc_hi,
                                           float *acc_lo, int *cnt_s) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d = DV > 0 ? DV : p.d;
    for (int q0 = 0; q0 < nb; q0 += 32) {
        const int q = q0 + lane;
        const int cb = q < nb ? tb[q] : -1;
        const int ca = (ta != nullptr && q < nb) ? ta[q] : -1;
        unsigned m = __ballot_sync(FULL_MASK, cb >= 0 && (cb % W) == w);
        for (int pass = 0; pass < 2; ++pass) {
            const float sign = pass == 0 ? 1.0f : -1.0f;
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                const int qq = q0 + bit;
                const int c = __shfl_sync(FULL_MASK, pass == 0 ? cb : ca, bit);
                for (int j = lane; j < d; j += 32) {
                    float x;
                    if constexpr (DV > 0) x = tl[qq * p.dpad + j];
                    else x = p.X[(lo + ti[qq]) * d + j];
                    x = x * sign;
                    if (p.acc_global)
                        atomicAdd(&p.part_S[(size_t)(c * d + j) * p.part_stride], (double)x);
                    else
                        two_sum_acc(&acc_hi[c * d + j], &acc_lo[c * d + j], x);
                }
                if (lane == 0) {
                    if (p.acc_global)
                        atomicAdd(reinterpret_cast<unsigned long long *>(&p.part_cnt[(size_t)c * p.part_stride]),
                                  (unsigned long long)(pass == 0 ? 1LL : -1LL));
                    else
                        cnt_s[c] += pass == 0 ? 1 : -1;
                }
            }
            if (pass == 0) m = __ballot_sync(FULL_MASK, ca >= 0 && (ca % W) == w);
        }
    }
}

// Writes this CTA's partial sums (hi + lo in FP64) and counts to its slot.
__device__ __forceinline__ void flush_partials(const IterParams &p, const float *acc_hi,
                                               const float *acc_lo, const int *cnt_s) {
    if (p.acc_global) return;
    const int kd = p.k * p.d;
    for (int e = threadIdx.x; e < kd; e += NT)
        p.part_S[(size_t)e * p.part_stride + blockIdx.x] = (double)acc_hi[e] + (double)acc_lo[e];
    for (int c = threadIdx.x; c < p.k; c += NT)
        p.part_cnt[(size_t)c * p.part_stride + blockIdx.x] = cnt_s[c];
}

// --------------------------------------------------------------- dense scan

// Every point scans every centroid (plain Lloyd, and the first MTI iteration
// or a scheduled full recompute).  Row tiles stream into padded shared memory
// with cp.async (two stages in flight when they fit); each thread owns one
// point, keeps its row in registers and walks the centroids four at a time.
// Sums are rebuilt from scratch (fresh).
template <int DV>
__global__ void __launch_bounds__(NT) k_dense(const IterParams p, const int32_t *mode_dense,
                                              int32_t *nslots, int32_t *fresh) {
    if (*mode_dense == 0) return;
    extern __shared__ __align__(16) unsigned char sm[];
    float *acc_hi = reinterpret_cast<float *>(sm + p.off_acc_hi);
    float *acc_lo = reinterpret_cast<float *>(sm + p.off_acc_lo);
    int *cnt_s = reinterpret_cast<int *>(sm + p.off_cnt);
    float *F_s = reinterpret_cast<float *>(sm + p.off_F);
    int *tb = reinterpret_cast<int *>(sm + p.off_tb);
    int *ti = reinterpret_cast<int *>(sm + p.off_ti);
    float *tile = reinterpret_cast<float *>(sm + p.off_tile);
    long long *misc = reinterpret_cast<long long *>(sm + p.off_misc);
    const int tid = threadIdx.x;
    const int d = DV > 0 ? DV : p.d;
    const int k = p.k;
    const int kd = k * d;
    if (blockIdx.x == 0 && tid == 0) {
        *nslots = p.acc_global ? 1 : (int)gridDim.x;
        *fresh = 1;
    }
    if (!p.acc_global) {
        for (int e = tid; e < kd; e += NT) { acc_hi[e] = 0.0f; acc_lo[e] = 0.0f; }
        for (int c = tid; c < k; c += NT) cnt_s[c] = 0;
    }
    const float *cent = p.C32;
    if (p.cent_smem) {
        float *cs = reinterpret_cast<float *>(sm + p.off_cent);
        for (int e = tid; e < kd; e += NT) cs[e] = p.C32[e];
        cent = cs;
    }
    const float *Fp = p.F;
    if (p.off_F >= 0) {
        for (int c = tid; c < k; c += NT) F_s[c] = p.F[c];
        Fp = F_s;
    }
    int64_t lo, hi;
    block_range(p.n, 1, lo, hi);
    const int nbatch = (int)((hi - lo + NT - 1) / NT);
    long long my_changed = 0;

    auto load_tile = [&](int stage, int64_t base, int rows) {
        if constexpr (DV > 0) {
            constexpr int CH = DV / 4;
            float *dst = tile + (size_t)stage * NT * p.dpad;
            const float *src = p.X + base * DV;
            for (int f = tid; f < rows * CH; f += NT) {
                const int r = f / CH, ch = f % CH;
                cp_async16(dst + r * p.dpad + ch * 4, src + (size_t)r * DV + ch * 4);
            }
        }
        cp_async_commit();
    };

    __syncthreads();
    if (nbatch > 0) load_tile(0, lo, (int)(int)min((int64_t)NT, hi - lo));
    for (int b = 0; b < nbatch; ++b) {
        const int64_t base = lo + (int64_t)b * NT;
        const int rows = (int)min((int64_t)NT, hi - base);
        const int stage = p.stages == 2 ? (b & 1) : 0;
        if (p.stages == 2) {
            if (b + 1 < nbatch) {
                load_tile(stage ^ 1, base + NT, (int)min((int64_t)NT, hi - base - NT));
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
        } else {
            // one stage: this batch's rows, after the previous batch's
            // trailing barrier released the tile
            if (b > 0) load_tile(0, base, rows);
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *tl = tile + (size_t)stage * NT * p.dpad;
        int best = -1;
        if (tid < rows) {
            const int64_t i = base + tid;
            float bd = CUDART_INF_F;
            best = 0;
            if constexpr (DV > 0) {
                unsigned long long x[DV / 2];
                load_x2<DV>(x, tl + tid * p.dpad);
                int c = 0;
                for (; c + 4 <= k; c += 4) {
                    float r[4];
                    d2_regN<DV, 4>(x, cent + (size_t)c * DV, r);
                    if (r[0] < bd) { bd = r[0]; best = c; }
                    if (r[1] < bd) { bd = r[1]; best = c + 1; }
                    if (r[2] < bd) { bd = r[2]; best = c + 2; }
                    if (r[3] < bd) { bd = r[3]; best = c + 3; }
                }
                for (; c < k; ++c) {
                    const float r = d2_reg<DV>(x, cent + (size_t)c * DV);
                    if (r < bd) { bd = r; best = c; }
                }
            } else {
                const float *xg = p.X + i * d;
                for (int c = 0; c < k; ++c) {
                    const float r = d2_gen(xg, cent + (size_t)c * d, d);
                    if (r < bd) { bd = r; best = c; }
                }
            }
            const PtState old = p.st[i];
            my_changed += (old.a != best);
            PtState ns;
            ns.a = best;
            ns.ub = p.mti ? __fsub_ru(bound_up(bd, p.g_up, p.tiny), Fp[best]) : 0.0f;
            p.st[i] = ns;
        }
        tb[tid] = best;
        ti[tid] = (int)(base - lo) + tid;
        __syncthreads();
        accumulate<DV>(p, rows, tb, nullptr, ti, tl, lo, acc_hi, acc_lo, cnt_s);
        __syncthreads();
    }
    flush_partials(p, acc_hi, acc_lo, cnt_s);
    const long long tot = block_sum_ll(my_changed, misc);
    if (tid == 0) {
        atomicAdd(&p.ctr->changed, (unsigned long long)tot);
        atomicAdd(&p.ctr->evals, (unsigned long long)((hi - lo) * (int64_t)k));
    }
}

// ----------------------------------------------------------------- MTI scan

// Phase A (bound test, Clause 1) streams the packed per-point state of this
// CTA's range, PA points per thread; points that cannot be skipped go to a
// shared ring queue in point order.  Each full batch of NT queued points is
// scanned one point per thread (phase B: tighten u to the exact distance,
// Clause 3, then test every other centroid against 1/2 d(c_a, c), Clause 2)
// and the rows that changed cluster are moved between cluster sums
// (phase C, deltas).
template <int DV>
__global__ void __launch_bounds__(NT) k_mti(const IterParams p, const int32_t *mode_dense,
                                            int32_t *nslots, int32_t *fresh) {
    if (*mode_dense != 0) return;
    extern __shared__ __align__(16) unsigned char sm[];
    float *acc_hi = reinterpret_cast<float *>(sm + p.off_acc_hi);
    float *acc_lo = reinterpret_cast<float *>(sm + p.off_acc_lo);
    int *cnt_s = reinterpret_cast<int *>(sm + p.off_cnt);
    int *tb = reinterpret_cast<int *>(sm + p.off_tb);
    int *ta = reinterpret_cast<int *>(sm + p.off_ta);
    int *ti = reinterpret_cast<int *>(sm + p.off_ti);
    float *tile = reinterpret_cast<float *>(sm + p.off_tile);
    int2 *queue = reinterpret_cast<int2 *>(sm + p.off_queue);
    int *misc = reinterpret_cast<int *>(sm + p.off_misc);
    int *qhead = misc, *qlen = misc + 1, *wsum = misc + 2;
    long long *lscratch = reinterpret_cast<long long *>(misc + 16);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int d = DV > 0 ? DV : p.d;
    const int k = p.k;
    const int kd = k * d;
    if (blockIdx.x == 0 && tid == 0) {
        *nslots = p.acc_global ? 1 : (int)gridDim.x;
        *fresh = 0;
    }
    if (!p.acc_global) {
        for (int e = tid; e < kd; e += NT) { acc_hi[e] = 0.0f; acc_lo[e] = 0.0f; }
        for (int c = tid; c < k; c += NT) cnt_s[c] = 0;
    }
    const float *cent = p.C32;
    if (p.cent_smem) {
        float *cs = reinterpret_cast<float *>(sm + p.off_cent);
        for (int e = tid; e < kd; e += NT) cs[e] = p.C32[e];
        cent = cs;
    }
    const float *halfD = p.halfD;
    if (p.halfD_smem) {
        float *hs = reinterpret_cast<float *>(sm + p.off_halfD);
        for (int e = tid; e < k * k; e += NT) hs[e] = p.halfD[e];
        halfD = hs;
    }
    const float *s_s = p.s, *F_s = p.F;
    if (p.off_s >= 0) {
        float *a1 = reinterpret_cast<float *>(sm + p.off_s);
        float *a2 = reinterpret_cast<float *>(sm + p.off_F);
        for (int c = tid; c < k; c += NT) { a1[c] = p.s[c]; a2[c] = p.F[c]; }
        s_s = a1;
        F_s = a2;
    }
    if (tid == 0) { *qhead = 0; *qlen = 0; }
    int64_t lo, hi;
    block_range(p.n, PA, lo, hi);
    long long my_skipped = 0, my_evals = 0, my_changed = 0;
    __syncthreads();

    for (int64_t cbase = lo; cbase < hi; cbase += (int64_t)NT * PA) {
        // ---- phase A: Clause 1 on PA consecutive points per thread
        const int64_t i0 = cbase + (int64_t)tid * PA;
        PtState ps[PA];
        if (i0 + PA <= hi) {
            const int4 *src = reinterpret_cast<const int4 *>(p.st + i0);
#pragma unroll
            for (int v = 0; v < PA / 2; ++v) {
                const int4 q = src[v];
                ps[2 * v].ub = __int_as_float(q.x);
                ps[2 * v].a = q.y;
                ps[2 * v + 1].ub = __int_as_float(q.z);
                ps[2 * v + 1].a = q.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < PA; ++u) {
                if (i0 + u < hi) ps[u] = p.st[i0 + u];
                else { ps[u].ub = 0.0f; ps[u].a = -2; }
            }
        }
        unsigned amask = 0;
        int nvalid = 0;
#pragma unroll
        for (int u = 0; u < PA; ++u) {
            const int a = ps[u].a;
            if (a == -2) continue;
            ++nvalid;
            bool act = true;
            if (a >= 0) {
                // u^t = ub + F^t(a): the bound carried by the drift of c_a
                const float uu = __fadd_ru(ps[u].ub, F_s[a]);
                act = !(__fmaf_ru(uu, p.onepk, p.tau) < s_s[a]);
            }
            amask |= (act ? 1u : 0u) << u;
        }
        const int na = __popc(amask);
        my_skipped += nvalid - na;
        int incl = na;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        int wofs = 0, total = 0;
#pragma unroll
        for (int ww = 0; ww < W; ++ww) {
            const int v = wsum[ww];
            wofs += ww < w ? v : 0;
            total += v;
        }
        int pos = *qhead + *qlen + wofs + incl - na;
#pragma unroll
        for (int u = 0; u < PA; ++u) {
            if ((amask >> u) & 1u) {
                queue[pos % QCAP] = make_int2((int)(i0 + u - lo), ps[u].a);
                ++pos;
            }
        }
        __syncthreads();
        if (tid == 0) *qlen += total;
        __syncthreads();

        // ---- phases B and C on every full batch (and the rest at the end)
        const bool last = cbase + (int64_t)NT * PA >= hi;
        while (true) {
            const int ql = *qlen;
            if (!(ql >= NT || (last && ql > 0))) break;
            const int nb = min(NT, ql);
            const int h = *qhead;
            int tbv = -1, tav = -1;
            if (tid < nb) {
                const int2 e = queue[(h + tid) % QCAP];
                const int64_t i = lo + e.x;
                const int a = e.y;
                int best;
                float bd;
                if constexpr (DV > 0) {
                    unsigned long long x[DV / 2];
                    ldg_x2<DV>(x, p.X + i * DV);
                    if (a < 0) {
                        bd = CUDART_INF_F;
                        best = 0;
                        for (int c = 0; c < k; ++c) {
                            const float r = d2_reg<DV>(x, cent + (size_t)c * DV);
                            if (r < bd) { bd = r; best = c; }
                        }
                        my_evals += k;
                    } else {
                        // Clause 3: tighten u to (a bound on) the exact d(v, c_a)
                        bd = d2_reg<DV>(x, cent + (size_t)a * DV);
                        best = a;
                        ++my_evals;
                        const float test = __fmaf_ru(bound_up(bd, p.g_up, p.tiny), p.onepk, p.tau);
                        const float *hrow = halfD + (size_t)a * k;
                        for (int c = 0; c < k; ++c) {
                            if (c == a) continue;
                            if (test < hrow[c]) continue; // Clause 2: c cannot be nearer
                            const float r = d2_reg<DV>(x, cent + (size_t)c * DV);
                            ++my_evals;
                            if (r < bd || (r == bd && c < best)) { bd = r; best = c; }
                        }
                    }
                    if (best != a) {
                        float *dst = tile + tid * p.dpad;
                        const float4 *src = reinterpret_cast<const float4 *>(p.X + i * DV);
#pragma unroll
                        for (int j = 0; j < DV; j += 4) *reinterpret_cast<float4 *>(dst + j) = __ldg(src + j / 4);
                    }
                } else {
                    const float *xg = p.X + i * d;
                    if (a < 0) {
                        bd = CUDART_INF_F;
                        best = 0;
                        for (int c = 0; c < k; ++c) {
                            const float r = d2_gen(xg, cent + (size_t)c * d, d);
                            if (r < bd) { bd = r; best = c; }
                        }
                        my_evals += k;
                    } else {
                        bd = d2_gen(xg, cent + (size_t)a * d, d);
                        best = a;
                        ++my_evals;
                        const float test = __fmaf_ru(bound_up(bd, p.g_up, p.tiny), p.onepk, p.tau);
                        const float *hrow = halfD + (size_t)a * k;
                        for (int c = 0; c < k; ++c) {
                            if (c == a) continue;
                            if (test < hrow[c]) continue;
                            const float r = d2_gen(xg, cent + (size_t)c * d, d);
                            ++my_evals;
                            if (r < bd || (r == bd && c < best)) { bd = r; best = c; }
                        }
                    }
                }
                PtState ns;
                ns.a = best;
                ns.ub = __fsub_ru(bound_up(bd, p.g_up, p.tiny), F_s[best]);
                p.st[i] = ns;
                if (best != a) {
                    tbv = best;
                    tav = a;
                    ++my_changed;
                }
                ti[tid] = e.x;
            }
            tb[tid] = tbv;
            ta[tid] = tav;
            __syncthreads();
            accumulate<DV>(p, nb, tb, ta, ti, tile, lo, acc_hi, acc_lo, cnt_s);
            __syncthreads();
            if (tid == 0) {
                *qhead = (h + nb) % QCAP;
                *qlen = ql - nb;
            }
            __syncthreads();
        }
    }
    flush_partials(p, acc_hi, acc_lo, cnt_s);
    const long long t1 = block_sum_ll(my_changed, lscratch);
    const long long t2 = block_sum_ll(my_skipped, lscratch);
    const long long t3 = block_sum_ll(my_evals, lscratch);
    if (tid == 0) {
        atomicAdd(&p.ctr->changed, (unsigned long long)t1);
        atomicAdd(&p.ctr->skipped, (unsigned long long)t2);
        atomicAdd(&p.ctr->evals, (unsigned long long)t3);
    }
}

// ---------------------------------------------------------- reduce / table

// mergePtStructs: one warp per (cluster, dim) element adds the per-CTA
// partials in a fixed order (lane-strided, then a fixed butterfly), so the
// FP64 sums do not depend on scheduling.  Then c = S / count in FP64; an
// empty cluster keeps its centroid and its sum is reset to exactly zero.
__global__ void k_reduce(const FinParams f, const int32_t *nslots, const int32_t *fresh_flag) {
    const int kd = f.k * f.d;
    const int e = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= kd) return;
    const int c = e / f.d, j = e % f.d;
    const int G = *nslots;
    const int fresh = *fresh_flag;
    double sum = 0.0;
    long long cs = 0;
    for (int g = lane; g < G; g += 32) {
        sum += f.part_S[(size_t)e * f.part_stride + g];
        cs += f.part_cnt[(size_t)c * f.part_stride + g];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(FULL_MASK, sum, o);
        cs += __shfl_xor_sync(FULL_MASK, cs, o);
    }
    if (lane != 0) return;
    const long long cn = (fresh ? 0LL : f.cnt[c]) + cs;
    double Sn = fresh ? sum : f.S[e] + sum;
    double cv = f.C64[e];
    if (cn > 0) cv = Sn / (double)cn;
    else Sn = 0.0;
    f.S[e] = Sn;
    f.C64[e] = cv;
    f.C32n[e] = __double2float_rn(cv);
    if (j == 0) {
        f.cnt_next[c] = cn;
        if (cn == 0) atomicAdd(&f.ctr->empty, 1ULL);
    }
}

// Per centroid a (one CTA each), from the FP32 scan copies in FP64 with
// directed rounding: the drift f(a) = d(c^t_a, c^{t-1}_a) rounded up and
// added (rounded up) to the cumulative drift F(a); 1/2 d(c_a, c) rounded down
// for every c; s(a) their minimum over c != a.  Then the new copy replaces
// the old one.  CTA 0 records the iteration's counters and decides whether
// the device-side loop continues.
// k_mti_sel's heavy threshold of cluster a from row a of the k x k table:
// theta[a] = the th_M-th smallest 1/2 d(c_a, c) over c != a (equal values
// ranked by index), +inf when th_M > k - 1.  One CTA per row.
__device__ void theta_row(const FinParams &f, int a) {
    const int k = f.k;
    const float *row = f.halfD + (size_t)a * k;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (c == a) continue;
        const float h = row[c];
        int rank = 0;
        for (int q = 0; q < k; ++q) {
            const float g = row[q];
            rank += (q != a && (g < h || (g == h && q < c))) ? 1 : 0;
        }
        if (rank == f.th_M - 1) f.theta[a] = h;
    }
    if (threadIdx.x == 0 && f.th_M > k - 1) f.theta[a] = CUDART_INF_F;
}

__global__ void k_theta(const FinParams f) { theta_row(f, blockIdx.x); }

__global__ void k_table(const FinParams f, int32_t *mode_dense, int32_t need_table,
                        int32_t recompute_every, int32_t always_dense) {
    const int a = blockIdx.x, k = f.k, d = f.d, tid = threadIdx.x;
    __shared__ double red[128];
    __shared__ float redf[128];
    if (need_table) {
        double acc = 0.0;
        for (int j = tid; j < d; j += blockDim.x) {
            const double x = f.C32n[(size_t)a * d + j], y = f.C32[(size_t)a * d + j];
            const double lo = __dsub_rd(x, y), hi = __dsub_ru(x, y);
            const double m = fmax(fabs(lo), fabs(hi));
            acc = __dadd_ru(acc, __dmul_ru(m, m));
        }
        red[tid] = acc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int i = 0; i < (int)blockDim.x; ++i) t = __dadd_ru(t, red[i]);
            const float fa = __double2float_ru(__dsqrt_ru(t));
            f.F[a] = __fadd_ru(f.F[a], fa);
        }
        float mymin = CUDART_INF_F;
        for (int c = tid; c < k; c += blockDim.x) {
            if (c == a) { f.halfD[(size_t)a * k + c] = 0.0f; continue; }
            double sdd = 0.0;
            for (int j = 0; j < d; ++j) {
                const double x = f.C32n[(size_t)a * d + j], y = f.C32n[(size_t)c * d + j];
                const double lo = __dsub_rd(x, y), hi = __dsub_ru(x, y);
                const double m = lo > 0.0 ? lo : (hi < 0.0 ? -hi : 0.0);
                sdd = __dadd_rd(sdd, __dmul_rd(m, m));
            }
            const float h = __double2float_rd(__dmul_rd(0.5, __dsqrt_rd(sdd)));
            f.halfD[(size_t)a * k + c] = h;
            mymin = fminf(mymin, h);
        }
        redf[tid] = mymin;
        __syncthreads();
        if (tid == 0) {
            float m = CUDART_INF_F;
            for (int i = 0; i < (int)blockDim.x; ++i) m = fminf(m, redf[i]);
            f.s[a] = m;
        }
        if (f.theta != nullptr) {
            __syncthreads(); // row a of the table is written and visible to the CTA
            theta_row(f, a);
        }
    }
    __syncthreads();
    for (int j = tid; j < d; j += blockDim.x) f.C32[(size_t)a * d + j] = f.C32n[(size_t)a * d + j];
    if (tid == 0) f.cnt_out[a] = f.cnt_next[a];
    if (a == 0 && tid == 0 && f.snapshot) {
        const int it = *f.run_iter;
        const int total = *f.total_iter + 1;
        IterStats r;
        r.changed = (long long)f.ctr->changed;
        r.clause1_skipped = (long long)f.ctr->skipped;
        r.dist_evals = (long long)f.ctr->evals;
        r.rechecked = (long long)f.ctr->rechecked;
        r.empty = (int32_t)f.ctr->empty;
        r.iteration = total;
        r.violations = (long long)f.ctr->violations; // debug checks add theirs later
        f.stats[it] = r;
        *f.run_iter = it + 1;
        *f.total_iter = total;
        f.ctr->changed = 0; f.ctr->skipped = 0; f.ctr->evals = 0;
        f.ctr->rechecked = 0; f.ctr->empty = 0; f.ctr->violations = 0;
        *mode_dense = always_dense || (recompute_every > 0 && ((total + 1) % recompute_every) == 0);
        if (f.cond_handle) {
            const unsigned go = (r.changed != 0 && it + 1 < *f.max_iters_dev) ? 1u : 0u;
            cudaGraphSetConditional((cudaGraphConditionalHandle)f.cond_handle, go);
        }
    }
}

// ------------------------------------------------------------- utilities

__global__ void k_validate(const float *X, int64_t count, unsigned long long *bad) {
    unsigned long long nb = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = X[i];
        if (!(fabsf(v) <= 1e15f)) ++nb; // also catches NaN and +-inf
    }
    for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(FULL_MASK, nb, o);
    if ((threadIdx.x & 31) == 0 && nb) atomicAdd(bad, nb);
}

__global__ void k_init_state(PtState *st, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        PtState s;
        s.ub = CUDART_INF_F;
        s.a = -1;
        st[i] = s;
    }
}

__global__ void k_gather_rows(const float *X, int32_t d, const int64_t *idx, int32_t k, double *C64) {
    const int64_t total = (int64_t)k * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / d, j = e % d;
        C64[e] = (double)X[idx[c] * d + j];
    }
}

__global__ void k_round_c32(const double *C64, float *C32, int64_t kd) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < kd; e += (int64_t)gridDim.x * blockDim.x)
        C32[e] = __double2float_rn(C64[e]);
}

__global__ void k_extract_assign(const PtState *st, int64_t n, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = st[i].a;
}

// Debug invariant: u = ub + F[a] must be >= the exact distance to c_a.  The
// exact distance is bounded from below in FP64 with rounding toward -inf, so
// a reported violation is certain.
__global__ void k_check_bounds(const float *X, int64_t n, int32_t d, const PtState *st, const float *C32,
                               const float *F, IterStats *stats, const int32_t *run_iter) {
    unsigned long long bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const PtState s = st[i];
        if (s.a < 0) continue;
        const float u = __fadd_ru(s.ub, F[s.a]);
        double acc = 0.0;
        for (int j = 0; j < d; ++j) {
            const double x = X[i * d + j], y = C32[(size_t)s.a * d + j];
            const double lo = __dsub_rd(x, y), hi = __dsub_ru(x, y);
            const double m = lo > 0.0 ? lo : (hi < 0.0 ? -hi : 0.0);
            acc = __dadd_rd(acc, __dmul_rd(m, m));
        }
        if ((double)u < __dsqrt_rd(acc)) ++bad;
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(FULL_MASK, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) {
        const int it = *run_iter - 1;
        if (it >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(&stats[it].violations), bad);
    }
}

// ------------------------------------------------------------- launchers

int supported_dv(int d) {
    switch (d) {
    case 4: case 8: case 16: case 32: case 64: case 128: return d;
    default: return 0;
    }
}

#define KNOR_DV_SWITCH(dv, FN, ...)                      \
    switch (dv) {                                        \
    case 4: return FN<4>(__VA_ARGS__);                   \
    case 8: return FN<8>(__VA_ARGS__);                   \
    case 16: return FN<16>(__VA_ARGS__);                 \
    case 32: return FN<32>(__VA_ARGS__);                 \
    case 64: return FN<64>(__VA_ARGS__);                 \
    case 128: return FN<128>(__VA_ARGS__);               \
    default: return FN<0>(__VA_ARGS__);                  \
    }

template <int DV>
static cudaError_t dense_attr_t(size_t smem, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_dense<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_dense<DV>, NT, smem);
}
template <int DV>
static cudaError_t mti_attr_t(size_t smem, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_mti<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_mti<DV>, NT, smem);
}
template <int DV>
static cudaError_t dense_launch_t(const IterParams &p, int grid, size_t smem, cudaStream_t s,
                                  const int32_t *md, int32_t *ns, int32_t *fr) {
    k_dense<DV><<<grid, NT, smem, s>>>(p, md, ns, fr);
    return cudaGetLastError();
}
template <int DV>
static cudaError_t mti_launch_t(const IterParams &p, int grid, size_t smem, cudaStream_t s,
                                const int32_t *md, int32_t *ns, int32_t *fr) {
    k_mti<DV><<<grid, NT, smem, s>>>(p, md, ns, fr);
    return cudaGetLastError();
}

cudaError_t dense_attr(int dv, size_t smem, int *bps) { KNOR_DV_SWITCH(dv, dense_attr_t, smem, bps) }
cudaError_t mti_attr(int dv, size_t smem, int *bps) { KNOR_DV_SWITCH(dv, mti_attr_t, smem, bps) }
cudaError_t launch_dense(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                         const int32_t *md, int32_t *ns, int32_t *fr) {
    KNOR_DV_SWITCH(dv, dense_launch_t, p, grid, smem, s, md, ns, fr)
}
cudaError_t launch_mti(int dv, const IterParams &p, int grid, size_t smem, cudaStream_t s,
                       const int32_t *md, int32_t *ns, int32_t *fr) {
    KNOR_DV_SWITCH(dv, mti_launch_t, p, grid, smem, s, md, ns, fr)
}

cudaError_t launch_reduce(const FinParams &f, const int32_t *nslots, const int32_t *fresh, cudaStream_t s) {
    const int64_t threads = (int64_t)f.k * f.d * 32;
    const int blocks = (int)((threads + 255) / 256);
    k_reduce<<<blocks, 256, 0, s>>>(f, nslots, fresh);
    return cudaGetLastError();
}

cudaError_t launch_theta(const FinParams &f, cudaStream_t s) {
    if (f.theta == nullptr) return cudaSuccess;
    k_theta<<<f.k, 128, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_table(const FinParams &f, int32_t *mode_dense, int need_table, int recompute_every,
                         int always_dense, cudaStream_t s) {
    k_table<<<f.k, 128, 0, s>>>(f, mode_dense, need_table, recompute_every, always_dense);
    return cudaGetLastError();
}

static int grid_for(int64_t count, int threads) {
    int64_t b = (count + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65536) b = 65536;
    return (int)b;
}

cudaError_t launch_validate(const float *X, int64_t count, unsigned long long *bad, cudaStream_t s) {
    k_validate<<<grid_for(count, 256), 256, 0, s>>>(X, count, bad);
    return cudaGetLastError();
}
cudaError_t launch_init_state(PtState *st, int64_t n, cudaStream_t s) {
    k_init_state<<<grid_for(n, 256), 256, 0, s>>>(st, n);
    return cudaGetLastError();
}
cudaError_t launch_gather_rows(const float *X, int32_t d, const int64_t *idx, int32_t k, double *C64,
                               cudaStream_t s) {
    k_gather_rows<<<grid_for((int64_t)k * d, 256), 256, 0, s>>>(X, d, idx, k, C64);
    return cudaGetLastError();
}
cudaError_t launch_round_c32(const double *C64, float *C32, int64_t kd, cudaStream_t s) {
    k_round_c32<<<grid_for(kd, 256), 256, 0, s>>>(C64, C32, kd);
    return cudaGetLastError();
}
cudaError_t launch_extract_assign(const PtState *st, int64_t n, int32_t *out, cudaStream_t s) {
    k_extract_assign<<<grid_for(n, 256), 256, 0, s>>>(st, n, out);
    return cudaGetLastError();
}
cudaError_t launch_check_bounds(const float *X, int64_t n, int32_t d, const PtState *st, const float *C32,
                                const float *F, IterStats *stats, const int32_t *run_iter, cudaStream_t s) {
    k_check_bounds<<<grid_for(n, 256), 256, 0, s>>>(X, n, d, st, C32, F, stats, run_iter);
    return cudaGetLastError();
}

} // namespace knor

// precision.cu -- the precision forms of the assignment step (BF16 or FP16
// tensor cores with an exact FP32 recheck).
//
// The distance block d~^2(x, c) = ||x||^2 - 2 x~.c~ + ||c||^2 is formed with
// x~, c~ the 16-bit roundings of the FP32 point and centroid (FP16 operands
// are first scaled by powers of two into range): the dot products run on the
// 5th-generation tensor cores (tcgen05.mma, kind::f16, FP32 accumulation in
// tensor memory), fed by TMA tiles in 128-byte-swizzled shared memory.  The
// epilogue keeps each point's smallest and second smallest d~^2 over all
// centroids.  A point whose gap min2 - min1 exceeds 2 E(x) -- E(x) bounds the
// error of d~^2 plus the error of the library's FP32 distance
// (prec_error_constants below) -- provably has the same nearest centroid under
// the FP32 distance of the plain path.  The other points are gathered and run
// through the same kernel a second time, which records every centroid within
// min1 + 2 E(x) (a handful); those candidates are re-scored exactly in FP32
// (all k when more than seven per half were recorded).  The assignments are
// therefore identical to the plain FP32 path's.  The cluster sums are then
// updated by the deltas of the points that changed cluster.
//
// The paper has no GEMM path (its serial baseline table notes that GEMM codes
// were slower on its CPUs); this form is an addition for the tensor cores.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cmath>

#include "device_common.cuh"
#include "knor_internal.cuh"

namespace knor {

// ------------------------------------------------------------ primitives

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after about a second (or as
// soon as another role has flagged an error), sets *err and returns false.
// No wait in these kernels can spin forever.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int32_t *err) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*reinterpret_cast<volatile int32_t *>(err)) return false;
        if (clock64() - t0 > 2000000000LL) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int c0, int c1, uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored by TMA
// with 128-byte swizzling: rows of 128 bytes (64 BF16), 8-row atoms of 1024
// bytes.  Fields: start address >> 4 (bits 0-13), leading byte offset >> 4
// (16-29; unused for this layout, 1), stride byte offset >> 4 (32-45: 1024 B
// between 8-row atoms), the fixed descriptor version 0b001 (46-48), base
// offset 0 (atoms are 1024-aligned), layout type 2 = 128-byte swizzle (61-63).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B of one format (bits 7-9 and 10-12: 0 = FP16, 1 = BF16; the two
// must match), both K-major (15, 16 = 0), N >> 3 (17-22), M >> 4 (24-28).
__host__ __device__ constexpr uint32_t idesc_f16kind(int M, int N, uint32_t ab_format) {
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
// kind::f8f6f4 uses the same fields; A and B format 0 = E4M3.
__host__ __device__ constexpr uint32_t idesc_f8kind(int M, int N) { return idesc_f16kind(M, N, 0u); }

__device__ __forceinline__ void mma_f16kind(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}
__device__ __forceinline__ void mma_f8kind(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane (asynchronous: the
// registers are valid after tmem_wait_ld).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                   "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// After tmem_wait_ld: passes the 32 loaded registers through an (empty)
// volatile asm that follows the wait, so no instruction that reads them can
// be scheduled before the wait (the load's outputs are not yet valid there).
__device__ __forceinline__ void tmem_regs_ready(uint32_t *r) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])::"memory");
}

// (a * b + c) lane by lane for packed FP32 pairs, each lane rounded like the
// scalar fma.
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Two d~^2 - ||x||^2 values, of adjacent columns c0 and c0 + 1, into a
// (smallest m1, its index i1, second smallest m2) chain: the smaller of the
// two (ties: t0) is compared with m1, the larger can only become the new
// second smallest.  The result equals taking t0 and then t1 one at a time
// (m1 and i1 replaced on a strictly smaller value, m2 = min(m2, max(m1, t))).
__device__ __forceinline__ void top2_pair(float &m1, float &m2, int &i1, float t0, float t1, int c0) {
    const float lo = fminf(t0, t1), hi = fmaxf(t0, t1);
    const int ilo = t1 < t0 ? c0 + 1 : c0;
    m2 = fminf(fminf(m2, hi), fmaxf(m1, lo));
    if (lo < m1) i1 = ilo;
    m1 = fminf(m1, lo);
}
// Merges chain b into chain a.  On equal minima the merged second smallest
// equals the smallest: the gap is 0 and the point is never certified, so the
// index kept does not matter.
__device__ __forceinline__ void top2_merge(float &m1, float &m2, int &i1, float b1, float b2, int bi) {
    m2 = fminf(fminf(m2, b2), fmaxf(m1, b1));
    if (b1 < m1) { m1 = b1; i1 = bi; }
}

// 2E(x) for a point with ||x||^2 = xn and, in the space the operands are
// rounded in (FP8: x / sigma and c . sigma, per-dimension scales; else x and
// c), ||x'||^2 = xdn (see prec_error_constants); every operation rounded up.
// C bounds ||c||, Cd bounds ||c'||, zeta bounds ||c~' - c'||, Czd = Cd + zeta.
__device__ __forceinline__ float prec_two_e(float xn, float xdn, float C, float Cd, float zeta, float Czd,
                                            const PrecParams &p) {
    const float X = __fsqrt_ru(__fmul_ru(fmaxf(xn, 0.0f), 1.0000005f)); // covers the rounding of xn
    const float Xd = __fsqrt_ru(__fmul_ru(fmaxf(xdn, 0.0f), 1.0000005f));
    const float xi = __fmaf_ru(p.uq, Xd, p.eta_x);                       // bound on ||x~' - x'||
    const float Xx = __fadd_ru(Xd, xi);
    // |x'.c' - acc| <= ||x'|| zeta + xi (C' + zeta) + g_tc (X' + xi)(C' + zeta)
    const float etc = __fmaf_ru(Xd, zeta, __fmaf_ru(xi, Czd, __fmul_ru(p.gtc, __fmul_ru(Xx, Czd))));
    const float e32 = __fmaf_ru(p.eA32, __fmul_ru(Xx, Czd), __fmul_ru(p.eB, __fmaf_ru(X, X, __fmul_ru(C, C))));
    return __fmul_ru(2.0f, __fmaf_ru(2.02f, etc, e32));
}

// ---------------------------------------------------------------- layout

constexpr int TM = 128;              // points per tile (MMA M)
constexpr int TN = 256;              // centroids per chunk (MMA N)
// a TMA box row is 128 bytes: 64 16-bit or 128 FP8 elements (PrecParams tkb)
constexpr int A_BOX = TM * 128;      // bytes of one A box (16 KB)
constexpr int B_BOX = TN * 128;      // bytes of one B box (32 KB)
constexpr int EPI_WARPS = 8;         // two epilogue warps per TMEM lane quarter
constexpr int PREC_THREADS = 64 + 32 * EPI_WARPS; // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int HALF = TN / 2;         // columns of each chunk read by one epilogue warp
constexpr int TMEM_COLS = 2 * TN;    // two accumulator buffers
constexpr int NBARS = 21;            // mbarriers, see the kernel

size_t prec_smem_bytes(int d, int k, int esize) {
    const int nkc = d * esize / 128;
    const size_t kpad = (size_t)(k + TN - 1) / TN * TN;
    return 1024 /* alignment */ + 2 * (size_t)nkc * A_BOX + 2 * (size_t)nkc * B_BOX + kpad * 4 +
           3 * TM * 4 /* pair hand-off */ + NBARS * 8 + 16;
}

// ------------------------------------------------------------- the kernel

// Persistent: one CTA per SM walks point tiles blockIdx.x, +gridDim.x, ...;
// per tile, ceil(k / 256) centroid chunks.  Warp 0 (one lane) issues TMA
// loads of point tiles (two stages) and centroid chunks (two stages); warp 1
// allocates 512 TMEM columns and one lane issues the MMAs into two
// accumulator buffers; warps 2-9 read a finished buffer (one TMEM lane per
// point; the two warps of a lane quarter take one half of the columns each)
// while the next chunk is being multiplied.
__global__ void __launch_bounds__(PREC_THREADS, 1)
    k_tc_assign(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmC,
                  const PrecParams p) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int nkc = p.nkc;
    unsigned char *sA = sm;                                  // [2][nkc][A_BOX]
    unsigned char *sB = sA + 2 * (size_t)nkc * A_BOX;        // [2][nkc][B_BOX]
    const int nchunk = (p.k + TN - 1) / TN;
    float *cn_s = reinterpret_cast<float *>(sB + 2 * (size_t)nkc * B_BOX); // [nchunk * TN], +inf past k
    float *hand = cn_s + (size_t)nchunk * TN;                                // [3][TM] pair hand-off
    uint64_t *bars = reinterpret_cast<uint64_t *>(hand + 3 * TM);
    uint64_t *fullA = bars, *emptyA = bars + 2, *fullB = bars + 4, *emptyB = bars + 6;
    uint64_t *tfull = bars + 8, *tempty = bars + 10, *done = bars + 12;
    uint64_t *hfull = bars + 13, *hfree = bars + 17; // per lane quarter
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + NBARS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nrows = p.mode ? (int64_t)*p.rcount : p.n; // mode 1: the gathered points
    const int64_t ntile = (nrows + TM - 1) / TM;

    for (int c = threadIdx.x; c < nchunk * TN; c += PREC_THREADS) cn_s[c] = c < p.k ? p.cn[c] : CUDART_INF_F;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&fullA[i], 1);
            mbar_init(&emptyA[i], 1);
            mbar_init(&fullB[i], 1);
            mbar_init(&emptyB[i], 1);
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], EPI_WARPS); // one arrive per epilogue warp
        }
        mbar_init(done, 1);
        for (int i = 0; i < 4; ++i) {
            mbar_init(&hfull[i], 32); // every lane of the quarter's second warp
            mbar_init(&hfree[i], 32); // every lane of the quarter's first warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t *>(tmem_holder);

    // Ring bookkeeping: the u-th use of a ring slot waits for the (u-1)-th
    // completion of its "empty" barrier (parity (u-1)&1); the consumer's u-th
    // wait on a "full" barrier uses parity u&1.
    if (warp == 0) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            uint32_t ia = 0, ib = 0; // loads issued into ring A, ring B
            for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
                const int sa = ia & 1;
                if ((ia >> 1) >= 1 && !mbar_wait(&emptyA[sa], ((ia >> 1) - 1) & 1, p.err)) break;
                mbar_expect_tx(&fullA[sa], (uint32_t)(nkc * A_BOX));
                for (int kc = 0; kc < nkc; ++kc)
                    tma_load_2d(sA + ((size_t)sa * nkc + kc) * A_BOX, &tmX, kc * p.tkb, (int)(t * TM), &fullA[sa]);
                ++ia;
                bool ok = true;
                for (int j = 0; j < nchunk; ++j) {
                    const int sb = ib & 1;
                    if ((ib >> 1) >= 1 && !mbar_wait(&emptyB[sb], ((ib >> 1) - 1) & 1, p.err)) { ok = false; break; }
                    mbar_expect_tx(&fullB[sb], (uint32_t)(nkc * B_BOX));
                    for (int kc = 0; kc < nkc; ++kc)
                        tma_load_2d(sB + ((size_t)sb * nkc + kc) * B_BOX, &tmC, kc * p.tkb, j * TN, &fullB[sb]);
                    ++ib;
                }
                if (!ok) break;
            }
            // drain: the latest fill of each slot must land before the CTA exits
            for (uint32_t q = ia >= 2 ? ia - 2 : 0; q < ia; ++q) mbar_wait(&fullA[q & 1], (q >> 1) & 1, p.err);
            for (uint32_t q = ib >= 2 ? ib - 2 : 0; q < ib; ++q) mbar_wait(&fullB[q & 1], (q >> 1) & 1, p.err);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = p.idesc;
            uint32_t ca = 0, cb = 0, cbuf = 0; // consumed A fills, B fills, accumulators issued
            for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
                const int sa = ca & 1;
                if (!mbar_wait(&fullA[sa], (ca >> 1) & 1, p.err)) break;
                tc_fence_after();
                bool ok = true;
                for (int j = 0; j < nchunk; ++j) {
                    const int sb = cb & 1, buf = cbuf & 1;
                    if (!mbar_wait(&fullB[sb], (cb >> 1) & 1, p.err)) { ok = false; break; }
                    if ((cbuf >> 1) >= 1 && !mbar_wait(&tempty[buf], ((cbuf >> 1) - 1) & 1, p.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t dcol = tmem_base + (uint32_t)(buf * TN);
                    for (int kc = 0; kc < nkc; ++kc) {
                        const uint32_t a0 = smem_u32(sA + ((size_t)sa * nkc + kc) * A_BOX);
                        const uint32_t b0 = smem_u32(sB + ((size_t)sb * nkc + kc) * B_BOX);
                        // four MMAs per 128-byte chunk: K = 16 (16-bit) or 32
                        // (FP8) elements, 32 bytes each
                        for (int kk = 0; kk < 4; ++kk) {
                            if (p.fp8)
                                mma_f8kind(dcol, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc,
                                           (kc | kk) != 0 ? 1u : 0u);
                            else
                                mma_f16kind(dcol, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc,
                                            (kc | kk) != 0 ? 1u : 0u);
                        }
                    }
                    mma_commit(&emptyB[sb]); // B slot free once these MMAs are done
                    mma_commit(&tfull[buf]); // accumulator ready for the epilogue
                    ++cb;
                    ++cbuf;
                }
                if (!ok) break;
                mma_commit(&emptyA[sa]); // A slot free after the tile's last chunk
                ++ca;
            }
            // every MMA issued by this thread completes before TMEM is freed
            mma_commit(done);
            mbar_wait(done, 0, p.err);
        }
    } else {
        // -------------------------------------------------------- epilogue
        // Values compared: t(c) = ||c||^2 - 2 x~.c~ = d~^2 - ||x||^2 (||x||^2
        // is common to the row and cancels from every comparison).
        // Mode 0 (all points): the smallest t (m1, at i1) and the second
        // smallest (m2); a point is certified when m2 - m1 > 2E, else it is
        // listed with its m1.  Mode 1 (the listed points, gathered): every
        // centroid with t <= m1 + 2E is recorded.  Each t + ||x||^2 is within
        // E_tc of the exact d^2 and each FP32 distance within E_f (E = E_tc +
        // E_f), so the FP32 nearest centroid c* has t(c*) + ||x||^2 <= d32(c*)
        // + E <= d32(i1) + E <= m1 + ||x||^2 + 2E: it is always among the
        // candidates, whichever pass computed the two t values.
        const int q = warp & 3;          // TMEM lane quarter this warp may access
        const int h = (warp - 2) >> 2;   // which half of each chunk's columns
        const int rloc = 32 * q + lane;
        float *hm1 = hand, *hm2 = hand + TM;
        int *hi1 = reinterpret_cast<int *>(hand + 2 * TM);
        uint32_t cons = 0;  // accumulators consumed
        uint32_t tiles = 0; // tiles handed between the quarter's two warps
        const float C = p.it->cnorm_max;
        const float Cd = p.it->cdnorm_max;
        const float neg2inv = p.it->neg2inv;
        const float zeta = __fmaf_ru(p.uq, Cd, p.it->eta_c); // bound on ||c~' - c'||
        const float Czd = __fadd_ru(Cd, zeta);
        for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
            const int64_t row = t * TM + rloc;
            const bool valid = row < nrows;
            const float xn = valid ? (p.mode ? p.rxn[row] : p.xn[row]) : 0.0f;
            const float xdn = valid ? (p.mode ? p.rxdn[row] : p.xdn[row]) : 0.0f;
            const float twoE = prec_two_e(xn, xdn, C, Cd, zeta, Czd, p);
            // twoE = +inf (an unrepresentable scale) sends every point to the
            // full FP32 scan
            // rows past the end of the gathered list hold stale operands (any
            // value, inf included): a NaN threshold matches nothing there
            const float thr = (p.mode && valid) ? __fadd_ru(p.rm1[row], twoE) : CUDART_NAN_F;
            const bool all_cands = p.mode && !(twoE < CUDART_INF_F);
            // four independent chains (columns u mod 4) keep the dependent
            // min/max sequences short
            float a1[4], a2[4];
            int ai[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) { a1[j] = CUDART_INF_F; a2[j] = CUDART_INF_F; ai[j] = 0; }
            int nc = 0; // mode 1: candidates met in this warp's columns
            int32_t *cd = p.rcand + (size_t)(valid ? row : 0) * PREC_CANDS + h * (PREC_CANDS / 2); // valid rows only
            bool ok = true;
            for (int j = 0; j < nchunk; ++j) {
                // lane 0 waits, the warp follows its outcome (the TMEM loads
                // below are warp-synchronous)
                int okw = 1;
                if (lane == 0) okw = mbar_wait(&tfull[cons & 1], (cons >> 1) & 1, p.err) ? 1 : 0;
                okw = __shfl_sync(FULL_MASK, okw, 0);
                if (!okw) { ok = false; break; }
                tc_fence_after();
                const int buf = cons & 1;
                const uint32_t taddr =
                    tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * TN + h * HALF);
#pragma unroll 1
                for (int cc = 0; cc < HALF; cc += 64) {
                    uint32_t r[64];
                    tmem_ld32(taddr + (uint32_t)cc, r);
                    tmem_ld32(taddr + (uint32_t)cc + 32, r + 32);
                    tmem_wait_ld();
                    tmem_regs_ready(r);
                    tmem_regs_ready(r + 32);
                    const int cb = j * TN + h * HALF + cc;
                    const float4 *cn4 = reinterpret_cast<const float4 *>(cn_s + cb);
                    if (p.mode == 0) {
                        // t = acc (-2 / (s_x s_c)) + ||c||^2 for two columns per
                        // packed fma (each lane rounded like the scalar one);
                        // pairs of adjacent columns into the four chains in turn
                        const unsigned long long n2 = pack2(neg2inv, neg2inv);
#pragma unroll
                        for (int v = 0; v < 16; ++v) {
                            const float4 cv = cn4[v];
                            float t0, t1, t2, t3;
                            unpack2(fma2(pack2(__uint_as_float(r[4 * v + 0]), __uint_as_float(r[4 * v + 1])), n2,
                                         pack2(cv.x, cv.y)), t0, t1);
                            unpack2(fma2(pack2(__uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3])), n2,
                                         pack2(cv.z, cv.w)), t2, t3);
                            const int ch = 2 * (v & 1);
                            top2_pair(a1[ch], a2[ch], ai[ch], t0, t1, cb + 4 * v);
                            top2_pair(a1[ch + 1], a2[ch + 1], ai[ch + 1], t2, t3, cb + 4 * v + 2);
                        }
                    } else {
                        // bit u of (mlo, mhi): column cb + u is a candidate
                        uint32_t mlo = 0, mhi = 0;
#pragma unroll
                        for (int v = 0; v < 16; ++v) {
                            const float4 cv = cn4[v];
                            const float tv[4] = {__fmaf_rn(__uint_as_float(r[4 * v + 0]), neg2inv, cv.x),
                                                 __fmaf_rn(__uint_as_float(r[4 * v + 1]), neg2inv, cv.y),
                                                 __fmaf_rn(__uint_as_float(r[4 * v + 2]), neg2inv, cv.z),
                                                 __fmaf_rn(__uint_as_float(r[4 * v + 3]), neg2inv, cv.w)};
#pragma unroll
                            for (int w = 0; w < 4; ++w) {
                                const int u = 4 * v + w;
                                if (tv[w] <= thr) {
                                    if (u < 32) mlo |= 1u << u;
                                    else mhi |= 1u << (u - 32);
                                }
                            }
                        }
                        if (!valid) mlo = mhi = 0;
                        while (mlo | mhi) { // a few per point: record them in column order
                            int u;
                            if (mlo) { u = __ffs(mlo) - 1; mlo &= mlo - 1; }
                            else { u = 32 + __ffs(mhi) - 1; mhi &= mhi - 1; }
                            if (nc < PREC_CANDS / 2 - 1) cd[1 + nc] = cb + u;
                            ++nc;
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
                ++cons;
            }
            if (!ok) break;
            if (p.mode == 1) {
                if (valid) cd[0] = (nc < PREC_CANDS / 2 && !all_cands) ? nc : -1;
                continue;
            }
            float m1 = a1[0], m2 = a2[0];
            int i1 = ai[0];
#pragma unroll
            for (int j = 1; j < 4; ++j) top2_merge(m1, m2, i1, a1[j], a2[j], ai[j]);
            // the quarter's second warp hands its half to the first
            if (h == 1) {
                if (tiles > 0) {
                    int okw = 1;
                    if (lane == 0) okw = mbar_wait(&hfree[q], (tiles - 1) & 1, p.err) ? 1 : 0;
                    okw = __shfl_sync(FULL_MASK, okw, 0);
                    if (!okw) break;
                }
                hm1[rloc] = m1;
                hm2[rloc] = m2;
                hi1[rloc] = i1;
                mbar_arrive(&hfull[q]);
                ++tiles;
                continue;
            }
            {
                int okw = 1;
                if (lane == 0) okw = mbar_wait(&hfull[q], tiles & 1, p.err) ? 1 : 0;
                okw = __shfl_sync(FULL_MASK, okw, 0);
                if (!okw) break;
                __syncwarp();
            }
            top2_merge(m1, m2, i1, hm1[rloc], hm2[rloc], hi1[rloc]);
            mbar_arrive(&hfree[q]);
            ++tiles;
            // certified when the gap exceeds twice the error bound E(x)
            const bool cert = valid && __fsub_rd(m2, m1) > twoE;
            if (cert) p.a_next[row] = i1;
            const bool push = valid && !cert;
            const unsigned pm = __ballot_sync(FULL_MASK, push); // warp-aggregated append
            unsigned base = 0;
            if (pm) {
                if (lane == __ffs(pm) - 1) base = atomicAdd(p.rcount, (unsigned)__popc(pm));
                base = __shfl_sync(FULL_MASK, base, __ffs(pm) - 1);
            }
            if (push) {
                const unsigned slot = base + __popc(pm & ((1u << lane) - 1u));
                p.rlist[slot] = (int32_t)row;
                p.rm1[slot] = m1;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

// Exact FP32 re-score of the points the tensor-core pass could not certify,
// with the library's FP32 distance and lowest index on ties: one thread per
// point over its recorded candidates (two lists, one per half of the
// columns; four candidates at a time, the point row streamed through L1), or,
// when a list overflowed, one warp over all centroids.
template <int DV>
__global__ void __launch_bounds__(256) k_recheck(const float *X, const float *C32, int32_t k, const int32_t *rlist,
                                                 const int32_t *rcand, const unsigned *rcount, int32_t *a_next,
                                                 Counters *ctr) {
    constexpr int HC = PREC_CANDS / 2;
    const unsigned cnt = *rcount;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    unsigned long long evals = 0;
    for (int64_t e = gtid; e < cnt; e += nthreads) {
        const int32_t *cd = rcand + (size_t)e * PREC_CANDS;
        const int n0 = cd[0], n1 = cd[HC];
        // overflow (or, defensively, an empty list): scored by the warp pass below
        if (n0 < 0 || n1 < 0 || n0 + n1 == 0) continue;
        const int nc = n0 + n1;
        const int32_t i = rlist[e];
        const float *xr = X + (int64_t)i * DV;
        float bd = CUDART_INF_F;
        int best = 0x7fffffff;
        for (int qb = 0; qb < nc; qb += 4) {
            const float *cr[4];
            int cc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int t = qb + q < nc ? qb + q : qb; // padding repeats a candidate
                cc[q] = t < n0 ? cd[1 + t] : cd[HC + 1 + (t - n0)];
                cr[q] = C32 + (size_t)cc[q] * DV;
            }
            unsigned long long acc[4] = {0ULL, 0ULL, 0ULL, 0ULL};
#pragma unroll 8
            for (int j = 0; j < DV; j += 4) {
                const float4 xv = __ldg(reinterpret_cast<const float4 *>(xr + j));
                const unsigned long long xa = pack2(xv.x, xv.y), xb = pack2(xv.z, xv.w);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 v = __ldg(reinterpret_cast<const float4 *>(cr[q] + j));
                    acc[q] = sqacc2(sub2(xa, pack2(v.x, v.y)), acc[q]);
                    acc[q] = sqacc2(sub2(xb, pack2(v.z, v.w)), acc[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float r = fold2(acc[q]);
                if (r < bd || (r == bd && cc[q] < best)) { bd = r; best = cc[q]; }
            }
        }
        evals += nc;
        a_next[i] = best;
    }
    // points with too many candidates: one warp per point, lanes over centroids
    const int lane = threadIdx.x & 31;
    const int64_t wid = gtid >> 5, nw = nthreads >> 5;
    for (int64_t e = wid; e < cnt; e += nw) {
        const int n0 = rcand[(size_t)e * PREC_CANDS], n1 = rcand[(size_t)e * PREC_CANDS + HC];
        if (n0 >= 0 && n1 >= 0 && n0 + n1 > 0) continue;
        const float *xr = X + (int64_t)rlist[e] * DV; // the same row for every lane
        float bd = CUDART_INF_F;
        int best = 0x7fffffff;
        for (int c = lane; c < k; c += 32) {
            const float *cr = C32 + (size_t)c * DV;
            unsigned long long acc = 0ULL;
#pragma unroll 8
            for (int j = 0; j < DV; j += 4) {
                const float4 xv = __ldg(reinterpret_cast<const float4 *>(xr + j));
                const float4 v = __ldg(reinterpret_cast<const float4 *>(cr + j));
                acc = sqacc2(sub2(pack2(xv.x, xv.y), pack2(v.x, v.y)), acc);
                acc = sqacc2(sub2(pack2(xv.z, xv.w), pack2(v.z, v.w)), acc);
            }
            const float r = fold2(acc);
            if (r < bd) { bd = r; best = c; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(FULL_MASK, bd, o);
            const int oi = __shfl_xor_sync(FULL_MASK, best, o);
            if (ob < bd || (ob == bd && oi < best)) { bd = ob; best = oi; }
        }
        if (lane == 0) { a_next[rlist[e]] = best; evals += k; }
    }
    for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(FULL_MASK, evals, o);
    if (lane == 0 && evals) atomicAdd(&ctr->evals, evals);
    if (gtid == 0) atomicAdd(&ctr->rechecked, (unsigned long long)cnt);
}

// Debug invariant of the precision form: every new assignment equals the
// FP32 argmin over all centroids (library distance, lowest index on ties);
// each point that differs adds 1 to *viol.  O(n k d): debug runs only.
__global__ void k_prec_verify(const float *X, int64_t n, int32_t d, const float *C32, int32_t k,
                              const int32_t *a_next, unsigned long long *viol) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float bd = CUDART_INF_F;
        int best = 0;
        for (int c = 0; c < k; ++c) {
            const float r = d2_gen(X + i * d, C32 + (size_t)c * d, d);
            if (r < bd) { bd = r; best = c; }
        }
        if (best != a_next[i]) atomicAdd(viol, 1ULL);
    }
}

// Gathers the operand rows (ROWB bytes each) and ||x||^2, ||x'||^2 of the
// listed points into a compact matrix for the candidate pass: one warp per
// point, 16 bytes per lane.
template <int ROWB>
__global__ void k_prec_gather(const unsigned char *Xb, const float *xn, const float *xdn, const int32_t *rlist,
                              const unsigned *rcount, unsigned char *Xc, float *rxn, float *rxdn) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned cnt = *rcount;
    constexpr int V = ROWB / 16; // 16-byte vectors per row
    for (int64_t e = wid; e < cnt; e += nw) {
        const int32_t i = rlist[e];
        if (lane < V)
            reinterpret_cast<int4 *>(Xc + (size_t)e * ROWB)[lane] =
                reinterpret_cast<const int4 *>(Xb + (size_t)i * ROWB)[lane];
        if (lane == 0) {
            rxn[e] = xn[i];
            rxdn[e] = xdn[i];
        }
    }
}

// Commits the new assignments and moves the rows that changed cluster
// between the sums (FP64 atomics into partial slot 0): one warp per 32
// points, lanes over dimensions.
__global__ void k_delta_sums(const float *X, int64_t n, int32_t d, PtState *st, const int32_t *a_next,
                             double *S, long long *cnt, Counters *ctr, int32_t k, int32_t *nslots,
                             int32_t *fresh) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *nslots = 1;
        *fresh = 0;
        atomicAdd(&ctr->evals, (unsigned long long)n * (unsigned long long)k); // the tensor-core scan
    }
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long changed = 0;
    for (int64_t base = wid * 32; base < n; base += nw * 32) {
        const int64_t i = base + lane;
        int anew = -1, aold = -1;
        bool ch = false;
        if (i < n) {
            anew = a_next[i];
            PtState s = st[i];
            aold = s.a;
            if (anew < 0 || anew >= k) {
                // no assignment was produced for this point (a library bug):
                // count it, keep the old one, touch no sums
                atomicAdd(&ctr->violations, 1ULL);
                anew = aold;
            }
            ch = aold != anew;
            if (ch) { s.a = anew; st[i] = s; }
        }
        unsigned m = __ballot_sync(FULL_MASK, ch);
        changed += __popc(m);
        while (m) {
            const int pl = __ffs(m) - 1;
            m &= m - 1;
            const int64_t ip = base + pl;
            const int cn = __shfl_sync(FULL_MASK, anew, pl);
            const int co = __shfl_sync(FULL_MASK, aold, pl);
            for (int j = lane; j < d; j += 32) {
                const double x = (double)X[ip * d + j];
                atomicAdd(&S[(size_t)cn * d + j], x);
                if (co >= 0) atomicAdd(&S[(size_t)co * d + j], -x);
            }
            if (lane == 0) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[cn]), 1ULL);
                if (co >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[co]), (unsigned long long)-1LL);
            }
        }
    }
    if (lane == 0 && changed) atomicAdd(&ctr->changed, changed);
}

// Storage of one operand of format FMT.
template <int FMT> struct OpT { using T = uint16_t; };
template <> struct OpT<PREC_FMT_FP8> { using T = uint8_t; };

template <int FMT>
__device__ __forceinline__ typename OpT<FMT>::T to_op(float v) {
    if constexpr (FMT == PREC_FMT_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    else if constexpr (FMT == PREC_FMT_FP16) return __half_as_ushort(__float2half_rn(v));
    else return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3); // never saturates: |v| <= 2^7
}

// Exponent e of the scale 2^e of an operand: the largest with absmax * 2^e
// <= 2^15 (FP16, half its range) or 2^7 (FP8 e4m3, whose largest value is
// 448), clamped to [-60, 60].  BF16 has the FP32 exponent range and is not
// scaled.
__host__ __device__ inline int scale_exp(int32_t fmt, float absmax) {
    if (fmt == PREC_FMT_BF16) return 0;
    if (!(absmax > 0.0f)) return 60;
    int ex;
    const float m = frexpf(absmax, &ex); // absmax = m 2^ex, m in [0.5, 1)
    const int cl = (m == 0.5f) ? ex - 1 : ex; // ceil(log2(absmax))
    const int e = (fmt == PREC_FMT_FP8 ? 7 : 15) - cl;
    return e < -60 ? -60 : (e > 60 ? 60 : e);
}

// Absolute error of one rounded scaled coordinate (half the smallest
// subnormal, with a factor 2 of margin): FP16 2^-24, FP8 e4m3 2^-9; for BF16
// anything above half its smallest subnormal (2^-134).
__host__ __device__ inline double op_eta(int32_t fmt) {
    return fmt == PREC_FMT_BF16 ? 0x1p-100 : (fmt == PREC_FMT_FP16 ? 0x1p-24 : 0x1p-9);
}

// Per iteration, step 1: ||c||^2 (FP64 sum of the FP32 values, rounded to
// nearest), max ||c|| (rounded up), and with the per-dimension scales sigma
// (FP8; NULL = 1) max ||c . sigma|| and max |c_j sigma_j|; one CTA per centroid.
__global__ void k_prec_cnorm(const float *C32, int32_t d, const float *sigma, float *cn, PrecIter *it) {
    const int c = blockIdx.x;
    __shared__ double red[128], redd[128];
    __shared__ float amax[128];
    double acc = 0.0, accd = 0.0;
    float am = 0.0f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float v = C32[(size_t)c * d + j];
        const float vd = sigma ? v * sigma[j] : v; // a power of two: exact
        acc += (double)v * (double)v;
        accd += (double)vd * (double)vd;
        am = fmaxf(am, fabsf(vd));
    }
    red[threadIdx.x] = acc;
    redd[threadIdx.x] = accd;
    amax[threadIdx.x] = am;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, td = 0.0;
        float m = 0.0f;
        for (int i = 0; i < (int)blockDim.x; ++i) { t += red[i]; td += redd[i]; m = fmaxf(m, amax[i]); }
        cn[c] = __double2float_rn(t);
        const float nrm = __double2float_ru(__dsqrt_ru(__dmul_ru(t, 1.0 + 1e-15)));
        const float nrmd = __double2float_ru(__dsqrt_ru(__dmul_ru(td, 1.0 + 1e-15)));
        // non-negative floats order as ints
        atomicMax(reinterpret_cast<int *>(&it->cnorm_max), __float_as_int(nrm));
        atomicMax(reinterpret_cast<int *>(&it->cdnorm_max), __float_as_int(nrmd));
        atomicMax(reinterpret_cast<int *>(&it->cabs_max), __float_as_int(m));
    }
}

// Per iteration, step 2: the scaled, rounded centroids c~' = fmt(c . sigma
// s_c), and (block 0) the scale-dependent constants.
template <int FMT>
__global__ void k_prec_conv(const float *C32, int64_t kd, int32_t d, float sx, const float *sigma,
                            typename OpT<FMT>::T *Cb, PrecIter *it) {
    const float M = it->cabs_max;
    const int ec = scale_exp(FMT, M);
    const float sc = ldexpf(1.0f, ec);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < kd; i += (int64_t)gridDim.x * blockDim.x)
        Cb[i] = to_op<FMT>(C32[i] * (sigma ? sigma[i % d] : 1.0f) * sc); // powers of two: exact
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int ex;
        frexpf(sx, &ex); // sx = 2^(ex - 1)
        it->neg2inv = ldexpf(-2.0f, -(ex - 1) - ec);
        float ec_bound = __double2float_ru(sqrt((double)d) * 1.000001 * op_eta(FMT) * ldexp(1.0, -ec));
        const float lim = FMT == PREC_FMT_FP8 ? 128.0f : 32768.0f;
        if (FMT != PREC_FMT_BF16 && !(M * sc <= lim)) ec_bound = CUDART_INF_F; // unrepresentable
        it->eta_c = ec_bound;
    }
}

// Largest |x_j| over the points (once per context, for the point scale).
__global__ void k_prec_absmax(const float *X, int64_t count, float *out) {
    float m = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(X[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));
}

// Largest |x_ij| per dimension j (FP8 per-dimension scales).
__global__ void k_prec_dim_absmax(const float *X, int64_t n, int32_t d, float *out) {
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        float m = 0.0f;
        for (int64_t i = blockIdx.x; i < n; i += gridDim.x) m = fmaxf(m, fabsf(X[i * d + j]));
        atomicMax(reinterpret_cast<int *>(out + j), __float_as_int(m));
    }
}

// Once per context: scaled, rounded points x~' = fmt(x / sigma s_x),
// ||x||^2 and ||x / sigma||^2 (FP64 sums, rounded to nearest).
template <int FMT>
__global__ void k_prec_points(const float *X, int64_t n, int32_t d, float sx, const float *sigma_inv,
                              typename OpT<FMT>::T *Xb, float *xn, float *xdn) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < n; i += nw) {
        double acc = 0.0, accd = 0.0;
        for (int j = lane; j < d; j += 32) {
            const float v = X[i * d + j];
            const float vd = sigma_inv ? v * sigma_inv[j] : v; // a power of two: exact
            Xb[i * d + j] = to_op<FMT>(vd * sx);
            acc += (double)v * (double)v;
            accd += (double)vd * (double)vd;
        }
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(FULL_MASK, acc, o);
            accd += __shfl_xor_sync(FULL_MASK, accd, o);
        }
        if (lane == 0) {
            xn[i] = __double2float_rn(acc);
            if (xdn != xn) xdn[i] = __double2float_rn(accd);
        }
    }
}

// ------------------------------------------------------------- launchers

// Constants of the certification bound.  With x', c' the vectors in the
// space the operands are rounded in (FP8: x / sigma and c . sigma with
// power-of-two per-dimension scales sigma, so that x'.c' = x.c; else x and
// c), x~', c~' the operands the tensor cores see (unscaled), u_q the unit
// roundoff of the format (BF16 2^-8, FP16 2^-11, FP8 e4m3 2^-4) and eta the
// absolute error of a rounded scaled coordinate (subnormals):
//   ||x~' - x'|| <= xi = u_q ||x'|| + sqrt(d) eta / s_x,  ||c~' - c'|| <= zeta
//   |x.c - x~'.c~'| <= ||x'|| zeta + xi (||c'|| + zeta)
//   tensor-core FP32 accumulation of d products: at most g_tc ||x~'|| ||c~'||
//     with g_tc = 2d 2^-23 / (1 - 2d 2^-23) for 16-bit operands (truncating
//     adds, a factor 2), 2d 2^-16 / (1 - 2d 2^-16) for FP8 (no accumulator
//     width is assumed beyond 17 bits)
//   epilogue t = fma(acc, -2/(s_x s_c), ||c||^2): ||c||^2 rounded once and
//     the fma once, <= u (||c||^2 + |t|) <= 2u ||x~'|| ||c~'|| + 2u ||c||^2
//   FP32 distance of the plain path: relative (d + 2) u / (1 - (d + 2) u)
//     of d^2 <= 2 (||x||^2 + ||c||^2)
// with u = 2^-24.  E = 2 (1.01) (dot error + accumulation) + eA32 ||x~'||
// ||c~'|| + eB (||x||^2 + ||c||^2), eA32 = 1.01 (2u), eB = 1.01 (3u + 2 g_d),
// each rounded up (prec_two_e evaluates it per point).
void prec_error_constants(int32_t fmt, int d, float sx, PrecParams &p) {
    const double u = std::ldexp(1.0, -24);
    const double ua = fmt == PREC_FMT_FP8 ? std::ldexp(1.0, -16) : std::ldexp(1.0, -23);
    const double gtc = 2.0 * d * ua / (1.0 - 2.0 * d * ua);
    const double g = (d + 2) * u / (1.0 - (d + 2) * u);
    p.uq = fmt == PREC_FMT_BF16 ? std::ldexp(1.0f, -8) : (fmt == PREC_FMT_FP16 ? std::ldexp(1.0f, -11)
                                                                               : std::ldexp(1.0f, -4));
    p.gtc = std::nextafter((float)gtc, INFINITY);
    p.eta_x = std::nextafter((float)(std::sqrt((double)d) * 1.000001 * op_eta(fmt) / sx), INFINITY);
    p.eA32 = std::nextafter((float)(1.01 * 2 * u), INFINITY);
    p.eB = std::nextafter((float)(1.01 * (3 * u + 2 * g)), INFINITY);
    p.idesc = fmt == PREC_FMT_FP8 ? idesc_f8kind(TM, TN) : idesc_f16kind(TM, TN, fmt == PREC_FMT_BF16 ? 1u : 0u);
    p.fp8 = fmt == PREC_FMT_FP8 ? 1 : 0;
    const int esize = fmt == PREC_FMT_FP8 ? 1 : 2;
    p.nkc = d * esize / 128;
    p.tkb = 128 / esize;
}

int prec_point_scale_exp(int32_t fmt, float absmax) { return scale_exp(fmt, absmax); }

cudaError_t prec_absmax(const float *X, int64_t count, float *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    k_prec_absmax<<<1024, 256, 0, s>>>(X, count, out);
    return cudaGetLastError();
}

cudaError_t prec_dim_absmax(const float *X, int64_t n, int32_t d, float *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * d, s);
    if (e != cudaSuccess) return e;
    k_prec_dim_absmax<<<1024, 128, 0, s>>>(X, n, d, out);
    return cudaGetLastError();
}

cudaError_t prec_points(const float *X, int64_t n, int32_t d, int32_t fmt, float sx, const float *sigma_inv,
                        void *Xb, float *xn, float *xdn, cudaStream_t s) {
    if (fmt == PREC_FMT_BF16)
        k_prec_points<PREC_FMT_BF16><<<1024, 256, 0, s>>>(X, n, d, sx, nullptr, static_cast<uint16_t *>(Xb), xn, xn);
    else if (fmt == PREC_FMT_FP16)
        k_prec_points<PREC_FMT_FP16><<<1024, 256, 0, s>>>(X, n, d, sx, nullptr, static_cast<uint16_t *>(Xb), xn, xn);
    else
        k_prec_points<PREC_FMT_FP8><<<1024, 256, 0, s>>>(X, n, d, sx, sigma_inv, static_cast<uint8_t *>(Xb), xn,
                                                         xdn);
    return cudaGetLastError();
}

cudaError_t prec_prep(const float *C32, int32_t k, int32_t d, int32_t fmt, float sx, const float *sigma, void *Cb,
                      float *cn, PrecIter *it, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(it, 0, sizeof(PrecIter), s);
    if (e != cudaSuccess) return e;
    const float *sg = fmt == PREC_FMT_FP8 ? sigma : nullptr;
    k_prec_cnorm<<<k, 128, 0, s>>>(C32, d, sg, cn, it);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t kd = (int64_t)k * d;
    const int grid = (int)std::min<int64_t>((kd + 255) / 256, 1024);
    if (fmt == PREC_FMT_BF16)
        k_prec_conv<PREC_FMT_BF16><<<grid, 256, 0, s>>>(C32, kd, d, sx, nullptr, static_cast<uint16_t *>(Cb), it);
    else if (fmt == PREC_FMT_FP16)
        k_prec_conv<PREC_FMT_FP16><<<grid, 256, 0, s>>>(C32, kd, d, sx, nullptr, static_cast<uint16_t *>(Cb), it);
    else
        k_prec_conv<PREC_FMT_FP8><<<grid, 256, 0, s>>>(C32, kd, d, sx, sg, static_cast<uint8_t *>(Cb), it);
    return cudaGetLastError();
}

cudaError_t prec_assign_attr(size_t smem) {
    return cudaFuncSetAttribute(k_tc_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t prec_assign_maps(const CUtensorMap &tmX, const CUtensorMap &tmC, const PrecParams &p, int grid, size_t smem, cudaStream_t s);
cudaError_t prec_assign(const void *tmX, const void *tmC, const PrecParams &p, int grid, size_t smem,
                        cudaStream_t s) {
    return prec_assign_maps(*static_cast<const CUtensorMap *>(tmX), *static_cast<const CUtensorMap *>(tmC), p, grid,
                            smem, s);
}

cudaError_t prec_assign_maps(const CUtensorMap &tmX, const CUtensorMap &tmC, const PrecParams &p, int grid,
                             size_t smem, cudaStream_t s) {
    k_tc_assign<<<grid, PREC_THREADS, smem, s>>>(tmX, tmC, p);
    return cudaGetLastError();
}

cudaError_t prec_recheck(int dv, const float *X, const float *C32, int32_t k, const int32_t *rlist,
                         const int32_t *rcand, const unsigned *rcount, int32_t *a_next, Counters *ctr, int grid,
                         cudaStream_t s) {
    switch (dv) {
    case 64: k_recheck<64><<<grid, 256, 0, s>>>(X, C32, k, rlist, rcand, rcount, a_next, ctr); break;
    case 128: k_recheck<128><<<grid, 256, 0, s>>>(X, C32, k, rlist, rcand, rcount, a_next, ctr); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t prec_gather(int row_bytes, const void *Xb, const float *xn, const float *xdn, const int32_t *rlist,
                        const unsigned *rcount, void *Xc, float *rxn, float *rxdn, int grid, cudaStream_t s) {
    const unsigned char *a = static_cast<const unsigned char *>(Xb);
    unsigned char *b = static_cast<unsigned char *>(Xc);
    switch (row_bytes) {
    case 128: k_prec_gather<128><<<grid, 256, 0, s>>>(a, xn, xdn, rlist, rcount, b, rxn, rxdn); break;
    case 256: k_prec_gather<256><<<grid, 256, 0, s>>>(a, xn, xdn, rlist, rcount, b, rxn, rxdn); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t prec_verify(const float *X, int64_t n, int32_t d, const float *C32, int32_t k, const int32_t *a_next,
                        unsigned long long *viol, cudaStream_t s) {
    k_prec_verify<<<1024, 128, 0, s>>>(X, n, d, C32, k, a_next, viol);
    return cudaGetLastError();
}

cudaError_t prec_delta_sums(const float *X, int64_t n, int32_t d, PtState *st, const int32_t *a_next, double *S,
                            long long *cnt, Counters *ctr, int32_t k, int32_t *nslots, int32_t *fresh, int grid,
                            cudaStream_t s) {
    k_delta_sums<<<grid, 256, 0, s>>>(X, n, d, st, a_next, S, cnt, ctr, k, nslots, fresh);
    return cudaGetLastError();
}

} // namespace knor

// device_common.cuh -- device helpers shared by the point kernels of
// libknor.so (distance, error bound, TwoSum, cp.async).
#pragma once

#include <math_constants.h>

#include "knor_internal.cuh"

namespace knor {

#define FULL_MASK 0xffffffffu

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The FP32 squared distance used by every scan of this library:
//   e = sum over even j, o = sum over odd j (each in increasing j, each term
//   t_j = x_j - c_j rounded, then e or o = fma(t_j, t_j, e or o) rounded),
//   d^2 = e + o rounded.
// Even and odd dimensions sit side by side in one 64-bit register, so a
// packed sub.rn.f32x2 / fma.rn.f32x2 does a step of both chains; every lane
// of a packed op rounds exactly like the scalar op.  Relative error of d^2:
// at most ceil(d/2) + 2 roundings on each chain plus the final add, within
// (1 - (d + 2) 2^-24)^-1 - 1 (see bound_up).

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long sqacc2(unsigned long long t, unsigned long long acc) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(t), "l"(acc));
    return r;
}
__device__ __forceinline__ float fold2(unsigned long long acc) {
    float e, o;
    unpack2(acc, e, o);
    return __fadd_rn(e, o);
}

// Point as DV/2 packed (x_j, x_{j+1}) pairs, from a 16-byte-aligned row.
template <int DV>
__device__ __forceinline__ void load_x2(unsigned long long (&x2)[DV / 2], const float *row) {
#pragma unroll
    for (int j = 0; j < DV; j += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(row + j);
        x2[j / 2] = pack2(v.x, v.y);
        x2[j / 2 + 1] = pack2(v.z, v.w);
    }
}
template <int DV>
__device__ __forceinline__ void ldg_x2(unsigned long long (&x2)[DV / 2], const float *row) {
#pragma unroll
    for (int j = 0; j < DV; j += 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(row + j));
        x2[j / 2] = pack2(v.x, v.y);
        x2[j / 2 + 1] = pack2(v.z, v.w);
    }
}

// The same for rows read once: not kept in L1 (which then holds the data
// that is reused, such as centroids and table rows).
template <int DV>
__device__ __forceinline__ void ldg_x2_stream(unsigned long long (&x2)[DV / 2], const float *row) {
#pragma unroll
    for (int j = 0; j < DV; j += 4) {
        float v0, v1, v2, v3;
        asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v0), "=f"(v1), "=f"(v2), "=f"(v3)
                     : "l"(row + j));
        x2[j / 2] = pack2(v0, v1);
        x2[j / 2 + 1] = pack2(v2, v3);
    }
}

// The same from a 32-byte-aligned row (DV a multiple of 8) with 32-byte
// loads: one request per lane and sector, where 16-byte loads take two.
template <int DV>
__device__ __forceinline__ void ldg_x2_w32(unsigned long long (&x2)[DV / 2], const float *row) {
    static_assert(DV % 8 == 0, "32-byte row loads need DV % 8 == 0");
#pragma unroll
    for (int j = 0; j < DV; j += 8) {
        float v0, v1, v2, v3, v4, v5, v6, v7;
        asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(v0), "=f"(v1), "=f"(v2), "=f"(v3), "=f"(v4), "=f"(v5), "=f"(v6), "=f"(v7)
                     : "l"(row + j));
        x2[j / 2] = pack2(v0, v1);
        x2[j / 2 + 1] = pack2(v2, v3);
        x2[j / 2 + 2] = pack2(v4, v5);
        x2[j / 2 + 3] = pack2(v6, v7);
    }
}

// d^2 to one centroid (16-byte aligned, smem or global).
template <int DV>
__device__ __forceinline__ float d2_reg(const unsigned long long (&x2)[DV / 2], const float *c) {
    unsigned long long acc = 0ULL; // (+0, +0)
#pragma unroll
    for (int j = 0; j < DV; j += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(c + j);
        acc = sqacc2(sub2(x2[j / 2], pack2(v.x, v.y)), acc);
        acc = sqacc2(sub2(x2[j / 2 + 1], pack2(v.z, v.w)), acc);
    }
    return fold2(acc);
}

// d^2 to NC consecutive centroids at once (independent chains, same values).
template <int DV, int NC>
__device__ __forceinline__ void d2_regN(const unsigned long long (&x2)[DV / 2], const float *c, float (&r)[NC]) {
    unsigned long long acc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = 0ULL;
#pragma unroll
    for (int j = 0; j < DV; j += 4) {
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const float4 v = *reinterpret_cast<const float4 *>(c + (size_t)q * DV + j);
            acc[q] = sqacc2(sub2(x2[j / 2], pack2(v.x, v.y)), acc[q]);
            acc[q] = sqacc2(sub2(x2[j / 2 + 1], pack2(v.z, v.w)), acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) r[q] = fold2(acc[q]);
}

// d^2 to two centroids anywhere (independent chains, same values as d2_reg).
template <int DV>
__device__ __forceinline__ void d2_reg2(const unsigned long long (&x2)[DV / 2], const float *c0, const float *c1,
                                        float &r0, float &r1) {
    unsigned long long a0 = 0ULL, a1 = 0ULL;
#pragma unroll
    for (int j = 0; j < DV; j += 4) {
        const float4 v0 = *reinterpret_cast<const float4 *>(c0 + j);
        const float4 v1 = *reinterpret_cast<const float4 *>(c1 + j);
        a0 = sqacc2(sub2(x2[j / 2], pack2(v0.x, v0.y)), a0);
        a1 = sqacc2(sub2(x2[j / 2], pack2(v1.x, v1.y)), a1);
        a0 = sqacc2(sub2(x2[j / 2 + 1], pack2(v0.z, v0.w)), a0);
        a1 = sqacc2(sub2(x2[j / 2 + 1], pack2(v1.z, v1.w)), a1);
    }
    r0 = fold2(a0);
    r1 = fold2(a1);
}

// d^2 to four centroids anywhere (independent chains, same values as d2_reg).
template <int DV>
__device__ __forceinline__ void d2_reg4(const unsigned long long (&x2)[DV / 2], const float *c0, const float *c1,
                                        const float *c2, const float *c3, float (&r)[4]) {
    const float *cs[4] = {c0, c1, c2, c3};
    unsigned long long acc[4] = {0ULL, 0ULL, 0ULL, 0ULL};
#pragma unroll
    for (int j = 0; j < DV; j += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = *reinterpret_cast<const float4 *>(cs[q] + j);
            acc[q] = sqacc2(sub2(x2[j / 2], pack2(v.x, v.y)), acc[q]);
            acc[q] = sqacc2(sub2(x2[j / 2 + 1], pack2(v.z, v.w)), acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) r[q] = fold2(acc[q]);
}

// Generic width: the same definition with scalar operations and a runtime d.
__device__ __forceinline__ float d2_gen(const float *x, const float *c, int d) {
    float e = 0.0f, o = 0.0f;
    int j = 0;
    for (; j + 1 < d; j += 2) {
        const float t0 = __fsub_rn(x[j], c[j]);
        const float t1 = __fsub_rn(x[j + 1], c[j + 1]);
        e = __fmaf_rn(t0, t0, e);
        o = __fmaf_rn(t1, t1, o);
    }
    if (j < d) {
        const float t0 = __fsub_rn(x[j], c[j]);
        e = __fmaf_rn(t0, t0, e);
    }
    return __fadd_rn(e, o);
}

// Upper bound on the exact distance whose square was computed as d2:
// the fma chain above has relative error <= (1 - (d+2) 2^-24)^-1 - 1 plus an
// absolute underflow term <= d 2^-150, so sqrt(d2 * g_up + tiny), with every
// operation rounded up, bounds the exact distance from above.
__device__ __forceinline__ float bound_up(float d2, float g_up, float tiny) {
    return __fsqrt_ru(__fmaf_ru(d2, g_up, tiny));
}

// Lower bound on the exact distance whose square was computed as d2 (the
// other side of bound_up): the exact square is at least (d2 - tiny) g^-1.
__device__ __forceinline__ float bound_down(float d2, float ginv_dn, float tiny) {
    return __fsqrt_rd(__fmul_rd(fmaxf(__fsub_rd(d2, tiny), 0.0f), ginv_dn));
}

// Error-free transformation of hi + x (Knuth's TwoSum): hi gets the rounded
// sum, lo collects the exact rounding error, so hi + lo carries the running
// sum to about FP32^2 precision.
__device__ __forceinline__ void two_sum_acc(float *hi, float *lo, float x) {
    const float h = *hi;
    const float s = __fadd_rn(h, x);
    const float bp = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    *hi = s;
    *lo = __fadd_rn(*lo, e);
}

// Adds x to the pair (h, l) held in registers (TwoSum; same arithmetic as
// two_sum_acc).
__device__ __forceinline__ void two_sum_reg(float &h, float &l, float x) {
    const float s = __fadd_rn(h, x);
    const float bp = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    h = s;
    l = __fadd_rn(l, e);
}

// (H, L) += (h, l): TwoSum of the high parts, low parts added with its error.
__device__ __forceinline__ void two_sum_merge(float &H, float &L, float h, float l) {
    const float s = __fadd_rn(H, h);
    const float bp = __fsub_rn(s, H);
    const float e = __fadd_rn(__fsub_rn(H, __fsub_rn(s, bp)), __fsub_rn(h, bp));
    H = s;
    L = __fadd_rn(__fadd_rn(L, l), e);
}

// Contiguous point range of this CTA, boundaries on multiples of `align`.
__device__ __forceinline__ void block_range(int64_t n, int64_t align, int64_t &lo, int64_t &hi) {
    const int64_t units = (n + align - 1) / align;
    const int64_t u0 = units * blockIdx.x / gridDim.x;
    const int64_t u1 = units * (blockIdx.x + 1) / gridDim.x;
    lo = min(n, u0 * align);
    hi = min(n, u1 * align);
}

} // namespace knor

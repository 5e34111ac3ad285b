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

// Squared distance, row in registers, centroid 16-byte aligned (smem or global).
template <int DV>
__device__ __forceinline__ float d2_reg(const float (&x)[DV], const float *c) {
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < DV; j += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(c + j);
        float t;
        t = __fsub_rn(x[j + 0], v.x); acc = __fmaf_rn(t, t, acc);
        t = __fsub_rn(x[j + 1], v.y); acc = __fmaf_rn(t, t, acc);
        t = __fsub_rn(x[j + 2], v.z); acc = __fmaf_rn(t, t, acc);
        t = __fsub_rn(x[j + 3], v.w); acc = __fmaf_rn(t, t, acc);
    }
    return acc;
}

// Four centroids at once (independent chains for ILP); each chain performs
// exactly the operations of d2_reg, so the values are identical.
template <int DV>
__device__ __forceinline__ void d2_reg4(const float (&x)[DV], const float *c, float &r0, float &r1,
                                        float &r2, float &r3) {
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
    for (int j = 0; j < DV; j += 4) {
        const float4 v0 = *reinterpret_cast<const float4 *>(c + j);
        const float4 v1 = *reinterpret_cast<const float4 *>(c + DV + j);
        const float4 v2 = *reinterpret_cast<const float4 *>(c + 2 * DV + j);
        const float4 v3 = *reinterpret_cast<const float4 *>(c + 3 * DV + j);
        float t;
#define KNOR_STEP(acc, xv, cv) t = __fsub_rn(xv, cv); acc = __fmaf_rn(t, t, acc);
        KNOR_STEP(a0, x[j], v0.x) KNOR_STEP(a1, x[j], v1.x) KNOR_STEP(a2, x[j], v2.x) KNOR_STEP(a3, x[j], v3.x)
        KNOR_STEP(a0, x[j + 1], v0.y) KNOR_STEP(a1, x[j + 1], v1.y) KNOR_STEP(a2, x[j + 1], v2.y) KNOR_STEP(a3, x[j + 1], v3.y)
        KNOR_STEP(a0, x[j + 2], v0.z) KNOR_STEP(a1, x[j + 2], v1.z) KNOR_STEP(a2, x[j + 2], v2.z) KNOR_STEP(a3, x[j + 2], v3.z)
        KNOR_STEP(a0, x[j + 3], v0.w) KNOR_STEP(a1, x[j + 3], v1.w) KNOR_STEP(a2, x[j + 3], v2.w) KNOR_STEP(a3, x[j + 3], v3.w)
#undef KNOR_STEP
    }
    r0 = a0; r1 = a1; r2 = a2; r3 = a3;
}

// Packed pair of FP32 values in one 64-bit register (for the f32x2 ops).
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

// Squared distances from one point to PG pairs of centroids with the packed
// sub.rn.f32x2 / fma.rn.f32x2 instructions.  Each lane of a pair performs
// exactly the operations of d2_reg (x_j - c_j rounded, then fma into its own
// accumulator, j = 0..DV-1 in order), so the results are bit-identical to
// d2_reg; two centroids per instruction halve the instruction count.
//   xx   x_j duplicated into both halves, j = 0..DV-1
//   cp   pair-major centroid copy: cp[(g*DV + j)] = (c_{2g}[j], c_{2g+1}[j])
template <int DV, int PG>
__device__ __forceinline__ void d2_pairs(const unsigned long long (&xx)[DV], const float2 *cp, float (&r)[2 * PG]) {
    unsigned long long acc[PG];
#pragma unroll
    for (int g = 0; g < PG; ++g) acc[g] = 0ULL; // (+0.0f, +0.0f)
#pragma unroll
    for (int j = 0; j < DV; j += 2) {
#pragma unroll
        for (int g = 0; g < PG; ++g) {
            const float4 v = *reinterpret_cast<const float4 *>(cp + (size_t)g * DV + j);
            unsigned long long t;
            asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(xx[j]), "l"(pack2(v.x, v.y)));
            asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc[g]) : "l"(t));
            asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(xx[j + 1]), "l"(pack2(v.z, v.w)));
            asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc[g]) : "l"(t));
        }
    }
#pragma unroll
    for (int g = 0; g < PG; ++g) unpack2(acc[g], r[2 * g], r[2 * g + 1]);
}

// Generic width: the same operation sequence with a runtime d.
__device__ __forceinline__ float d2_gen(const float *x, const float *c, int d) {
    float acc = 0.0f;
    for (int j = 0; j < d; ++j) {
        const float t = __fsub_rn(x[j], c[j]);
        acc = __fmaf_rn(t, t, acc);
    }
    return acc;
}

// Upper bound on the exact distance whose square was computed as d2:
// the fma chain above has relative error <= (1 - (d+2) 2^-24)^-1 - 1 plus an
// absolute underflow term <= d 2^-150, so sqrt(d2 * g_up + tiny), with every
// operation rounded up, bounds the exact distance from above.
__device__ __forceinline__ float bound_up(float d2, float g_up, float tiny) {
    return __fsqrt_ru(__fmaf_ru(d2, g_up, tiny));
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

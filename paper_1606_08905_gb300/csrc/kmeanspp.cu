// kmeanspp.cu -- k-means++ seeding on the GPU (knor_create with
// KNOR_INIT_KMEANSPP).
//
// k-means++ (Arthur and Vassilvitskii, SODA 2007; the paper lists it among
// the variants to come): the first centroid is a uniformly drawn point, every
// further one a point drawn with probability proportional to D^2, its squared
// distance to the nearest centroid chosen so far.  A draw is reproducible bit
// for bit: D^2 is the library's FP32 distance between the FP32 rows; the
// weights are D^2 on a power-of-two grid fixed per round, w = floor(D^2 2^E)
// with E = 32 - e and max D^2 < 2^e, so every weight is an exact integer below
// 2^32 and every sum exact; the draws are SplitMix64 outputs reduced by the
// multiply-shift (knor.h states the whole rule).  Each round runs three
// kernels: D^2 = min(D^2, distance to the last chosen point) with the round's
// maximum; the weights' sums over fixed contiguous ranges; then one CTA scans
// the one range that holds the draw.
#include "device_common.cuh"
#include "knor_internal.cuh"

namespace knor {
namespace {

constexpr int KPP_THREADS = 256;

// D2[i] = min(D2[i], d^2(x_i, c)) (first round: the distance itself); the
// largest D2 as float bits (D2 >= +0, so the bits order like the values).
template <int DV>
__global__ void __launch_bounds__(KPP_THREADS) k_kpp_update(const float *X, int64_t n, int32_t d,
                                                            const float *c, float *D2, int32_t first,
                                                            unsigned *maxbits) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        float v;
        if constexpr (DV > 0) {
            unsigned long long x2[DV / 2];
            ldg_x2<DV>(x2, X + i * DV);
            v = d2_reg<DV>(x2, c);
        } else {
            v = d2_gen(X + i * d, c, d);
        }
        if (!first) v = fminf(D2[i], v);
        D2[i] = v;
        mx = max(mx, __float_as_uint(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, mx);
}

__device__ __forceinline__ unsigned long long kpp_weight(float v, double scale) {
    return (unsigned long long)floor((double)v * scale); // exact: scale is a power of two
}

// The sum of the weights over CTA b's contiguous range (block_range).
__global__ void __launch_bounds__(KPP_THREADS) k_kpp_sums(const float *D2, int64_t n, double scale,
                                                          unsigned long long *sums) {
    int64_t lo, hi;
    block_range(n, 1, lo, hi);
    unsigned long long s = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += kpp_weight(D2[i], scale);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
    __shared__ unsigned long long ws[KPP_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < KPP_THREADS / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// One CTA: the first point of [lo, hi) whose running weight sum exceeds t.
__global__ void __launch_bounds__(1024) k_kpp_find(const float *D2, int64_t lo, int64_t hi, double scale,
                                                   unsigned long long t, int64_t *out) {
    __shared__ unsigned long long ws[32];
    __shared__ int64_t found;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) found = -1;
    __syncthreads();
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        const int64_t i = base + tid;
        const unsigned long long wi = i < hi ? kpp_weight(D2[i], scale) : 0ull;
        unsigned long long incl = wi; // inclusive scan over the chunk
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) ws[w] = incl;
        __syncthreads();
        unsigned long long before = 0, total = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            before += q < w ? ws[q] : 0ull;
            total += ws[q];
        }
        incl += before;
        if (i < hi && incl > t && incl - wi <= t) found = i; // exactly one point qualifies
        __syncthreads();
        if (found >= 0) break;
        t -= total;
        __syncthreads();
    }
    if (tid == 0) *out = found;
}

template <int DV>
cudaError_t kpp_update_t(const float *X, int64_t n, int32_t d, const float *c, float *D2, int first,
                         unsigned *maxbits, int grid, cudaStream_t s) {
    k_kpp_update<DV><<<grid, KPP_THREADS, 0, s>>>(X, n, d, c, D2, first, maxbits);
    return cudaGetLastError();
}

} // namespace

cudaError_t kpp_update(int dv, const float *X, int64_t n, int32_t d, const float *c, float *D2, int first,
                       unsigned *maxbits, int grid, cudaStream_t s) {
    switch (dv) {
    case 4: return kpp_update_t<4>(X, n, d, c, D2, first, maxbits, grid, s);
    case 8: return kpp_update_t<8>(X, n, d, c, D2, first, maxbits, grid, s);
    case 16: return kpp_update_t<16>(X, n, d, c, D2, first, maxbits, grid, s);
    case 32: return kpp_update_t<32>(X, n, d, c, D2, first, maxbits, grid, s);
    case 64: return kpp_update_t<64>(X, n, d, c, D2, first, maxbits, grid, s);
    case 128: return kpp_update_t<128>(X, n, d, c, D2, first, maxbits, grid, s);
    default: return kpp_update_t<0>(X, n, d, c, D2, first, maxbits, grid, s);
    }
}

cudaError_t kpp_sums(const float *D2, int64_t n, double scale, unsigned long long *sums, int grid, cudaStream_t s) {
    k_kpp_sums<<<grid, KPP_THREADS, 0, s>>>(D2, n, scale, sums);
    return cudaGetLastError();
}

cudaError_t kpp_find(const float *D2, int64_t lo, int64_t hi, double scale, unsigned long long t, int64_t *out,
                     cudaStream_t s) {
    k_kpp_find<<<1, 1024, 0, s>>>(D2, lo, hi, scale, t, out);
    return cudaGetLastError();
}

} // namespace knor

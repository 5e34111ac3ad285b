// noalloc.cu -- one Lloyd step on caller-owned device buffers that allocates
// no device memory (knor_lloyd_step_noalloc in include/knor.h).
//
// The other entry points allocate their working memory when a context is
// created.  This one is for callers that cannot do that: code whose device
// memory is handed out by another allocator (a framework caching allocator
// that has already reserved most of HBM, or an embedding application with a
// fixed memory budget), and latency-sensitive loops that must not call
// cudaMalloc/cudaFree because those calls synchronise the device.  Its only
// scratch memory is the fixed array below, which lives in the library's
// device image: every GPU that loads the library holds it until the process
// exits.
#include "device_common.cuh"
#include "knor.h"
#include "knor_internal.cuh"

#include <mutex>
#include <string>

namespace knor {

namespace {

// Scratch layout: NA_SLOTS per-CTA slots of (k*d FP64 sums, k int64 counts).
constexpr int NA_SLOTS = 256;
constexpr int NA_MAX_KD1 = 4096; // k * (d + 1) limit, so the slots fit below
constexpr size_t NA_BYTES = (size_t)NA_SLOTS * NA_MAX_KD1 * 8;

// One step: each of the NA_SLOTS single-warp CTAs scans a contiguous range of
// points (FP32 direct-form distance, index order, lowest index on ties, the
// same arithmetic as the context kernels), writes the assignments, and sums
// its rows per cluster in TwoSum FP32 pairs (lanes walk the dimensions, rows
// in point order, so the sums are deterministic).  Every CTA overwrites its
// whole slot, so nothing in the scratch has to start at zero.
__global__ void __launch_bounds__(32) k_step_noalloc(const float *X, int64_t n, int32_t d, int32_t k,
                                                     const float *C, int32_t *assign, unsigned char *scratch) {
    extern __shared__ __align__(16) unsigned char sm[];
    float *hi = reinterpret_cast<float *>(sm);
    float *lo = hi + (size_t)k * d;
    int *cnt = reinterpret_cast<int *>(lo + (size_t)k * d);
    const int lane = threadIdx.x;
    for (int e = lane; e < k * d; e += 32) { hi[e] = 0.0f; lo[e] = 0.0f; }
    for (int c = lane; c < k; c += 32) cnt[c] = 0;
    __syncwarp();
    const int64_t r0 = n * blockIdx.x / gridDim.x, r1 = n * (blockIdx.x + 1) / gridDim.x;
    for (int64_t base = r0; base < r1; base += 32) {
        const int64_t i = base + lane;
        const bool valid = i < r1;
        int best = -1;
        if (valid) {
            const float *x = X + i * d;
            float bd = CUDART_INF_F;
            for (int c = 0; c < k; ++c) {
                const float r = d2_gen(x, C + (size_t)c * d, d);
                if (r < bd) { bd = r; best = c; }
            }
            assign[i] = best;
        }
        unsigned rem = __ballot_sync(FULL_MASK, valid);
        while (rem) {
            const int c = __shfl_sync(FULL_MASK, best, __ffs(rem) - 1);
            const unsigned grp = __ballot_sync(FULL_MASK, valid && best == c);
            rem &= ~grp;
            for (int j = lane; j < d; j += 32) {
                float h = 0.0f, l = 0.0f;
                unsigned m = grp;
                while (m) {
                    const int pl = __ffs(m) - 1;
                    m &= m - 1;
                    two_sum_reg(h, l, X[(base + pl) * d + j]);
                }
                float H = hi[c * d + j], L = lo[c * d + j];
                two_sum_merge(H, L, h, l);
                hi[c * d + j] = H;
                lo[c * d + j] = L;
            }
            if (lane == 0) cnt[c] += __popc(grp);
            __syncwarp();
        }
    }
    __syncwarp();
    double *S = reinterpret_cast<double *>(scratch) + (size_t)blockIdx.x * k * (d + 1);
    long long *N = reinterpret_cast<long long *>(S + (size_t)k * d);
    for (int e = lane; e < k * d; e += 32) S[e] = (double)hi[e] + (double)lo[e];
    for (int c = lane; c < k; c += 32) N[c] = cnt[c];
}

// Adds the slots in slot order into the caller's FP64 sums and counts.
__global__ void k_merge_noalloc(int32_t d, int32_t k, const unsigned char *scratch, double *sums,
                                int64_t *counts) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t kd = (int64_t)k * d;
    if (e >= kd + k) return;
    const size_t stride = (size_t)k * (d + 1);
    const double *S = reinterpret_cast<const double *>(scratch);
    if (e < kd) {
        double s = 0.0;
        for (int g = 0; g < NA_SLOTS; ++g) s += S[g * stride + e];
        sums[e] = s;
    } else {
        const int64_t c = e - kd;
        long long s = 0;
        for (int g = 0; g < NA_SLOTS; ++g) s += reinterpret_cast<const long long *>(S + g * stride + kd)[c];
        counts[c] = s;
    }
}

// The scratch array.  In host code its name is only a host-side stand-in:
// kernels get the device address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
void *g_na_addr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on each device).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_na_mutex);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return cudaSuccess;
}

} // namespace
} // namespace knor

extern "C" knor_status knor_lloyd_step_noalloc(const float *points, int64_t n, int32_t d, int32_t k,
                                               const float *centroids, int32_t *assign_out, double *sums_out,
                                               int64_t *counts_out, void *stream) {
    using namespace knor;
    set_global_error("");
    if (!points || !centroids || !assign_out || !sums_out || !counts_out) {
        set_global_error("knor_lloyd_step_noalloc: NULL buffer");
        return KNOR_ERR_ARG;
    }
    if (n < 1 || d < 1 || k < 1) {
        set_global_error("knor_lloyd_step_noalloc: need n >= 1, d >= 1, k >= 1");
        return KNOR_ERR_ARG;
    }
    if ((int64_t)k * (d + 1) > NA_MAX_KD1) {
        set_global_error("knor_lloyd_step_noalloc: k * (d + 1) exceeds 4096, the size of the fixed scratch "
                         "array (use a context from knor_create instead)");
        return KNOR_ERR_ARG;
    }
    // every buffer must be device memory of the current device: a host
    // pointer, or memory of another GPU without peer access, would fault the
    // kernel (and the scratch array looked up below is the current device's)
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        set_global_error("knor_lloyd_step_noalloc: no current CUDA device");
        return KNOR_ERR_CUDA;
    }
    const void *bufs[] = {points, centroids, assign_out, sums_out, counts_out};
    for (const void *b : bufs) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, b) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            set_global_error("knor_lloyd_step_noalloc: every buffer must be device memory");
            return KNOR_ERR_ARG;
        }
        if (at.type == cudaMemoryTypeDevice && at.device != cur) {
            set_global_error("knor_lloyd_step_noalloc: a buffer is on another device than the current one");
            return KNOR_ERR_ARG;
        }
    }
    void *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_global_error((std::string("knor_lloyd_step_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
        return KNOR_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t smem = (size_t)k * d * 8 + (size_t)k * 4;
    k_step_noalloc<<<NA_SLOTS, 32, smem, s>>>(points, n, d, k, centroids, assign_out,
                                                static_cast<unsigned char *>(scratch));
    const int64_t m = (int64_t)k * d + k;
    k_merge_noalloc<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(d, k, static_cast<unsigned char *>(scratch),
                                                                  sums_out, counts_out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_global_error((std::string("knor_lloyd_step_noalloc: ") + cudaGetErrorString(e)).c_str());
        return KNOR_ERR_CUDA;
    }
    return KNOR_OK;
}

// FP64 reductions: maximum (Fig. 1's maximum(Ci) for dt), dot products and
// the inverse problem's loss 1/2||A-B||^2.  Sums use a fixed partition into
// kReduceBlocks blocks and a fixed tree order, so results do not depend on
// scheduling.  Workspace layout: [0, 8) max key, [64, 64 + 8*kReduceBlocks)
// per-block partial sums.
#include "internal.h"

namespace psd {

constexpr int kRThreads = 256;

__device__ __forceinline__ unsigned long long order_key(double x) {
    // monotone map of doubles to unsigned integers (total order on non-NaN values)
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_value(unsigned long long k) {
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

template <typename E>
__global__ void __launch_bounds__(kRThreads)
k_max(const E *__restrict__ A, int64_t n, unsigned long long *__restrict__ key) {
    double m = -INFINITY;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        m = fmax(m, (double)A[p]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double sm[kRThreads / 32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kRThreads / 32; ++w) m = fmax(m, sm[w]);
        atomicMax(key, order_key(m));
    }
}

__global__ void k_max_finish(const unsigned long long *__restrict__ key, double *__restrict__ out) {
    *out = key_value(*key);
}

// Block-level fixed-order sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (threadIdx.x < 32) {
        v = threadIdx.x < (unsigned)nw ? sm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// kind 0: sum A*B; kind 1: sum (A-B)^2 and optionally R = A - B.
template <typename E, int kind>
__global__ void __launch_bounds__(kRThreads)
k_partial(const E *__restrict__ A, const E *__restrict__ B, E *__restrict__ R, int64_t n,
          double *__restrict__ partial) {
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        if (kind == 0) {
            acc += (double)A[p] * (double)B[p];
        } else {
            const E r = A[p] - B[p];
            if (R) R[p] = r;
            const double rd = (double)A[p] - (double)B[p];
            acc += rd * rd;
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kReduceBlocks)
k_final(const double *__restrict__ partial, double scale, double *__restrict__ out) {
    const double s = block_sum(partial[threadIdx.x]);
    if (threadIdx.x == 0) *out = scale * s;
}

static double *partials(void *ws) { return (double *)((char *)ws + 64); }

cudaError_t launch_maximum(double *out_dev, const void *A, int64_t n, int dtype, void *ws,
                           cudaStream_t s) {
    auto *key = (unsigned long long *)ws;
    cudaError_t e = cudaMemsetAsync(key, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (n + kRThreads - 1) / kRThreads;
    if (blocks > 4LL * sm_count()) blocks = 4LL * sm_count();
    if (dtype == PS_F64)
        k_max<double><<<(unsigned)blocks, kRThreads, 0, s>>>((const double *)A, n, key);
    else
        k_max<float><<<(unsigned)blocks, kRThreads, 0, s>>>((const float *)A, n, key);
    k_max_finish<<<1, 1, 0, s>>>(key, out_dev);
    return cudaGetLastError();
}

template <int kind>
static cudaError_t launch_sum(double *out_dev, void *R, const void *A, const void *B, int64_t n,
                              int dtype, void *ws, double scale, cudaStream_t s) {
    if (dtype == PS_F64)
        k_partial<double, kind><<<kReduceBlocks, kRThreads, 0, s>>>(
            (const double *)A, (const double *)B, (double *)R, n, partials(ws));
    else
        k_partial<float, kind><<<kReduceBlocks, kRThreads, 0, s>>>(
            (const float *)A, (const float *)B, (float *)R, n, partials(ws));
    k_final<<<1, kReduceBlocks, 0, s>>>(partials(ws), scale, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_dot(double *out_dev, const void *A, const void *B, int64_t n, int dtype,
                       void *ws, cudaStream_t s) {
    return launch_sum<0>(out_dev, nullptr, A, B, n, dtype, ws, 1.0, s);
}

cudaError_t launch_half_sq_dist(double *out_dev, void *R, const void *A, const void *B, int64_t n,
                                int dtype, void *ws, cudaStream_t s) {
    return launch_sum<1>(out_dev, R, A, B, n, dtype, ws, 0.5, s);
}

}  // namespace psd

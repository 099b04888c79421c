// Dot product that allocates nothing: its scratch lives in a file-scope
// device array that is part of the library image.
//
// Some callers cannot allocate device memory at all - for example a plugin
// that runs inside a host application which owns every device allocation, or
// a loop that must not pay for (or risk failing) an allocation while it
// runs.  ps_dot needs a caller-allocated workspace for its per-block partial
// sums; ps_dot_static keeps them in g_static_partials instead.  That array
// is created when the library is loaded and stays resident on every GPU that
// uses the library until the process exits.
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace psd {

constexpr int kStaticThreads = 256;
constexpr int64_t kStaticChunk = 4096;      // elements summed by one block
constexpr int kStaticPartials = 32768;      // 256 KiB: one double per block
constexpr int kStaticFinalThreads = 1024;

static __device__ __align__(256) double g_static_partials[kStaticPartials];

// Host-side copies of the array's device address, one per device, each with the
// generation of the context it was looked up in.  In host code the name
// g_static_partials is only a stand-in for the symbol, not a device address, so
// the address is looked up with cudaGetSymbolAddress once per device and context
// (again after cudaDeviceReset, which loads the library's module anew).
static double *g_static_ptr[64] = {nullptr};
static unsigned g_static_gen[64] = {0};
static std::mutex g_static_mu;

static cudaError_t static_partials(double **out) {
    const int d = current_device();
    if (d < 0 || d >= 64) return cudaErrorInvalidDevice;
    const unsigned gen = context_generation();
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[d] || g_static_gen[d] != gen) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) return e;
        g_static_ptr[d] = (double *)p;
        g_static_gen[d] = gen;
    }
    *out = g_static_ptr[d];
    return cudaSuccess;
}

__device__ __forceinline__ double static_block_sum(double v) {
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

// Block b sums A*B over elements [b*kStaticChunk, (b+1)*kStaticChunk) in FP64.
template <typename E>
__global__ void __launch_bounds__(kStaticThreads)
k_dot_chunks(const E *__restrict__ A, const E *__restrict__ B, int64_t n, double *__restrict__ partial) {
    const int64_t begin = (int64_t)blockIdx.x * kStaticChunk;
    const int64_t end = begin + kStaticChunk < n ? begin + kStaticChunk : n;
    double acc = 0.0;
    for (int64_t p = begin + threadIdx.x; p < end; p += kStaticThreads)
        acc += (double)A[p] * (double)B[p];
    const double s = static_block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// One block adds the nparts partials in a fixed order.
__global__ void __launch_bounds__(kStaticFinalThreads)
k_dot_chunks_final(const double *__restrict__ partial, int nparts, double *__restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kStaticFinalThreads) acc += partial[i];
    const double s = static_block_sum(acc);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace psd

using namespace psd;

extern "C" int ps_dot_static(double *out_dev, const void *A, const void *B, int64_t n, int dtype,
                             void *stream) {
    if (!out_dev || !A || !B) return api_fail(PS_ERR_ARG, "ps_dot_static: out_dev, A or B is NULL");
    if (dtype != PS_F32 && dtype != PS_F64) return api_fail(PS_ERR_ARG, "ps_dot_static: bad dtype");
    const uintptr_t esz = dtype == PS_F64 ? 8u : 4u;  // the kernel reads one element at a time
    if (((uintptr_t)A | (uintptr_t)B) & (esz - 1u))
        return api_fail(PS_ERR_ALIGN, "ps_dot_static: A and B must be aligned to their element size");
    if (n < 1) return api_fail(PS_ERR_ARG, "ps_dot_static: n < 1");
    const int64_t nmax = kStaticChunk * kStaticPartials;
    if (n > nmax) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "ps_dot_static: n = %lld exceeds the static scratch capacity of %lld elements "
                 "(use ps_dot with a workspace)",
                 (long long)n, (long long)nmax);
        return api_fail(PS_ERR_UNSUPPORTED, msg);
    }
    double *partial = nullptr;
    cudaError_t e = static_partials(&partial);
    if (e != cudaSuccess) return api_cuda_fail(e, "ps_dot_static: cudaGetSymbolAddress");
    const int nparts = (int)((n + kStaticChunk - 1) / kStaticChunk);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == PS_F64)
        k_dot_chunks<double><<<nparts, kStaticThreads, 0, s>>>((const double *)A, (const double *)B, n, partial);
    else
        k_dot_chunks<float><<<nparts, kStaticThreads, 0, s>>>((const float *)A, (const float *)B, n, partial);
    k_dot_chunks_final<<<1, kStaticFinalThreads, 0, s>>>(partial, nparts, out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return api_cuda_fail(e, "ps_dot_static");
    return PS_OK;
}

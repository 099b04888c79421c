// Boundary copy (Fig. 1's T2 = copy(T), restricted to the boundary faces)
// and the FP32 deviation conversions.
#include "internal.h"

namespace psd {

// blockIdx.y selects the face: 0/1 z = 0 / nz-1, 2/3 y = 0 / ny-1, 4/5 x = 0 / nx-1.
// A thread takes face nodes t = blockIdx.x*blockDim.x + threadIdx.x (grid-stride), finds
// each node's offset once, reads it once and stores it into all `count` destination grids
// (dst + c * gstride): consecutive threads hold consecutive nodes of a face, so the stores
// into one grid are coalesced wherever the face is (the z and y faces, rows of x).  Edges
// and corners belong to several faces and are written with the same value more than once.
template <typename E>
__global__ void k_copy_boundary(E *__restrict__ dst, const E *__restrict__ src, int64_t nx,
                                int64_t ny, int64_t nz, int64_t gstride, int64_t count) {
    const int face = blockIdx.y;
    const int64_t rows = face < 2 ? ny : nz;            // the face is rows x cols nodes
    const int64_t cols = face < 4 ? nx : ny;
    const int64_t nodes = rows * cols;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nodes; t += stride) {
        const int64_t r = t / cols, q = t - r * cols;   // one division per node, not per grid
        int64_t p;
        if (face < 2)
            p = q + nx * (r + ny * (face == 0 ? 0 : nz - 1));
        else if (face < 4)
            p = q + nx * ((face == 2 ? 0 : ny - 1) + ny * r);
        else
            p = (face == 4 ? 0 : nx - 1) + nx * (q + ny * r);
        const E v = src[p];
        E *d = dst + p;
        for (int64_t c = 0; c < count; ++c, d += gstride) *d = v;
    }
}

// z_faces_only: the two z faces (planes 0 and nz-1) alone, for grids whose x and y faces
// the steps write themselves.
cudaError_t launch_copy_boundary_many(void *dst, int64_t count, int64_t gstride, const void *T,
                                      Grid3 g, int elem_bytes, cudaStream_t s, bool z_faces_only) {
    if (count <= 0) return cudaSuccess;
    const int64_t maxface = g.nx * g.ny > g.nx * g.nz ? g.nx * g.ny : g.nx * g.nz;
    const int64_t mf = maxface > g.ny * g.nz ? maxface : g.ny * g.nz;
    int64_t blocks = (mf + 255) / 256;
    const int64_t cap = 2LL * sm_count();  // six faces: about 12 blocks per SM in all
    if (blocks > cap) blocks = cap;
    const dim3 grid((unsigned)blocks, z_faces_only ? 2 : 6, 1);  // faces 0 .. grid.y-1
    if (elem_bytes == 8)
        k_copy_boundary<unsigned long long><<<grid, 256, 0, s>>>(
            (unsigned long long *)dst, (const unsigned long long *)T, g.nx, g.ny, g.nz, gstride, count);
    else
        k_copy_boundary<unsigned><<<grid, 256, 0, s>>>((unsigned *)dst, (const unsigned *)T, g.nx, g.ny,
                                                      g.nz, gstride, count);
    return cudaGetLastError();
}

cudaError_t launch_copy_boundary(void *T2, const void *T, Grid3 g, int elem_bytes,
                                 cudaStream_t s) {
    return launch_copy_boundary_many(T2, 1, g.nx * g.ny * g.nz, T, g, elem_bytes, s);
}

__global__ void k_to_deviation(float *__restrict__ D, const double *__restrict__ T, double t_ref,
                               int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        D[p] = __double2float_rn(T[p] - t_ref);
}

__global__ void k_from_deviation(double *__restrict__ T, const float *__restrict__ D, double t_ref,
                                 int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        T[p] = (double)D[p] + t_ref;
}

// Two-float deviation: v = T - t_ref in FP64, D = v rounded to float, E = v - D
// rounded to float (D + E carries about 48 bits of v).
__global__ void k_to_deviation_pair(float *__restrict__ D, float *__restrict__ E,
                                    const double *__restrict__ T, double t_ref, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const double v = T[p] - t_ref;
        const float d = __double2float_rn(v);
        D[p] = d;
        E[p] = __double2float_rn(v - (double)d);
    }
}

__global__ void k_from_deviation_pair(double *__restrict__ T, const float *__restrict__ D,
                                      const float *__restrict__ E, double t_ref, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        T[p] = ((double)D[p] + (double)E[p]) + t_ref;
}

__global__ void k_scale_ci(double *__restrict__ Cs, const double *__restrict__ Ci, double K, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) Cs[p] = K * Ci[p];
}

static unsigned ew_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = 8LL * sm_count();
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

cudaError_t launch_to_deviation(float *D, const double *T, double t_ref, int64_t n,
                                cudaStream_t s) {
    k_to_deviation<<<ew_blocks(n), 256, 0, s>>>(D, T, t_ref, n);
    return cudaGetLastError();
}

cudaError_t launch_from_deviation(double *T, const float *D, double t_ref, int64_t n,
                                  cudaStream_t s) {
    k_from_deviation<<<ew_blocks(n), 256, 0, s>>>(T, D, t_ref, n);
    return cudaGetLastError();
}

cudaError_t launch_to_deviation_pair(float *D, float *E, const double *T, double t_ref, int64_t n,
                                     cudaStream_t s) {
    k_to_deviation_pair<<<ew_blocks(n), 256, 0, s>>>(D, E, T, t_ref, n);
    return cudaGetLastError();
}

cudaError_t launch_from_deviation_pair(double *T, const float *D, const float *E, double t_ref, int64_t n,
                                       cudaStream_t s) {
    k_from_deviation_pair<<<ew_blocks(n), 256, 0, s>>>(T, D, E, t_ref, n);
    return cudaGetLastError();
}

}  // namespace psd

namespace psd {

cudaError_t launch_scale_ci(double *Cs, const double *Ci, double K, int64_t n, cudaStream_t s) {
    k_scale_ci<<<ew_blocks(n), 256, 0, s>>>(Cs, Ci, K, n);
    return cudaGetLastError();
}

}  // namespace psd

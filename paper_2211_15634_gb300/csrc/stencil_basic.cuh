// Plain 7-point step kernels: one thread per interior (i, j) column,
// marching along z with a three-value register queue.  x/y neighbours are
// read through the L1/L2 caches.  These are the straightforward kernels
// (FP64 instructions for FP64 data); the tiled kernels replace them on the
// hot path.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "emu64.cuh"
#include "node.cuh"

namespace psd {

template <typename F>
struct CoefT {
    F dtlam, ax, ay, az;
};

// Same column march for FP64 data with the one-DFMA emulated arithmetic of
// emu64.cuh (used when the TMA kernel cannot serve the grid, e.g. odd nx).
template <bool kIso, bool kScaled>
__global__ void __launch_bounds__(256)
k_step_basic_emu(double *__restrict__ T2, const double *__restrict__ T,
                 const double *__restrict__ Ci, EmuCoef c, int64_t nx, int64_t ny, int64_t nz,
                 int kchunk) {
    const int64_t i = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = 1 + (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i > nx - 2 || j > ny - 2) return;
    const int64_t k0 = 1 + (int64_t)blockIdx.z * kchunk;
    const int64_t k1 = k0 + kchunk < nz - 1 ? k0 + kchunk : nz - 1;
    if (k0 >= k1) return;
    const int64_t sy = nx, sz = nx * ny;
    const unsigned long long *__restrict__ Tb = (const unsigned long long *)T;
    int64_t p = i + sy * (j + ny * k0);
    unsigned long long tm = Tb[p - sz], tc = Tb[p];
    for (int64_t k = k0; k < k1; ++k, p += sz) {
        const unsigned long long tp = Tb[p + sz];
        if (kScaled)  // Ci holds dt*lam*_d^2*Ci (isotropic grid)
            T2[p] = emu_step_node_scaled(tc, Tb[p - 1], Tb[p + 1], Tb[p - sy], Tb[p + sy], tm, tp, Ci[p]);
        else
            T2[p] = emu_step_node<kIso, false>(tc, Tb[p - 1], Tb[p + 1], Tb[p - sy], Tb[p + sy], tm,
                                               tp, Ci[p], c);
        tm = tc;
        tc = tp;
    }
}

inline cudaError_t launch_step_basic_emu(double *T2, const double *T, const double *Ci,
                                         const EmuCoef &c, bool iso, int64_t nx, int64_t ny,
                                         int64_t nz, int nsm, cudaStream_t s, bool scaled = false) {
    const dim3 block(32, 8, 1);
    const int64_t gx = (nx - 2 + block.x - 1) / block.x, gy = (ny - 2 + block.y - 1) / block.y;
    int64_t want = (8LL * nsm + gx * gy - 1) / (gx * gy);
    int64_t kchunk = (nz - 2 + want - 1) / want;
    if (kchunk < 16) kchunk = 16;
    const int64_t gz = (nz - 2 + kchunk - 1) / kchunk;
    if (gx > 0x7fffffff || gy > 65535 || gz > 65535) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)gz);
    if (scaled)
        k_step_basic_emu<true, true><<<grid, block, 0, s>>>(T2, T, Ci, c, nx, ny, nz, (int)kchunk);
    else if (iso)
        k_step_basic_emu<true, false><<<grid, block, 0, s>>>(T2, T, Ci, c, nx, ny, nz, (int)kchunk);
    else
        k_step_basic_emu<false, false><<<grid, block, 0, s>>>(T2, T, Ci, c, nx, ny, nz, (int)kchunk);
    return cudaGetLastError();
}

// Fig. 1 step!: T2 = T + dt*lam*Ci*((d2x*_dx^2 + d2y*_dy^2) + d2z*_dz^2) at
// interior nodes; the z-range of this block is [k0, k1).  kComp (FP32): the state
// is the two-float pair (T, E) and (T2, E2) receives the compensated step
// (comp32_node, node.cuh).
template <typename F, bool kComp>
__global__ void __launch_bounds__(256)
k_step_basic(F *__restrict__ T2, const F *__restrict__ T, F *__restrict__ E2,
             const F *__restrict__ E, const F *__restrict__ Ci, CoefT<F> c, int64_t nx, int64_t ny,
             int64_t nz, int kchunk) {
    const int64_t i = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = 1 + (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i > nx - 2 || j > ny - 2) return;
    const int64_t k0 = 1 + (int64_t)blockIdx.z * kchunk;
    const int64_t k1 = k0 + kchunk < nz - 1 ? k0 + kchunk : nz - 1;
    if (k0 >= k1) return;
    const int64_t sy = nx, sz = nx * ny;
    int64_t p = i + sy * (j + ny * k0);
    F tm = T[p - sz], tc = T[p];
    for (int64_t k = k0; k < k1; ++k, p += sz) {
        const F tp = T[p + sz];
        if constexpr (kComp) {
            float e2;
            T2[p] = comp32_node(tc, T[p - 1], T[p + 1], T[p - sy], T[p + sy], tm, tp, E[p], E[p - 1],
                                E[p + 1], E[p - sy], E[p + sy], E[p - sz], E[p + sz], Ci[p], c.dtlam,
                                c.ax, c.ay, c.az, &e2);
            E2[p] = e2;
        } else {
            const F d2x = (T[p + 1] - tc) - (tc - T[p - 1]);
            const F d2y = (T[p + sy] - tc) - (tc - T[p - sy]);
            const F d2z = (tp - tc) - (tc - tm);
            const F lap = (d2x * c.ax + d2y * c.ay) + d2z * c.az;
            T2[p] = tc + c.dtlam * (Ci[p] * lap);
        }
        tm = tc;
        tc = tp;
    }
}

template <typename F, bool kComp>
cudaError_t launch_step_basic(F *T2, const F *T, F *E2, const F *E, const F *Ci, CoefT<F> c, int64_t nx,
                              int64_t ny, int64_t nz, int nsm, cudaStream_t s) {
    const dim3 block(32, 8, 1);
    const int64_t gx = (nx - 2 + block.x - 1) / block.x, gy = (ny - 2 + block.y - 1) / block.y;
    // enough z-chunks for about 8 blocks per SM, each chunk at least 16 planes
    int64_t want = (8LL * nsm + gx * gy - 1) / (gx * gy);
    int64_t kchunk = (nz - 2 + want - 1) / want;
    if (kchunk < 16) kchunk = 16;
    const int64_t gz = (nz - 2 + kchunk - 1) / kchunk;
    if (gx > 0x7fffffff || gy > 65535 || gz > 65535) return cudaErrorInvalidConfiguration;
    k_step_basic<F, kComp><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), block, 0, s>>>(
        T2, T, E2, E, Ci, c, nx, ny, nz, (int)kchunk);
    return cudaGetLastError();
}

}  // namespace psd

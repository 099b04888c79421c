// Batched step: many independent problems of different sizes in one
// persistent launch.  The device table holds a header, one record per
// problem and a static work list of (problem, x-y tile, z-chunk) items; CTA
// b processes items b, b + gridDim.x, ... (no atomics, no counters, so a
// captured graph replays the same schedule every time).
#include "internal.h"

namespace psd {

constexpr int kBatchThreads = 256;

template <typename F>
__device__ __forceinline__ void batch_item(const BatchItem item, const BatchProblem &P, int parity,
                                           int tx, int ty, int tz) {
    const F *__restrict__ T = (const F *)(parity ? P.T2 : P.T);
    F *__restrict__ T2 = (F *)(parity ? P.T : P.T2);
    const F *__restrict__ Ci = (const F *)P.Ci;
    const F dtlam = (F)P.dtlam, ax = (F)P.ax, ay = (F)P.ay, az = (F)P.az;
    const int64_t nx = P.nx, ny = P.ny, nz = P.nz, sy = nx, sz = nx * ny;
    const int64_t k0 = item.k0, k1 = k0 + tz < nz - 1 ? k0 + tz : nz - 1;
    for (int t = threadIdx.x; t < tx * ty; t += blockDim.x) {
        const int64_t i = item.i0 + t % tx, j = item.j0 + t / tx;
        if (i > nx - 2 || j > ny - 2) continue;
        int64_t p = i + sy * (j + ny * k0);
        F tm = T[p - sz], tc = T[p];
        for (int64_t k = k0; k < k1; ++k, p += sz) {
            const F tp = T[p + sz];
            const F d2x = (T[p + 1] - tc) - (tc - T[p - 1]);
            const F d2y = (T[p + sy] - tc) - (tc - T[p - sy]);
            const F d2z = (tp - tc) - (tc - tm);
            const F lap = (d2x * ax + d2y * ay) + d2z * az;
            T2[p] = tc + dtlam * (Ci[p] * lap);
            tm = tc;
            tc = tp;
        }
    }
}

template <typename F>
__global__ void __launch_bounds__(kBatchThreads) k_batch_step(const char *__restrict__ table,
                                                               int parity) {
    const BatchHeader *h = (const BatchHeader *)table;
    const BatchProblem *probs = (const BatchProblem *)(table + h->problems_offset);
    const BatchItem *items = (const BatchItem *)(table + h->items_offset);
    const int64_t nitems = h->nitems;
    const int tx = h->tile_x, ty = h->tile_y, tz = h->tile_z;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem item = items[it];
        batch_item<F>(item, probs[item.prob], parity, tx, ty, tz);
    }
}

int batch_default_tile(int dtype, int *tx, int *ty, int *tz) {
    (void)dtype;
    *tx = 32;
    *ty = 8;
    *tz = 32;
    return 0;
}

cudaError_t launch_batch_step(const void *dev_table, int parity, int dtype, cudaStream_t s) {
    const unsigned grid = (unsigned)(8 * sm_count());
    if (dtype == PS_F64)
        k_batch_step<double><<<grid, kBatchThreads, 0, s>>>((const char *)dev_table, parity);
    else
        k_batch_step<float><<<grid, kBatchThreads, 0, s>>>((const char *)dev_table, parity);
    return cudaGetLastError();
}

}  // namespace psd

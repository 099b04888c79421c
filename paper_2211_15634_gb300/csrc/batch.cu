// Batched step: many independent problems of different sizes in one
// persistent launch.  The device table holds a header, one record per
// problem and a static work list of (problem, x-y tile, z-chunk) items, the
// largest first; CTA b processes items b, b + gridDim.x, ... (no atomics and
// no counters, so a captured graph replays the same schedule every time).
//
// Rows are P.pitch elements apart (nx for contiguous fields), planes pitch*ny.
// Within an item every thread owns one interior (i, j) column of the tile and
// marches along z with a three-value register queue; x/y neighbours are read
// through L1/L2 (problems of 32^3..160^3 are small enough for the caches to
// serve the reuse, and any nx works - the TMA path needs 16-byte row pitches).
// FP64 problems use the emulated one-DFMA arithmetic of emu64.cuh.
#include "emu64.cuh"
#include "internal.h"

namespace psd {

constexpr int kBatchThreads = 256;

__device__ unsigned g_batch_error;  // bit 1: a table built for the z-march kernel was given

template <typename F>
__device__ __forceinline__ void batch_item(const BatchItem &item, const BatchProblem &P, int parity) {
    const F *__restrict__ T = (const F *)(parity ? P.T2 : P.T);
    F *__restrict__ T2 = (F *)(parity ? P.T : P.T2);
    const F *__restrict__ Ci = (const F *)P.Ci;
    // batch problems hold fewer than 2^31 nodes (checked when the table is
    // built), so 32-bit offsets suffice and keep the register count low
    const int ny = (int)P.ny, sy = (int)P.pitch, sz = sy * ny;
    const int ni = item.ni, nj = item.nj;
    const int k0 = item.k0, k1 = k0 + item.nk;
    for (int t = threadIdx.x; t < ni * nj; t += blockDim.x) {
        const int i = item.i0 + t % ni, j = item.j0 + t / ni;
        int p = i + sy * (j + ny * k0);
        if (sizeof(F) == 8 && P.iso < 0) {  // coefficients the emulation cannot take: plain FP64
            const F dtlam = (F)P.dtlam, ax = (F)P.ax, ay = (F)P.ay, az = (F)P.az;
            F tm = T[p - sz], tc = T[p];
            for (int kk = k0; kk < k1; ++kk, p += sz) {
                const F tp = T[p + sz];
                const F d2x = (T[p + 1] - tc) - (tc - T[p - 1]);
                const F d2y = (T[p + sy] - tc) - (tc - T[p - sy]);
                const F d2z = (tp - tc) - (tc - tm);
                T2[p] = tc + dtlam * (Ci[p] * ((d2x * ax + d2y * ay) + d2z * az));
                tm = tc;
                tc = tp;
            }
        } else if constexpr (sizeof(F) == 8) {
            const unsigned long long *__restrict__ Tb = (const unsigned long long *)T;
            const EmuCoef k{EmuK{P.kxm, P.kxe}, EmuK{P.kym, P.kye}, EmuK{P.kzm, P.kze},
                            P.dtlam, P.ax, P.ay, P.az, 0.0};
            unsigned long long tm = Tb[p - sz], tc = Tb[p];
            if (P.iso) {
                for (int kk = k0; kk < k1; ++kk, p += sz) {
                    const unsigned long long tp = Tb[p + sz];
                    T2[p] = emu_step_node<true, false>(tc, Tb[p - 1], Tb[p + 1], Tb[p - sy],
                                                       Tb[p + sy], tm, tp, Ci[p], k);
                    tm = tc;
                    tc = tp;
                }
            } else {
                for (int kk = k0; kk < k1; ++kk, p += sz) {
                    const unsigned long long tp = Tb[p + sz];
                    T2[p] = emu_step_node<false, false>(tc, Tb[p - 1], Tb[p + 1], Tb[p - sy],
                                                        Tb[p + sy], tm, tp, Ci[p], k);
                    tm = tc;
                    tc = tp;
                }
            }
        } else {
            const F dtlam = (F)P.dtlam, ax = (F)P.ax, ay = (F)P.ay, az = (F)P.az;
            F tm = T[p - sz], tc = T[p];
            // loads of plane k+1 issued before plane k is computed (one plane of latency
            // hidden behind the arithmetic: measured 11% faster on the 256-problem batch;
            // the FP64 loop, register-bound, is faster without it)
            F tp = T[p + sz], xl = T[p - 1], xr = T[p + 1], yl = T[p - sy], yr = T[p + sy], ci = Ci[p];
            for (int kk = k0; kk < k1; ++kk, p += sz) {
                const int q = kk + 1 < k1 ? p + sz : p;
                const F tp2 = T[q + sz], xl2 = T[q - 1], xr2 = T[q + 1], yl2 = T[q - sy],
                        yr2 = T[q + sy], ci2 = Ci[q];
                const F d2x = (xr - tc) - (tc - xl);
                const F d2y = (yr - tc) - (tc - yl);
                const F d2z = (tp - tc) - (tc - tm);
                const F lap = (d2x * ax + d2y * ay) + d2z * az;
                T2[p] = tc + dtlam * (ci * lap);
                tm = tc;
                tc = tp;
                tp = tp2;
                xl = xl2;
                xr = xr2;
                yl = yl2;
                yr = yr2;
                ci = ci2;
            }
        }
    }
}

// Resident CTAs per SM the register budget is sized for: the FP32 march with
// its loads one plane ahead fits 5 x 256 threads without spills; the FP64
// emulated arithmetic 4 x 256.
template <typename F>
struct BatchOcc {
    static constexpr int min_blocks = sizeof(F) == 8 ? 4 : 5;
};

template <typename F>
__global__ void __launch_bounds__(kBatchThreads, BatchOcc<F>::min_blocks)
k_batch_step(const char *__restrict__ table, int parity) {
    const BatchHeader *h = (const BatchHeader *)table;
    if (h->kernel != 0) {  // items of the z-march kernel: not this kernel's work
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&g_batch_error, 2u);
        return;
    }
    const BatchProblem *probs = (const BatchProblem *)(table + h->problems_offset);
    const BatchItem *items = (const BatchItem *)(table + h->items_offset);
    const int64_t nitems = h->nitems;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem item = items[it];
        batch_item<F>(item, probs[item.prob], parity);
    }
}

int batch_default_tile(int dtype, int *tx, int *ty, int *tz) {
    (void)dtype;
    *tx = 32;
    *ty = 8;
    *tz = 32;
    return 0;
}

// Persistent grid = exactly the CTAs that can be resident at once: the static
// round-robin hand-out only balances when no CTA waits for a second wave.
template <typename F>
static unsigned resident_grid() {
    static int per_sm[64] = {0};
    const int d = current_device();
    int v = (d >= 0 && d < 64) ? per_sm[d] : 0;
    if (v == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_batch_step<F>, kBatchThreads, 0) !=
                cudaSuccess ||
            v < 1)
            v = 1;
        if (d >= 0 && d < 64) per_sm[d] = v;
    }
    return (unsigned)(v * sm_count());
}

unsigned batch_device_error(bool clear) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_batch_error, sizeof(v));
    if (clear) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_batch_error, &z, sizeof(z));
    }
    return v;
}

void batch_prepare(int dtype) {  // occupancy query outside any stream capture
    if (dtype == PS_F64)
        resident_grid<double>();
    else
        resident_grid<float>();
}

cudaError_t launch_batch_step(const void *dev_table, int parity, int dtype, cudaStream_t s) {
    if (dtype == PS_F64)
        k_batch_step<double><<<resident_grid<double>(), kBatchThreads, 0, s>>>((const char *)dev_table,
                                                                            parity);
    else
        k_batch_step<float><<<resident_grid<float>(), kBatchThreads, 0, s>>>((const char *)dev_table,
                                                                          parity);
    return cudaGetLastError();
}

}  // namespace psd

// FP32 transposed step as a TMA-fed z-march with every read prefetched.
//
// For ybar = dL/dT_{t+1} and the state T = T_t the forward step read (deviation
// storage does not change the step's Jacobian):
//   w[q]      = Ci[q]*ybar[q] at interior q, 0 elsewhere (and outside the grid),
//   Tbar[p]   = ybar[p] + sum_d (w[p-e_d] - 2 w[p] + w[p+e_d]) * K_d         (every p),
//   Cibar[q] += ybar[q] * sum_d (T[q-e_d] - 2 T[q] + T[q+e_d]) * K_d         (interior q),
// with K_d = dt*lam*_d^2.
//
// A CTA owns a 128 x BY x-y tile (one warp per row, four nodes per thread,
// 16-byte accesses) and a chunk of z-planes of the whole grid.  For plane q one
// thread issues four TMA boxes into one ring stage, counted on the stage's one
// mbarrier: T, ybar and Ci with a one-node y halo and a 16-byte x halo, and
// Cibar's own tile (output planes only).  So the kernel's only plain global
// accesses are its 16-byte stores.  w is not staged: each thread forms the ten
// x-y neighbour values of w it needs from the ybar and Ci boxes (FP32 products
// are cheap), and keeps its own w, T and ybar of planes k-1, k, k+1 in
// registers.  One barrier per plane frees the stage of plane k, which takes
// plane k + NST: the copies run NST-1 planes ahead of the arithmetic.
#include <cudaTypedefs.h>

#include <cstdlib>

#include "internal.h"
#include "tma.cuh"
#include "zmarch.h"

namespace psd {

__device__ unsigned g_adj32_error;  // set when an mbarrier wait times out

struct Adj32Params {
    int nx, ny, nz;
    int kchunk, ntx;
    float Kx, Ky, Kz;
};

template <int BY, int NST, int MINB>
__global__ void __launch_bounds__(32 * BY, MINB)
k_adjoint_f32(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmY,
              const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmB,
              float *__restrict__ Tbar, float *__restrict__ Cibar, const Adj32Params p) {
    constexpr int PX = 4, HX = 4, BX = 128, W = BX + 2 * HX, H = BY + 2;
    constexpr unsigned HB = W * H * 4, CB = BX * BY * 4;  // halo box, Cibar box bytes
    constexpr unsigned HBA = (HB + 127) / 128 * 128, CBA = (CB + 127) / 128 * 128;
    constexpr unsigned SB = 3 * HBA + CBA;  // stage bytes
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = (uint64_t *)(smem + NST * SB);
    __shared__ int s_abort;

    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int X0 = (int)(blockIdx.x % p.ntx) * BX, Y0 = (int)(blockIdx.x / p.ntx) * BY;
    const int k0 = (int)blockIdx.y * p.kchunk;
    const int k1 = min(k0 + p.kchunk, p.nz);  // output planes [k0, k1)
    const int nx = p.nx, ny = p.ny, nz = p.nz;

    auto sT = [&](int s) { return (const float *)(smem + s * SB); };
    auto sY = [&](int s) { return (const float *)(smem + s * SB + HBA); };
    auto sC = [&](int s) { return (const float *)(smem + s * SB + 2 * HBA); };
    auto sB = [&](int s) { return (const float *)(smem + s * SB + 3 * HBA); };
    auto issue = [&](int s, int q) {  // plane q into stage s (q = -1 and q = nz read zeros)
        const bool out = q >= k0 && q < k1;
        unsigned char *st = smem + s * SB;
        mbar_expect_tx(&bar[s], 3 * HB + (out ? CB : 0u));
        tma_load_3d(st, &tmT, &bar[s], X0 - HX, Y0 - 1, q);
        tma_load_3d(st + HBA, &tmY, &bar[s], X0 - HX, Y0 - 1, q);
        tma_load_3d(st + 2 * HBA, &tmC, &bar[s], X0 - HX, Y0 - 1, q);
        if (out) tma_load_3d(st + 3 * HBA, &tmB, &bar[s], X0, Y0, q);
    };
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // plane q = k0-1+i lives in stage i % NST
    if (threadIdx.x == 0)
        for (int s = 0; s < NST; ++s)
            if (k0 - 1 + s <= k1) issue(s, k0 - 1 + s);

    unsigned par = 0u;  // bit s: parity of the next completion of stage s
    auto nexts = [](int s) { return s + 1 == NST ? 0 : s + 1; };
    auto acquire = [&](int s) -> bool {
        const unsigned ph = (par >> s) & 1u;
        par ^= 1u << s;
        return mbar_wait(&bar[s], ph);
    };
    // After a timed-out wait: bounded waits for the copies of the last NST planes issued
    // (up to plane q_iss), so that no TMA write lands after the CTA exits.
    auto drain = [&](int q_iss) {
        for (int q = max(k0 - 1, q_iss - NST + 1); q <= q_iss; ++q) {
            const int i = q - (k0 - 1);
            mbar_wait(&bar[i % NST], (unsigned)(i / NST) & 1u);
        }
    };

    const int row = ty + 1, col = HX + lane * PX;
    const int gy = Y0 + ty, gx0 = X0 + lane * PX;
    // interior masks: own nodes, the rows above and below, the nodes left and right
    const bool iy = gy >= 1 && gy <= ny - 2, iyu = gy - 1 >= 1 && gy - 1 <= ny - 2,
               iyd = gy + 1 >= 1 && gy + 1 <= ny - 2;
    bool ix[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) ix[i] = gx0 + i >= 1 && gx0 + i <= nx - 2;
    const bool ixl = gx0 - 1 >= 1 && gx0 - 1 <= nx - 2, ixr = gx0 + PX >= 1 && gx0 + PX <= nx - 2;
    const bool row_out = gy <= ny - 1, all_x = gx0 + PX - 1 <= nx - 1;
    const bool all_in = ix[0] && ix[PX - 1];

    // own w of plane q from its stage
    auto w_own = [&](int s, int q, const float4 &y) -> float4 {
        const float4 c = *(const float4 *)(sC(s) + row * W + col);
        const bool iz = q >= 1 && q <= nz - 2 && iy;
        float4 w;
        w.x = (iz && ix[0]) ? c.x * y.x : 0.f;
        w.y = (iz && ix[1]) ? c.y * y.y : 0.f;
        w.z = (iz && ix[2]) ? c.z * y.z : 0.f;
        w.w = (iz && ix[3]) ? c.w * y.w : 0.f;
        return w;
    };

    // ---- prologue: planes k0-1 and k0
    int s_m = 0, s_c = 1 % NST;
    bool ok = acquire(s_m);
    ok = acquire(s_c) && ok;
    float4 tm = *(const float4 *)(sT(s_m) + row * W + col);
    float4 wm = w_own(s_m, k0 - 1, *(const float4 *)(sY(s_m) + row * W + col));
    float4 tc = *(const float4 *)(sT(s_c) + row * W + col);
    float4 yc = *(const float4 *)(sY(s_c) + row * W + col);
    float4 wc = w_own(s_c, k0, yc);
    if (!ok) {
        s_abort = 1;
        atomicOr(&g_adj32_error, 1u);
    }
    __syncthreads();  // every thread is done with plane k0-1's stage
    if (s_abort) {
        drain(min(k0 - 2 + NST, k1));
        return;
    }
    if (threadIdx.x == 0 && k0 - 1 + NST <= k1) issue(s_m, k0 - 1 + NST);

    const float Kx = p.Kx, Ky = p.Ky, Kz = p.Kz;
    int64_t base = (int64_t)gx0 + (int64_t)nx * ((int64_t)gy + (int64_t)ny * k0);
    const int64_t plane = (int64_t)nx * ny;
    for (int k = k0; k < k1; ++k, base += plane) {
        const int s_n = nexts(s_c);  // stage of plane k+1
        ok = acquire(s_n);
        const float *Tk = sT(s_c), *Yk = sY(s_c), *Ck = sC(s_c);
        const float4 tp = *(const float4 *)(sT(s_n) + row * W + col);
        const float4 yp = *(const float4 *)(sY(s_n) + row * W + col);
        const float4 wp = w_own(s_n, k + 1, yp);
        if (row_out) {
            const bool iz = k >= 1 && k <= nz - 2;
            // x-y neighbours of w in plane k
            const float4 yu = *(const float4 *)(Yk + (row - 1) * W + col);
            const float4 cu = *(const float4 *)(Ck + (row - 1) * W + col);
            const float4 yd = *(const float4 *)(Yk + (row + 1) * W + col);
            const float4 cd = *(const float4 *)(Ck + (row + 1) * W + col);
            const bool mu = iz && iyu, md = iz && iyd;
            float wu[PX], wd[PX];
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                wu[i] = (mu && ix[i]) ? (&cu.x)[i] * (&yu.x)[i] : 0.f;
                wd[i] = (md && ix[i]) ? (&cd.x)[i] * (&yd.x)[i] : 0.f;
            }
            const float wl = (iz && iy && ixl) ? Ck[row * W + col - 1] * Yk[row * W + col - 1] : 0.f;
            const float wr = (iz && iy && ixr) ? Ck[row * W + col + PX] * Yk[row * W + col + PX] : 0.f;
            float4 tb;
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                const float c = (&wc.x)[i];
                const float xm = i == 0 ? wl : (&wc.x)[i - 1];
                const float xp = i == PX - 1 ? wr : (&wc.x)[i + 1];
                const float d2x = (xp - c) - (c - xm);
                const float d2y = (wd[i] - c) - (c - wu[i]);
                const float d2z = ((&wp.x)[i] - c) - (c - (&wm.x)[i]);
                (&tb.x)[i] = (&yc.x)[i] + ((d2x * Kx + d2y * Ky) + d2z * Kz);
            }
            if (all_x) {
                *(float4 *)(Tbar + base) = tb;
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i)
                    if (gx0 + i <= nx - 1) Tbar[base + i] = (&tb.x)[i];
            }
            if (iz && iy) {
                const float4 tu = *(const float4 *)(Tk + (row - 1) * W + col);
                const float4 td = *(const float4 *)(Tk + (row + 1) * W + col);
                const float tl = Tk[row * W + col - 1], tr = Tk[row * W + col + PX];
                float4 cb = *(const float4 *)(sB(s_c) + ty * BX + lane * PX);
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    const float t = (&tc.x)[i];
                    const float txm = i == 0 ? tl : (&tc.x)[i - 1];
                    const float txp = i == PX - 1 ? tr : (&tc.x)[i + 1];
                    const float t2x = (txp - t) - (t - txm);
                    const float t2y = ((&td.x)[i] - t) - (t - (&tu.x)[i]);
                    const float t2z = ((&tp.x)[i] - t) - (t - (&tm.x)[i]);
                    const float L = (t2x * Kx + t2y * Ky) + t2z * Kz;
                    (&cb.x)[i] = (&cb.x)[i] + (&yc.x)[i] * L;
                }
                if (all_in) {
                    *(float4 *)(Cibar + base) = cb;
                } else {
#pragma unroll
                    for (int i = 0; i < PX; ++i)
                        if (ix[i]) Cibar[base + i] = (&cb.x)[i];
                }
            }
        }
        if (!ok) {
            s_abort = 1;
            atomicOr(&g_adj32_error, 1u);
        }
        __syncthreads();  // every thread is done with plane k's stage
        if (s_abort) {
            drain(min(k - 1 + NST, k1));
            return;
        }
        if (threadIdx.x == 0 && k + NST <= k1) issue(s_c, k + NST);
        tm = tc;
        tc = tp;
        yc = yp;
        wm = wc;
        wc = wp;
        s_c = s_n;
    }
}

template <int BY, int NST, int MINB>
static cudaError_t launch_adj32_t(float *Tbar, float *Cibar, const float *ybar, const float *T,
                                  const float *Ci, Grid3 g, Adj32Params p, int kchunk, cudaStream_t s) {
    constexpr int BX = 128, W = BX + 8, H = BY + 2;
    constexpr unsigned HBA = (W * H * 4 + 127) / 128 * 128, CBA = (BX * BY * 4 + 127) / 128 * 128;
    constexpr size_t smem = NST * (3 * HBA + CBA) + NST * 8;
    static bool attr_done[64] = {false};
    const int dev = current_device();
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_adjoint_f32<BY, NST, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    CUtensorMap mT, mY, mC, mB;
    if (!make_tensor_map_3d(&mT, T, 4, g, W, H) || !make_tensor_map_3d(&mY, ybar, 4, g, W, H) ||
        !make_tensor_map_3d(&mC, Ci, 4, g, W, H) || !make_tensor_map_3d(&mB, Cibar, 4, g, BX, BY))
        return cudaErrorInvalidValue;
    const int64_t ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY, tiles = ntx * nty;
    if (kchunk <= 0) {
        // 16-plane chunks (each chunk re-reads two planes); 32 where 16 would leave
        // fewer than four waves of CTAs and 32 still gives one and a half.  Measured:
        // 128^3 best at 16, 256^3 at 32 (5% ahead of 16), 512^3 and 768^3 at 16 (1-4%).
        const int64_t slots = (int64_t)MINB * sm_count(), cols = g.nz * tiles;
        kchunk = (cols < 4 * 16 * slots && 2 * cols >= 3 * 32 * slots) ? 32 : 16;
    }
    const int64_t gz = (g.nz + kchunk - 1) / kchunk;
    if (tiles > 0x7fffffffLL || gz > 65535) return cudaErrorInvalidConfiguration;
    p.nx = (int)g.nx;
    p.ny = (int)g.ny;
    p.nz = (int)g.nz;
    p.ntx = (int)ntx;
    p.kchunk = kchunk;
    k_adjoint_f32<BY, NST, MINB><<<dim3((unsigned)tiles, (unsigned)gz, 1), 32 * BY, smem, s>>>(
        mT, mY, mC, mB, Tbar, Cibar, p);
    return cudaGetLastError();
}

bool adjoint_f32_supported(Grid3 g, const void *const *ptrs, int nptr) {
    uintptr_t acc = 0;
    for (int i = 0; i < nptr; ++i) acc |= (uintptr_t)ptrs[i];
    if (acc & 15u) return false;
    if ((g.nx * 4) % 16 != 0) return false;
    // 32-bit plane and row indices in the kernel; TMA coordinates are 32-bit as well
    if (g.nx > (1LL << 31) - 256 || g.ny > (1LL << 31) - 64 || g.nz > (1LL << 31) - 64) return false;
    return zmarch_supported(g, 4, ptrs[0], ptrs[0], ptrs[0]);
}

cudaError_t launch_adjoint_f32_tma(float *Tbar, float *Cibar, const float *ybar, const float *T,
                                   const float *Ci, StepCoef c, Grid3 g, cudaStream_t s) {
    Adj32Params p{};
    p.Kx = (float)(c.dtlam * c.ax);
    p.Ky = (float)(c.dtlam * c.ay);
    p.Kz = (float)(c.dtlam * c.az);
    const char *v = getenv("PS_ADJ_KCHUNK");
    const int kchunk = v ? atoi(v) : 0;
    // 4-row tiles, four stages (three planes of copies ahead), four CTAs per SM
    // (48 KB of shared memory each); measured at 256^3 and 512^3 against 8-row
    // tiles with four or five stages at two CTAs per SM and 4-row tiles with six
    // stages at three: equal at 512^3, 1-8% faster at 256^3.
    return launch_adj32_t<4, 4, 4>(Tbar, Cibar, ybar, T, Ci, g, p, kchunk, s);
}

unsigned adjoint_f32_device_error(bool clear) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_adj32_error, sizeof(v));
    if (clear) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_adj32_error, &z, sizeof(z));
    }
    return v;
}

}  // namespace psd

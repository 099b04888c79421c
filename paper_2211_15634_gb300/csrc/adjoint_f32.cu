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


#include "adj32_node.cuh"
#include "internal.h"
#include "pdl.cuh"
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
    grid_dep_wait();  // the previous launch's writes (and its reads of Tbar) are complete
    grid_dep_launch();

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
        w.x = a32_w(c.x, y.x, iz && ix[0]);
        w.y = a32_w(c.y, y.y, iz && ix[1]);
        w.z = a32_w(c.z, y.z, iz && ix[2]);
        w.w = a32_w(c.w, y.w, iz && ix[3]);
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
                wu[i] = a32_w((&cu.x)[i], (&yu.x)[i], mu && ix[i]);
                wd[i] = a32_w((&cd.x)[i], (&yd.x)[i], md && ix[i]);
            }
            const float wl = a32_w(Ck[row * W + col - 1], Yk[row * W + col - 1], iz && iy && ixl);
            const float wr = a32_w(Ck[row * W + col + PX], Yk[row * W + col + PX], iz && iy && ixr);
            float4 tb;
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                const float c = (&wc.x)[i];
                const float xm = i == 0 ? wl : (&wc.x)[i - 1];
                const float xp = i == PX - 1 ? wr : (&wc.x)[i + 1];
                (&tb.x)[i] = a32_tbar((&yc.x)[i], a32_lap(c, xm, xp, wu[i], wd[i], (&wm.x)[i], (&wp.x)[i],
                                                          Kx, Ky, Kz));
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
                    (&cb.x)[i] = a32_cibar((&cb.x)[i], (&yc.x)[i],
                                           a32_lap(t, txm, txp, (&tu.x)[i], (&td.x)[i], (&tm.x)[i],
                                                   (&tp.x)[i], Kx, Ky, Kz));
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

// Two transposed steps per pass (temporal blocking of depth 2).  With y2 = dL/dT_{t+2},
// the first transposed step (state S1 = T_{t+1}) gives y1 = y2 + L(C*y2) and adds
// y2*L(S1) to Cibar; the second (state S0 = T_t) gives Tbar = y1 + L(C*y1) and adds
// y1*L(S0).  y1 never leaves the chip.  A CTA owns a 128 x 8 tile and a chunk of
// output planes [k0, k1).  Iteration k computes, in one phase, y1 of plane k+1 on the
// tile and its one-node cross ring (own nodes in registers, all of it into one of two
// shared y1 tiles), and Tbar and Cibar of plane k (y1 tile of plane k complete since
// the last barrier).  y1 on the ring needs C*y2 two nodes out, so ybar and Ci arrive
// as boxes with a 2-row y halo (ring NYC: plane q read in iterations q-2 .. q); the
// states and Cibar as boxes with a 1-row halo and Cibar's own tile (ring NS: plane q
// read in iterations q-1, q).  Per-node arithmetic is adj32_node.cuh's: the result is
// bit for bit that of two one-step launches.  Traffic per pass: read ybar, S1, S0, Ci,
// Cibar, write Tbar, Cibar - 7 arrays for two steps instead of 12.
template <int NYC, int NS>
__global__ void __launch_bounds__(256, 2)
k_adjoint2_f32(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmC,
               const __grid_constant__ CUtensorMap tmS1, const __grid_constant__ CUtensorMap tmS0,
               const __grid_constant__ CUtensorMap tmB, float *__restrict__ Tbar,
               float *__restrict__ Cibar, const Adj32Params p) {
    constexpr int BY = 8, PX = 4, BX = 128, W = BX + 8, HY = BY + 4, HS = BY + 2;
    constexpr unsigned YB = W * HY * 4, SB = W * HS * 4, CB = BX * BY * 4;
    constexpr unsigned YBA = (YB + 127) / 128 * 128, SBA = (SB + 127) / 128 * 128;
    constexpr unsigned YCS = 2 * YBA, SS = 2 * SBA + CB;  // stage bytes of the two rings
    static_assert(NYC >= 4 && NS >= 3, "ring depths");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *ringY = smem, *ringS = smem + NYC * YCS, *tiles = ringS + NS * SS;
    uint64_t *barY = (uint64_t *)(tiles + 2 * SBA), *barS = barY + NYC;
    __shared__ int s_abort;
    grid_dep_wait();
    grid_dep_launch();

    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int X0 = (int)(blockIdx.x % p.ntx) * BX, Y0 = (int)(blockIdx.x / p.ntx) * BY;
    const int k0 = (int)blockIdx.y * p.kchunk;
    const int k1 = min(k0 + p.kchunk, p.nz);  // output planes [k0, k1)
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const float Kx = p.Kx, Ky = p.Ky, Kz = p.Kz;

    auto Yb = [&](int s) { return (const float *)(ringY + s * YCS); };
    auto Cb = [&](int s) { return (const float *)(ringY + s * YCS + YBA); };
    auto S1b = [&](int s) { return (const float *)(ringS + s * SS); };
    auto S0b = [&](int s) { return (const float *)(ringS + s * SS + SBA); };
    auto Bb = [&](int s) { return (const float *)(ringS + s * SS + 2 * SBA); };
    auto tile = [&](int q) { return (float *)(tiles + ((q - k0) & 1) * SBA); };  // y1 of plane q
    // ybar, Ci of planes k0-2 .. k1+1 in stage (q - (k0-2)) % NYC; S1, S0 of planes
    // k0-1 .. k1 (and Cibar of the output planes) in stage (q - (k0-1)) % NS
    const int qYmax = k1 + 1, qSmax = k1;
    auto issueY = [&](int q) {
        const int s = (q - (k0 - 2)) % NYC;
        unsigned char *st = ringY + s * YCS;
        mbar_expect_tx(&barY[s], 2 * YB);
        tma_load_3d(st, &tmY, &barY[s], X0 - 4, Y0 - 2, q);
        tma_load_3d(st + YBA, &tmC, &barY[s], X0 - 4, Y0 - 2, q);
    };
    auto issueS = [&](int q) {
        const int s = (q - (k0 - 1)) % NS;
        const bool out = q >= k0 && q < k1;
        unsigned char *st = ringS + s * SS;
        mbar_expect_tx(&barS[s], 2 * SB + (out ? CB : 0u));
        tma_load_3d(st, &tmS1, &barS[s], X0 - 4, Y0 - 1, q);
        tma_load_3d(st + SBA, &tmS0, &barS[s], X0 - 4, Y0 - 1, q);
        if (out) tma_load_3d(st + 2 * SBA, &tmB, &barS[s], X0, Y0, q);
    };
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NYC; ++s) mbar_init(&barY[s], 1);
        for (int s = 0; s < NS; ++s) mbar_init(&barS[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = k0 - 2; q <= min(k0 - 3 + NYC, qYmax); ++q) issueY(q);
        for (int q = k0 - 1; q <= min(k0 - 2 + NS, qSmax); ++q) issueS(q);
    }
    unsigned ypar = 0u, spar = 0u;  // bit s: parity of the next completion of stage s
    auto waitY = [&](int q) -> bool {
        const int s = (q - (k0 - 2)) % NYC;
        const unsigned ph = (ypar >> s) & 1u;
        ypar ^= 1u << s;
        return mbar_wait(&barY[s], ph);
    };
    auto waitS = [&](int q) -> bool {
        const int s = (q - (k0 - 1)) % NS;
        const unsigned ph = (spar >> s) & 1u;
        spar ^= 1u << s;
        return mbar_wait(&barS[s], ph);
    };
    // after a timed-out wait: bounded waits for the copies still in flight (ybar/Ci
    // planes up to qy, state planes up to qs), so that no TMA write lands after exit
    auto drain = [&](int qy, int qs) {
        for (int q = max(k0 - 2, qy - NYC + 1); q <= qy; ++q) {
            const int i = q - (k0 - 2);
            mbar_wait(&barY[i % NYC], (unsigned)(i / NYC) & 1u);
        }
        for (int q = max(k0 - 1, qs - NS + 1); q <= qs; ++q) {
            const int i = q - (k0 - 1);
            mbar_wait(&barS[i % NS], (unsigned)(i / NS) & 1u);
        }
    };
    auto sY = [&](int q) { return (q - (k0 - 2)) % NYC; };
    auto sS = [&](int q) { return (q - (k0 - 1)) % NS; };

    // own nodes: rows rY (ybar/Ci boxes) and rS (state boxes, y1 tiles), columns col .. col+3
    const int rY = ty + 2, rS = ty + 1, col = 4 + lane * PX;
    const int gy = Y0 + ty, gx0 = X0 + lane * PX;
    auto inx = [&](int x) { return x >= 1 && x <= nx - 2; };
    auto iny = [&](int y) { return y >= 1 && y <= ny - 2; };
    auto inz = [&](int z) { return z >= 1 && z <= nz - 2; };
    bool ix[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) ix[i] = inx(gx0 + i);
    const bool ixl = inx(gx0 - 1), ixr = inx(gx0 + PX), iy = iny(gy), iyu = iny(gy - 1), iyd = iny(gy + 1);
    const bool row_out = gy <= ny - 1, all_x = gx0 + PX - 1 <= nx - 1, all_in = ix[0] && ix[PX - 1];
    // ring positions of this thread: one on the rows above / below the tile, and for
    // threads 0 .. 15 one on the columns left / right of it
    const int t = threadIdx.x;
    const bool top = t < BX;
    const int rx = X0 + (top ? t : t - BX), ry = top ? Y0 - 1 : Y0 + BY;
    const int rrY = top ? 1 : BY + 2, rrS = top ? 0 : BY + 1, rc = 4 + (top ? t : t - BX);
    const bool hasc = t < 2 * BY;
    const int cx = t < BY ? X0 - 1 : X0 + BX, cy = Y0 + (t < BY ? t : t - BY);
    const int crY = (t < BY ? t : t - BY) + 2, crS = crY - 1, cc = t < BY ? 3 : 4 + BX;

    // y1 of plane q at the own nodes (from ybar/Ci of planes q-1, q, q+1); y2own = ybar there
    auto y1_own = [&](int q, float4 &y2own) -> float4 {
        const float *Yc = Yb(sY(q)), *Cc = Cb(sY(q)), *Ym = Yb(sY(q - 1)), *Cm = Cb(sY(q - 1));
        const float *Yp = Yb(sY(q + 1)), *Cp = Cb(sY(q + 1));
        const int o = rY * W + col;
        const float4 yc4 = *(const float4 *)(Yc + o), cc4 = *(const float4 *)(Cc + o);
        const float4 yu4 = *(const float4 *)(Yc + o - W), cu4 = *(const float4 *)(Cc + o - W);
        const float4 yd4 = *(const float4 *)(Yc + o + W), cd4 = *(const float4 *)(Cc + o + W);
        const float4 ym4 = *(const float4 *)(Ym + o), cm4 = *(const float4 *)(Cm + o);
        const float4 yp4 = *(const float4 *)(Yp + o), cp4 = *(const float4 *)(Cp + o);
        const bool zc = inz(q), zm = inz(q - 1), zp = inz(q + 1);
        const float wl = a32_w(Cc[o - 1], Yc[o - 1], zc && iy && ixl);
        const float wr = a32_w(Cc[o + PX], Yc[o + PX], zc && iy && ixr);
        float wc[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) wc[i] = a32_w((&cc4.x)[i], (&yc4.x)[i], zc && iy && ix[i]);
        float4 out;
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            const float wu = a32_w((&cu4.x)[i], (&yu4.x)[i], zc && iyu && ix[i]);
            const float wd = a32_w((&cd4.x)[i], (&yd4.x)[i], zc && iyd && ix[i]);
            const float wzm = a32_w((&cm4.x)[i], (&ym4.x)[i], zm && iy && ix[i]);
            const float wzp = a32_w((&cp4.x)[i], (&yp4.x)[i], zp && iy && ix[i]);
            const float xm = i == 0 ? wl : wc[i - 1], xp = i == PX - 1 ? wr : wc[i + 1];
            (&out.x)[i] = a32_tbar((&yc4.x)[i], a32_lap(wc[i], xm, xp, wu, wd, wzm, wzp, Kx, Ky, Kz));
        }
        y2own = yc4;
        return out;
    };
    // y1 of plane q at one node (x, y) = box row r, column c
    auto y1_at = [&](int q, int r, int c, int x, int y) -> float {
        const float *Yc = Yb(sY(q)), *Cc = Cb(sY(q)), *Ym = Yb(sY(q - 1)), *Cm = Cb(sY(q - 1));
        const float *Yp = Yb(sY(q + 1)), *Cp = Cb(sY(q + 1));
        const int o = r * W + c;
        const bool zc = inz(q), yin = iny(y), xin = inx(x);
        const float wc = a32_w(Cc[o], Yc[o], zc && yin && xin);
        const float wxm = a32_w(Cc[o - 1], Yc[o - 1], zc && yin && inx(x - 1));
        const float wxp = a32_w(Cc[o + 1], Yc[o + 1], zc && yin && inx(x + 1));
        const float wym = a32_w(Cc[o - W], Yc[o - W], zc && iny(y - 1) && xin);
        const float wyp = a32_w(Cc[o + W], Yc[o + W], zc && iny(y + 1) && xin);
        const float wzm = a32_w(Cm[o], Ym[o], inz(q - 1) && yin && xin);
        const float wzp = a32_w(Cp[o], Yp[o], inz(q + 1) && yin && xin);
        return a32_tbar(Yc[o], a32_lap(wc, wxm, wxp, wym, wyp, wzm, wzp, Kx, Ky, Kz));
    };
    // y1 of plane q on the tile and its ring into the tile of plane q; own values returned
    auto y1_plane = [&](int q, float4 &y2own) -> float4 {
        float *T1 = tile(q);
        const float4 v = y1_own(q, y2own);
        *(float4 *)(T1 + rS * W + col) = v;
        T1[rrS * W + rc] = y1_at(q, rrY, rc, rx, ry);
        if (hasc) T1[crS * W + cc] = y1_at(q, crY, cc, cx, cy);
        return v;
    };
    // w1 = C*y1 at the own nodes of plane q
    auto w1_own = [&](int q, const float4 &y1) -> float4 {
        const float4 c4 = *(const float4 *)(Cb(sY(q)) + rY * W + col);
        const bool z = inz(q) && iy;
        float4 w;
#pragma unroll
        for (int i = 0; i < PX; ++i) (&w.x)[i] = a32_w((&c4.x)[i], (&y1.x)[i], z && ix[i]);
        return w;
    };

    // ---- prologue: y1 own of plane k0-1, y1 tile of plane k0, state z-queues
    bool ok = waitY(k0 - 2);
    ok = waitY(k0 - 1) && ok;
    ok = waitY(k0) && ok;
    ok = waitY(k0 + 1) && ok;
    ok = waitS(k0 - 1) && ok;
    ok = waitS(k0) && ok;
    float4 y2m, y2c;
    float4 y1m = y1_own(k0 - 1, y2m);
    float4 w1m = w1_own(k0 - 1, y1m);
    float4 y1c = y1_plane(k0, y2c);
    float4 w1c = w1_own(k0, y1c);
    float4 s1m = *(const float4 *)(S1b(sS(k0 - 1)) + rS * W + col);
    float4 s0m = *(const float4 *)(S0b(sS(k0 - 1)) + rS * W + col);
    float4 s1c = *(const float4 *)(S1b(sS(k0)) + rS * W + col);
    float4 s0c = *(const float4 *)(S0b(sS(k0)) + rS * W + col);
    if (!ok) {
        s_abort = 1;
        atomicOr(&g_adj32_error, 1u);
    }
    __syncthreads();  // y1 tile of plane k0 complete; planes k0-2, k0-1 no longer read
    if (s_abort) {
        drain(min(k0 - 3 + NYC, qYmax), min(k0 - 2 + NS, qSmax));
        return;
    }
    if (threadIdx.x == 0) {
        if (k0 - 2 + NYC <= qYmax) issueY(k0 - 2 + NYC);
        if (k0 - 1 + NYC <= qYmax) issueY(k0 - 1 + NYC);
        if (k0 - 1 + NS <= qSmax) issueS(k0 - 1 + NS);
    }

    int64_t base = (int64_t)gx0 + (int64_t)nx * ((int64_t)gy + (int64_t)ny * k0);
    const int64_t plane = (int64_t)nx * ny;
    for (int k = k0; k < k1; ++k, base += plane) {
        ok = waitY(k + 2);
        ok = waitS(k + 1) && ok;
        // y1 of plane k+1 (tile and ring) and its own w1
        float4 y2p;
        const float4 y1p = y1_plane(k + 1, y2p);
        const float4 w1p = w1_own(k + 1, y1p);
        const float4 s1p = *(const float4 *)(S1b(sS(k + 1)) + rS * W + col);
        const float4 s0p = *(const float4 *)(S0b(sS(k + 1)) + rS * W + col);
        if (row_out) {
            // Tbar of plane k: y1 + L(C*y1), x-y neighbours from the y1 tile of plane k
            const float *T1 = tile(k), *Ck = Cb(sY(k));
            const int o1 = rS * W + col, oY = rY * W + col;
            const bool iz = inz(k);
            const float4 yu4 = *(const float4 *)(T1 + o1 - W), yd4 = *(const float4 *)(T1 + o1 + W);
            const float4 cu4 = *(const float4 *)(Ck + oY - W), cd4 = *(const float4 *)(Ck + oY + W);
            const float wl = a32_w(Ck[oY - 1], T1[o1 - 1], iz && iy && ixl);
            const float wr = a32_w(Ck[oY + PX], T1[o1 + PX], iz && iy && ixr);
            float4 tb;
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                const float wu = a32_w((&cu4.x)[i], (&yu4.x)[i], iz && iyu && ix[i]);
                const float wd = a32_w((&cd4.x)[i], (&yd4.x)[i], iz && iyd && ix[i]);
                const float c = (&w1c.x)[i];
                const float xm = i == 0 ? wl : (&w1c.x)[i - 1], xp = i == PX - 1 ? wr : (&w1c.x)[i + 1];
                (&tb.x)[i] = a32_tbar((&y1c.x)[i],
                                      a32_lap(c, xm, xp, wu, wd, (&w1m.x)[i], (&w1p.x)[i], Kx, Ky, Kz));
            }
            if (all_x) {
                *(float4 *)(Tbar + base) = tb;
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i)
                    if (gx0 + i <= nx - 1) Tbar[base + i] = (&tb.x)[i];
            }
            // Cibar of plane k: + y2*L(S1), then + y1*L(S0)
            if (iz && iy) {
                const float *A = S1b(sS(k)), *B = S0b(sS(k));
                const float4 au = *(const float4 *)(A + o1 - W), ad = *(const float4 *)(A + o1 + W);
                const float4 bu = *(const float4 *)(B + o1 - W), bd = *(const float4 *)(B + o1 + W);
                const float al = A[o1 - 1], ar = A[o1 + PX], bl = B[o1 - 1], br = B[o1 + PX];
                float4 cb = *(const float4 *)(Bb(sS(k)) + ty * BX + lane * PX);
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    const float a = (&s1c.x)[i], b = (&s0c.x)[i];
                    const float axm = i == 0 ? al : (&s1c.x)[i - 1], axp = i == PX - 1 ? ar : (&s1c.x)[i + 1];
                    const float bxm = i == 0 ? bl : (&s0c.x)[i - 1], bxp = i == PX - 1 ? br : (&s0c.x)[i + 1];
                    float v = a32_cibar((&cb.x)[i], (&y2c.x)[i],
                                        a32_lap(a, axm, axp, (&au.x)[i], (&ad.x)[i], (&s1m.x)[i], (&s1p.x)[i],
                                                Kx, Ky, Kz));
                    (&cb.x)[i] = a32_cibar(v, (&y1c.x)[i],
                                           a32_lap(b, bxm, bxp, (&bu.x)[i], (&bd.x)[i], (&s0m.x)[i],
                                                   (&s0p.x)[i], Kx, Ky, Kz));
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
        __syncthreads();  // y1 tile of plane k+1 complete; plane k's stages no longer read
        if (s_abort) {
            drain(min(k - 1 + NYC, qYmax), min(k - 1 + NS, qSmax));
            return;
        }
        if (threadIdx.x == 0) {
            if (k + NYC <= qYmax) issueY(k + NYC);
            if (k + NS <= qSmax) issueS(k + NS);
        }
        y2m = y2c;
        y2c = y2p;
        y1m = y1c;
        y1c = y1p;
        w1m = w1c;
        w1c = w1p;
        s1m = s1c;
        s1c = s1p;
        s0m = s0c;
        s0c = s0p;
    }
}

template <int NYC, int NS>
static cudaError_t launch_adj2_t(float *Tbar, float *Cibar, const float *ybar, const float *S1,
                                 const float *S0, const float *Ci, Grid3 g, Adj32Params p, int kchunk,
                                 cudaStream_t s) {
    constexpr int BY = 8, BX = 128, W = BX + 8;
    constexpr unsigned YBA = (W * (BY + 4) * 4 + 127) / 128 * 128, SBA = (W * (BY + 2) * 4 + 127) / 128 * 128;
    constexpr size_t smem = NYC * 2 * YBA + NS * (2 * SBA + BX * BY * 4) + 2 * SBA + (NYC + NS) * 8;
    static unsigned attr_gen[64] = {0};
    cudaError_t ae;
    if (!set_smem_attr_once((const void *)k_adjoint2_f32<NYC, NS>, (int)smem, attr_gen, &ae)) return ae;
    CUtensorMap mY, mC, mS1, mS0, mB;
    if (!make_tensor_map_3d(&mY, ybar, 4, g, W, BY + 4) || !make_tensor_map_3d(&mC, Ci, 4, g, W, BY + 4) ||
        !make_tensor_map_3d(&mS1, S1, 4, g, W, BY + 2) || !make_tensor_map_3d(&mS0, S0, 4, g, W, BY + 2) ||
        !make_tensor_map_3d(&mB, Cibar, 4, g, BX, BY))
        return cudaErrorInvalidValue;
    const int64_t ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY, tiles = ntx * nty;
    if (kchunk <= 0) kchunk = 32;  // each chunk re-reads four planes and recomputes two of y1
    const int64_t gz = (g.nz + kchunk - 1) / kchunk;
    if (tiles > 0x7fffffffLL || gz > 65535) return cudaErrorInvalidConfiguration;
    p.nx = (int)g.nx;
    p.ny = (int)g.ny;
    p.nz = (int)g.nz;
    p.ntx = (int)ntx;
    p.kchunk = kchunk;
    return launch_pdl(k_adjoint2_f32<NYC, NS>, dim3((unsigned)tiles, (unsigned)gz, 1), dim3(256), smem, s, mY, mC,
                      mS1, mS0, mB, Tbar, Cibar, p);
}

cudaError_t launch_adjoint2_f32(float *Tbar, float *Cibar, const float *ybar, const float *S1,
                                const float *S0, const float *Ci, StepCoef c, Grid3 g, cudaStream_t s) {
    Adj32Params p{};
    p.Kx = (float)(c.dtlam * c.ax);
    p.Ky = (float)(c.dtlam * c.ay);
    p.Kz = (float)(c.dtlam * c.az);
    const int kchunk = launch_override(PS_OVERRIDE_ADJ_KCHUNK);
    return launch_adj2_t<4, 3>(Tbar, Cibar, ybar, S1, S0, Ci, g, p, kchunk, s);
}

template <int BY, int NST, int MINB>
static cudaError_t launch_adj32_t(float *Tbar, float *Cibar, const float *ybar, const float *T,
                                  const float *Ci, Grid3 g, Adj32Params p, int kchunk, cudaStream_t s) {
    constexpr int BX = 128, W = BX + 8, H = BY + 2;
    constexpr unsigned HBA = (W * H * 4 + 127) / 128 * 128, CBA = (BX * BY * 4 + 127) / 128 * 128;
    constexpr size_t smem = NST * (3 * HBA + CBA) + NST * 8;
    static unsigned attr_gen[64] = {0};
    cudaError_t ae;
    if (!set_smem_attr_once((const void *)k_adjoint_f32<BY, NST, MINB>, (int)smem, attr_gen, &ae)) return ae;
    CUtensorMap mT, mY, mC, mB;
    if (!make_tensor_map_3d(&mT, T, 4, g, W, H) || !make_tensor_map_3d(&mY, ybar, 4, g, W, H) ||
        !make_tensor_map_3d(&mC, Ci, 4, g, W, H) || !make_tensor_map_3d(&mB, Cibar, 4, g, BX, BY))
        return cudaErrorInvalidValue;
    const int64_t ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY, tiles = ntx * nty;
    if (kchunk <= 0) {
        // One wave when it takes chunks of 32-96 planes: every tile's z-range split into
        // as many chunks as there are CTA slots per tile, all CTAs resident at once (no
        // tail).  Else 16-plane chunks (each chunk re-reads two planes); 32 where 16
        // would leave fewer than four waves of CTAs and 32 still gives one and a half.
        // Measured: 128^3 best at 16, 256^3 at 64 (one wave; 4.5% ahead of 32, 8% of
        // 16), 512^3 and 768^3 at 16-24 (within 1%).
        const int64_t slots = (int64_t)MINB * sm_count(), cols = g.nz * tiles;
        const int64_t per_tile = tiles > 0 ? slots / tiles : 0;
        const int64_t one_wave = per_tile > 0 ? (g.nz + per_tile - 1) / per_tile : 0;
        if (one_wave >= 32 && one_wave <= 96)
            kchunk = (int)one_wave;
        else
            kchunk = (cols < 4 * 16 * slots && 2 * cols >= 3 * 32 * slots) ? 32 : 16;
    }
    const int64_t gz = (g.nz + kchunk - 1) / kchunk;
    if (tiles > 0x7fffffffLL || gz > 65535) return cudaErrorInvalidConfiguration;
    p.nx = (int)g.nx;
    p.ny = (int)g.ny;
    p.nz = (int)g.nz;
    p.ntx = (int)ntx;
    p.kchunk = kchunk;
    return launch_pdl(k_adjoint_f32<BY, NST, MINB>, dim3((unsigned)tiles, (unsigned)gz, 1), dim3(32 * BY), smem,
                      s, mT, mY, mC, mB, Tbar, Cibar, p);
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
    const int kchunk = launch_override(PS_OVERRIDE_ADJ_KCHUNK);
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

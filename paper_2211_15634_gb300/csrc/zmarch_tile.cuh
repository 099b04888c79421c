// Body of the TMA-fed z-march step (one CTA, one x-y tile, a chunk of planes),
// shared by the single-grid kernel k_zmarch (zmarch.cu) and the batched kernel
// k_batch_zmarch (batch_tma.cu), so that a batched problem is stepped by the
// very same arithmetic as a single grid.
//
// A CTA owns one x-y tile of BX x BY nodes (BX = LPR threads * PX nodes per
// thread, LPR = 32: one warp per tile row; LPR = 16: two rows per warp, for
// narrow grids) and a chunk of z-planes.  For every plane a
// single thread issues one TMA box load of the tile plus a one-node halo in
// y and a 16-byte halo in x (so every box starts on a 16-byte boundary) into
// a ring of NST shared-memory stages, together with the box of Ci of the same
// plane (output planes only), both counted on the stage's one mbarrier.  Each
// thread keeps its PX centre values of planes k-1, k, k+1 in registers (the
// z-neighbours) and reads x/y neighbours of plane k from shared memory, so
// every T value is read from HBM once (plus halos that mostly hit in L2).
// T2 is written with 16-byte stores.  Boundary nodes are never written.
// The compensated FP32 mode stages the correction field E of its two-float
// state like T (same box, same stage) and writes E2 beside T2.
#pragma once

#include <cuda.h>

#include "emu64.cuh"
#include "node.cuh"
#include "tma.cuh"
#include "zmarch.h"

namespace psd {

template <int MODE>
struct ZTraits;
template <>
struct ZTraits<Z_F64_EMU_ISO> {
    using E = double;
    using V = double2;
    static constexpr int PX = 2;
};
template <>
struct ZTraits<Z_F64_EMU_ANISO> : ZTraits<Z_F64_EMU_ISO> {};
template <>
struct ZTraits<Z_F64_NATIVE> : ZTraits<Z_F64_EMU_ISO> {};
template <>
struct ZTraits<Z_F64_EMU_ISO_DMUL> : ZTraits<Z_F64_EMU_ISO> {};
template <>
struct ZTraits<Z_F64_SCALED> : ZTraits<Z_F64_EMU_ISO> {};
template <>
struct ZTraits<Z_F64_SCALED4> {
    using E = double;
    using V = double4;
    static constexpr int PX = 4;
};
template <>
struct ZTraits<Z_F32> {
    using E = float;
    using V = float4;
    static constexpr int PX = 4;
};
template <>
struct ZTraits<Z_F32_COMP> : ZTraits<Z_F32> {};

template <typename V, typename E>
__device__ __forceinline__ E vget(const V &v, int i) {
    return reinterpret_cast<const E *>(&v)[i];
}

// One CTA (BY * LPR threads): output planes [k0, k1) of the BX x BY tile at (X0, Y0) (the
// tile's node coordinates, boundary included; only interior nodes are written, and with
// kBnd the x and y boundary nodes of those planes too, as copies of T's).
// tmT / tmC: tensor maps of T (box W x H) and Ci (box BX x BY), in parameter or
// global memory.  Rows are p.pitch elements apart, planes p.pitch * p.ny.
// Z_F32_COMP (two-float state D + E): tmE maps E (box W x H, staged with T in the same
// stage) and E2v receives the new correction field; other modes ignore both.
// A timed-out wait sets bit 0 of *err and the CTA leaves after draining its copies.
template <int MODE, int BY, int NST, int LPR = 32, bool kBnd = false>
__device__ __forceinline__ void zmarch_tile(const CUtensorMap *tmT, const CUtensorMap *tmC,
                                            void *__restrict__ T2v, void *__restrict__ E2v,
                                            const ZParams &p, int X0, int Y0, int k0, int k1,
                                            unsigned *err, const CUtensorMap *tmE = nullptr) {
    using Tr = ZTraits<MODE>;
    using E = typename Tr::E;
    using V = typename Tr::V;
    static_assert(LPR == 32 || LPR == 16, "a tile row is one warp or half a warp");
    constexpr int PX = Tr::PX, HX = PX, BX = LPR * PX, W = BX + 2 * HX, H = BY + 2;
    constexpr unsigned TB = W * H * sizeof(E), CB = BX * BY * sizeof(E);
    constexpr unsigned TBA = (TB + 127) / 128 * 128, CBA = (CB + 127) / 128 * 128;
    constexpr bool kComp = MODE == Z_F32_COMP;
    constexpr unsigned EBA = kComp ? TBA : 0u;  // E boxes (two-float state) after the Ci boxes
    extern __shared__ __align__(128) unsigned char smem[];
    E *sT = (E *)smem;
    E *sC = (E *)(smem + NST * TBA);
    E *sE = (E *)(smem + NST * (TBA + CBA));
    uint64_t *bar = (uint64_t *)(smem + NST * (TBA + CBA + EBA));
    __shared__ int s_abort;

    const int lane = threadIdx.x % LPR, ty = threadIdx.x / LPR;  // column group, tile row

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Plane q (q = k0-1 .. k1) lives in stage (q - (k0-1)) % NST: its T box, and its Ci
    // box when it is an output plane, counted on the stage's one mbarrier.
    constexpr unsigned TSTRIDE = TBA / sizeof(E), CSTRIDE = CBA / sizeof(E);
    auto issue = [&](int s, int q) {
        const bool ci = q >= k0 && q < k1;
        mbar_expect_tx(&bar[s], TB + (ci ? CB : 0u) + (kComp ? TB : 0u));
        tma_load_3d(sT + s * TSTRIDE, tmT, &bar[s], X0 - HX, Y0 - 1, q);
        if (ci) tma_load_3d(sC + s * CSTRIDE, tmC, &bar[s], X0, Y0, q);
        if constexpr (kComp) tma_load_3d(sE + s * TSTRIDE, tmE, &bar[s], X0 - HX, Y0 - 1, q);
    };
    if (threadIdx.x == 0)
        for (int s = 0; s < NST; ++s)
            if (k0 - 1 + s <= k1) issue(s, k0 - 1 + s);
    // bit s of tpar is the parity of the next completion of stage s
    unsigned tpar = 0u;
    auto tnext = [](int s) { return s + 1 == NST ? 0 : s + 1; };
    auto acquire = [&](int s) -> bool {
        const unsigned ph = (tpar >> s) & 1u;
        tpar ^= 1u << s;
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
    bool ok = acquire(0);
    V qm = *(const V *)(sT + row * W + col);
    V eqm{}, eqc{};  // E of planes k-1 and k at the own nodes (two-float state)
    if constexpr (kComp) eqm = *(const V *)(sE + row * W + col);
    ok = acquire(1 % NST) && ok;
    V qc = *(const V *)(sT + (1 % NST) * TSTRIDE + row * W + col);
    if constexpr (kComp) eqc = *(const V *)(sE + (1 % NST) * TSTRIDE + row * W + col);
    if (!ok) {
        s_abort = 1;
        atomicOr(err, 1u);
    }
    __syncthreads();
    if (s_abort) {
        drain(min(k0 - 2 + NST, k1));
        return;
    }
    if (threadIdx.x == 0 && k0 - 1 + NST <= k1) issue(0, k0 - 1 + NST);  // stage 0 held plane k0-1

    const int gy = Y0 + ty;
    const int gx0 = X0 + lane * PX;
    const bool row_ok = gy >= 1 && gy <= p.ny - 2;
    // lanes of this warp that compute (the fast-path vote below runs inside row_ok;
    // with two tile rows per warp, row_ok can differ between the halves)
    const unsigned rmask = LPR == 32 ? 0xffffffffu : __ballot_sync(0xffffffffu, row_ok);
    bool all_x = gx0 >= 1 && gx0 + PX - 1 <= p.nx - 2;
    E *__restrict__ T2 = (E *)T2v;
    E *__restrict__ E2 = (E *)E2v;
    int sk = 1 % NST;  // stage of plane k
    const int64_t plane = p.pitch * p.ny;
    int64_t base = (int64_t)gx0 + p.pitch * ((int64_t)gy + p.ny * (int64_t)k0);  // own nodes, plane k

    for (int k = k0; k < k1; ++k, base += plane) {
        const int sk1 = tnext(sk);
        ok = acquire(sk1);  // plane k+1 (plane k, with its Ci, was acquired before)
        const E *Tk = sT + sk * TSTRIDE;
        const V qn = *(const V *)(sT + sk1 * TSTRIDE + row * W + col);
        const E left = Tk[row * W + col - 1], right = Tk[row * W + col + PX];
        const V up = *(const V *)(Tk + (row - 1) * W + col);
        const V dn = *(const V *)(Tk + (row + 1) * W + col);
        const V civ = *(const V *)(sC + sk * CSTRIDE + ty * BX + lane * PX);
        V eqn{}, eup{}, edn{};  // E of plane k+1 and the y-neighbours of plane k
        E eleft{}, eright{};
        if constexpr (kComp) {
            const E *Ek = sE + sk * TSTRIDE;
            eqn = *(const V *)(sE + sk1 * TSTRIDE + row * W + col);
            eleft = Ek[row * W + col - 1];
            eright = Ek[row * W + col + PX];
            eup = *(const V *)(Ek + (row - 1) * W + col);
            edn = *(const V *)(Ek + (row + 1) * W + col);
        }

        if (row_ok) {
            V cv{};  // E2 at the own nodes (two-float state)
            V out;
            if constexpr (MODE == Z_F64_EMU_ISO || MODE == Z_F64_EMU_ANISO ||
                          MODE == Z_F64_EMU_ISO_DMUL || MODE == Z_F64_SCALED || MODE == Z_F64_SCALED4) {
                constexpr bool kIso = MODE != Z_F64_EMU_ANISO;
                constexpr bool kDmul = MODE == Z_F64_EMU_ISO_DMUL;
                constexpr bool kScaled = MODE == Z_F64_SCALED || MODE == Z_F64_SCALED4;
                unsigned long long c[PX], xm[PX], xp[PX], ym[PX], yp[PX], zm[PX], zp[PX];
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    c[i] = dbits((double)vget<V, E>(qc, i));
                    xm[i] = dbits((double)(i == 0 ? left : vget<V, E>(qc, i - 1)));
                    xp[i] = dbits((double)(i == PX - 1 ? right : vget<V, E>(qc, i + 1)));
                    ym[i] = dbits((double)vget<V, E>(up, i));
                    yp[i] = dbits((double)vget<V, E>(dn, i));
                    zm[i] = dbits((double)vget<V, E>(qm, i));
                    zp[i] = dbits((double)vget<V, E>(qn, i));
                }
                // one check over the 5*PX + 2 distinct values of this thread's PX stencils
                unsigned hw[5 * PX + 1];
                hw[0] = (unsigned)(xm[0] >> 32);
                hw[1] = (unsigned)(xp[PX - 1] >> 32);
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    hw[2 + 4 * i] = (unsigned)(ym[i] >> 32);
                    hw[3 + 4 * i] = (unsigned)(yp[i] >> 32);
                    hw[4 + 4 * i] = (unsigned)(zm[i] >> 32);
                    hw[5 + 4 * i] = (unsigned)(zp[i] >> 32);
                }
#pragma unroll
                for (int i = 1; i < PX; ++i) hw[1 + 4 * PX + i] = (unsigned)(c[i] >> 32);
                unsigned hc = (unsigned)(c[0] >> 32);
                if (!all_x) {
                    // Lanes at the grid's x edges: a node that is not stored (x = 0,
                    // x = nx-1, or past the grid where TMA filled zeros) must not
                    // send the warp to the general path, so its private values are
                    // replaced by the reference word.
                    bool use[PX];
#pragma unroll
                    for (int i = 0; i < PX; ++i) use[i] = gx0 + i >= 1 && gx0 + i <= p.nx - 2;
                    bool any_use = false;
#pragma unroll
                    for (int i = 0; i < PX; ++i) any_use = any_use || use[i];
                    // a lane that stores none of its nodes (past the grid: zeros) votes for the
                    // fast path: its reference is 1.0's word (its outputs are never stored)
                    if (!any_use) hc = 0x3ff00000u;
                    if (!use[0]) hw[0] = hc;       // left: x-neighbour of node 0 only
                    if (!use[PX - 1]) hw[1] = hc;  // right: x-neighbour of the last node only
#pragma unroll
                    for (int i = 0; i < PX; ++i) {
                        if (!use[i]) {  // y and z neighbours belong to node i alone
                            hw[2 + 4 * i] = hc;
                            hw[3 + 4 * i] = hc;
                            hw[4 + 4 * i] = hc;
                            hw[5 + 4 * i] = hc;
                        }
                    }
#pragma unroll
                    for (int i = 1; i < PX; ++i) {  // centre i is also node i-1's and i+1's x-neighbour
                        const bool need = use[i] || use[i - 1] || (i + 1 < PX && use[i + 1]);
                        if (!need) hw[1 + 4 * PX + i] = hc;
                    }
                }
                const bool fast = emu_same_binade_hi(hw, hc);
                // warp-uniform branch: smooth fields take the short fast path
                if (__all_sync(rmask, fast)) {
#pragma unroll
                    for (int i = 0; i < PX; ++i) {
                        const double ci = (double)vget<V, E>(civ, i);
                        if constexpr (kScaled)
                            reinterpret_cast<E *>(&out)[i] =
                                emu_fast_node_scaled(c[i], xm[i], xp[i], ym[i], yp[i], zm[i], zp[i], ci);
                        else
                            reinterpret_cast<E *>(&out)[i] = emu_fast_node<kIso, kDmul>(
                                c[i], xm[i], xp[i], ym[i], yp[i], zm[i], zp[i], ci, p.ek);
                    }
                } else {
                    // one path for the whole warp (emu64.cuh): values of one sign within
                    // five binades take the cheap exact conversion, anything else the
                    // general one
                    double ci[PX], o[PX];
#pragma unroll
                    for (int i = 0; i < PX; ++i) ci[i] = (double)vget<V, E>(civ, i);
                    unsigned ewin;
                    const bool near = emu_window_hi(hw, hc, &ewin);
                    if (__all_sync(rmask, near))
                        emu_lane_window<PX, kScaled, kIso>(c, xm[0], xp[PX - 1], ym, yp, zm, zp, ci, p.ek,
                                                           ewin, o);
                    else
                        emu_lane_general<PX, kScaled, kIso>(c, xm[0], xp[PX - 1], ym, yp, zm, zp, ci,
                                                            p.ek, o);
#pragma unroll
                    for (int i = 0; i < PX; ++i) reinterpret_cast<E *>(&out)[i] = o[i];
                }
            } else
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                const E c = vget<V, E>(qc, i);
                const E xm = i == 0 ? left : vget<V, E>(qc, i - 1);
                const E xp = i == PX - 1 ? right : vget<V, E>(qc, i + 1);
                const E ym = vget<V, E>(up, i), yp = vget<V, E>(dn, i);
                const E zm = vget<V, E>(qm, i), zp = vget<V, E>(qn, i);
                const E ci = vget<V, E>(civ, i);
                E r;
                if constexpr (MODE == Z_F64_NATIVE) {
                    const double d2x = (xp - c) - (c - xm), d2y = (yp - c) - (c - ym);
                    const double d2z = (zp - c) - (c - zm);
                    r = c + p.ek.dtlam * (ci * ((d2x * p.ek.ax + d2y * p.ek.ay) + d2z * p.ek.az));
                } else if constexpr (MODE == Z_F32) {
                    r = f32_node(c, xm, xp, ym, yp, zm, zp, ci, p.fdtlam, p.fax, p.fay, p.faz);
                } else {  // Z_F32_COMP
                    const E el = i == 0 ? eleft : vget<V, E>(eqc, i - 1);
                    const E er = i == PX - 1 ? eright : vget<V, E>(eqc, i + 1);
                    float e2;
                    r = comp32_node(c, xm, xp, ym, yp, zm, zp, vget<V, E>(eqc, i), el, er,
                                    vget<V, E>(eup, i), vget<V, E>(edn, i), vget<V, E>(eqm, i),
                                    vget<V, E>(eqn, i), ci, p.fdtlam, p.fax, p.fay, p.faz, &e2);
                    reinterpret_cast<E *>(&cv)[i] = e2;
                }
                reinterpret_cast<E *>(&out)[i] = r;
            }
            if (all_x) {
                *(V *)(T2 + base) = out;
                if constexpr (kComp) *(V *)(E2 + base) = cv;
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    const int gx = gx0 + i;
                    if (gx >= 1 && gx <= p.nx - 2) {
                        T2[base + i] = vget<V, E>(out, i);
                        if constexpr (kComp) E2[base + i] = vget<V, E>(cv, i);
                    } else if (kBnd && !kComp && gx <= p.nx - 1) {
                        T2[base + i] = vget<V, E>(qc, i);  // x = 0 or nx-1: T's boundary value
                    }
                }
            }
        } else if (kBnd && !kComp && gy <= p.ny - 1) {
            // y = 0 or ny-1: a boundary row, stored as T's (its values are in the ring)
            if (gx0 + PX - 1 <= p.nx - 1) {
                *(V *)(T2 + base) = qc;
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i)
                    if (gx0 + i <= p.nx - 1) T2[base + i] = vget<V, E>(qc, i);
            }
        }
        if (!ok) {
            s_abort = 1;
            atomicOr(err, 1u);
        }
        __syncthreads();  // every thread is done with plane k's stage (T and Ci)
        if (s_abort) {
            drain(min(k - 1 + NST, k1));
            return;
        }
        if (threadIdx.x == 0 && k + NST <= k1) issue(sk, k + NST);  // plane k's stage
        sk = sk1;
        qm = qc;
        qc = qn;
        if constexpr (kComp) {
            eqm = eqc;
            eqc = eqn;
        }
    }
}

}  // namespace psd

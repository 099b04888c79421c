// Body of the two-steps-per-pass z-march (temporal blocking of depth 2): one CTA,
// one x-y tile, a chunk of output planes; shared by the single-grid kernel
// k_zmarch2 (zmarch2.cu) and the batched kernel (batch_tma.cu).
//
// T2 = step(step(T)).  A CTA owns a BX x BY output tile (one warp per row, PX
// nodes per thread) and a chunk of output planes [k0, k1).  For the
// intermediate state T1 = step(T) it needs the tile plus a one-node ring
// around it, so:
//   * T arrives as one TMA box per plane (tile + 2-node y halo + 16-byte x
//     halo) in an NT-stage ring, Ci as one box per plane (tile + 1-node y halo
//     + 16-byte x halo) in an NC-stage ring;
//   * iteration z computes, in one phase, T1 of plane z+1 (from T planes
//     z .. z+2 and Ci plane z+1) into one of two shared T1 tiles - every
//     thread its own PX nodes, and 2*BX + 2*BY ring values spread one per
//     thread (T1 at the tile's corners is not needed by a 7-point stencil) -
//     and T2 of plane z from T1's tile of plane z (complete since the last
//     barrier) and the thread's own T1 values of planes z-1, z+1 in registers;
//   * the plane's single barrier then frees T plane z and Ci plane z, whose
//     stages take planes z+NT and z+NC: each copy has NT-3 (NC-2) whole
//     iterations to land.  HBM traffic per pass is that of one step
// (read T and Ci, write T2: halo planes and columns come from L2), so T_eff
// can reach twice the one-step rate when arithmetic keeps up.
//
// Per-node arithmetic is node.cuh's, the same as the one-step kernels':
// the result is bit for bit that of two single steps.  Nodes of T1 that are
// not interior keep T's value (the boundary is fixed); T2's boundary is not
// written (the caller's buffer already holds it).
#pragma once

#include <cuda.h>

#include "node.cuh"
#include "tma.cuh"

namespace psd {

template <typename E>
struct Z2Traits;
template <>
struct Z2Traits<double> {
    using V = double2;
    static constexpr int PX = 2;
};
template <>
struct Z2Traits<float> {
    using V = float4;
    static constexpr int PX = 4;
};

struct Z2Params {
    int64_t nx, ny, nz;
    int64_t pitch;  // elements between consecutive rows (nx for a contiguous grid)
    int kchunk, ntx;
    float dtlam, ax, ay, az;  // FP32 coefficients (FP64 runs on the pre-scaled Cs)
};

template <typename E>
__device__ __forceinline__ E z2_node(E c, E xm, E xp, E ym, E yp, E zm, E zp, E ci, const Z2Params &p) {
    if constexpr (sizeof(E) == 8)
        return f64s_node(c, xm, xp, ym, yp, zm, zp, ci);
    else
        return f32_node(c, xm, xp, ym, yp, zm, zp, ci, p.dtlam, p.ax, p.ay, p.az);
}

template <typename V, typename E>
__device__ __forceinline__ E z2get(const V &v, int i) {
    return reinterpret_cast<const E *>(&v)[i];
}
template <typename V, typename E>
__device__ __forceinline__ void z2set(V &v, int i, E x) {
    reinterpret_cast<E *>(&v)[i] = x;
}

// FP32: 4 T stages, 3 Ci stages (52 KB, four CTAs per SM); FP64 (register-bound at
// three CTAs): 5 and 4.
template <typename E>
struct Z2Ring {
    static constexpr int NT = sizeof(E) == 8 ? 5 : 4, NC = sizeof(E) == 8 ? 4 : 3;
    static constexpr int MINB = sizeof(E) == 8 ? 3 : 4;
};

// One CTA (32 * BY threads): T2 = step(step(T)) at output planes [k0, k1) of the
// BX x BY tile at (X0, Y0) (boundary included; only interior nodes are written).
// tmT / tmC: tensor maps of T (box W x (BY+4)) and Ci (box W x (BY+2)), in
// parameter or global memory.  Rows are p.pitch elements apart, planes
// p.pitch * p.ny.  A timed-out wait sets bit 0 of *err and the CTA leaves after
// draining its copies.
// kStates (the state-keeping loop of a reverse sweep): the intermediate state
// T1 = step(T) goes to T1o as well, and both T1o and T2 are written at every node of
// the output planes, their x and y faces as copies of T's (the boundary is fixed),
// so that fresh state grids need only their two z faces set.
template <typename E, int BY, int NT, int NC, bool kStates = false>
__device__ __forceinline__ void zmarch2_tile(const CUtensorMap *tmT, const CUtensorMap *tmC,
                                             E *__restrict__ T2, const Z2Params &p, int X0, int Y0,
                                             int k0, int k1, unsigned *err, E *__restrict__ T1o = nullptr) {
    using V = typename Z2Traits<E>::V;
    constexpr int PX = Z2Traits<E>::PX, HX = 16 / (int)sizeof(E), BX = 32 * PX, W = BX + 2 * HX;
    constexpr int H0 = BY + 4, H1 = BY + 2;         // T box rows, Ci box / T1 tile rows
    constexpr int NW = 2;                            // T1 tiles
    static_assert(NT >= 4 && NC >= 3, "ring depths");
    static_assert(NW == 2, "T1 tile z+2 reuses tile z's slot after the barrier of plane z");
    constexpr int NTH = 32 * BY, NH = 2 * BX + 2 * BY;  // threads, T1 ring values
    constexpr unsigned TB = W * H0 * sizeof(E), CB = W * H1 * sizeof(E);
    constexpr unsigned TBA = (TB + 127) / 128 * 128, CBA = (CB + 127) / 128 * 128;
    constexpr int TS = TBA / sizeof(E), CS = CBA / sizeof(E);  // stage strides in elements
    extern __shared__ __align__(128) unsigned char smem[];
    E *sT = (E *)smem;
    E *sC = (E *)(smem + NT * TBA);
    E *sW = (E *)(smem + NT * TBA + NC * CBA);
    uint64_t *barT = (uint64_t *)(smem + NT * TBA + (NC + NW) * CBA);
    uint64_t *barC = barT + NT;
    __shared__ int s_abort;

    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int nx = (int)p.nx, ny = (int)p.ny, nz = (int)p.nz;

    // T plane q lives in T stage (q - (k0-2)) % NT, Ci plane q in Ci stage (q - (k0-1)) % NC,
    // T1 plane q in tile (q - k0) % 2; the loop advances the stage numbers one by one
    // instead of dividing.
    auto issueT = [&](int s, int q) {
        mbar_expect_tx(&barT[s], TB);
        tma_load_3d(sT + s * TS, tmT, &barT[s], X0 - HX, Y0 - 2, q);
    };
    auto issueC = [&](int s, int q) {
        mbar_expect_tx(&barC[s], CB);
        tma_load_3d(sC + s * CS, tmC, &barC[s], X0 - HX, Y0 - 1, q);
    };
    auto nT = [](int s) { return s + 1 == NT ? 0 : s + 1; };
    auto nC = [](int s) { return s + 1 == NC ? 0 : s + 1; };

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NT; ++s) mbar_init(&barT[s], 1);
        for (int s = 0; s < NC; ++s) mbar_init(&barC[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // the last planes each ring ever needs: T up to k1+1, Ci up to k1 (k1 <= nz-1;
    // planes -1 and nz read zeros)
    const int qTmax = k1 + 1, qCmax = k1;
    if (threadIdx.x == 0) {
        for (int q = k0 - 2; q <= min(k0 - 3 + NT, qTmax); ++q) issueT(q - (k0 - 2), q);
        for (int q = k0 - 1; q <= min(k0 - 2 + NC, qCmax); ++q) issueC(q - (k0 - 1), q);
    }
    unsigned tpar = 0u, cpar = 0u;  // bit s: parity of the next completion of stage s
    auto waitT = [&](int s) -> bool {
        const unsigned ph = (tpar >> s) & 1u;
        tpar ^= 1u << s;
        return mbar_wait(&barT[s], ph);
    };
    auto waitC = [&](int s) -> bool {
        const unsigned ph = (cpar >> s) & 1u;
        cpar ^= 1u << s;
        return mbar_wait(&barC[s], ph);
    };
    // after a timed-out wait: bounded waits for every copy still in flight (T planes
    // up to qT, Ci planes up to qC), so that no TMA write lands after the CTA exits
    auto drain = [&](int qT, int qC) {
        for (int q = max(k0 - 2, qT - NT + 1); q <= qT; ++q) {
            const int i = q - (k0 - 2);
            mbar_wait(&barT[i % NT], (unsigned)(i / NT) & 1u);
        }
        for (int q = max(k0 - 1, qC - NC + 1); q <= qC; ++q) {
            const int i = q - (k0 - 1);
            mbar_wait(&barC[i % NC], (unsigned)(i / NC) & 1u);
        }
    };

    // own nodes: T1 tile / Ci box row r1 (T box row r1 + 1), columns c0 .. c0+PX-1
    const int r1 = ty + 1, c0 = HX + lane * PX;
    const int gy = Y0 + ty, gx0 = X0 + lane * PX;
    const bool yin = gy >= 1 && gy <= ny - 2;
    bool in[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) in[i] = yin && gx0 + i >= 1 && gx0 + i <= nx - 2;
    // T1 ring values of this thread (one, or two when NH > threads)
    constexpr int NHT = (NH + NTH - 1) / NTH;
    int hidx[NHT];
    bool hval[NHT], hin[NHT];
#pragma unroll
    for (int j = 0; j < NHT; ++j) {
        const int t = threadIdx.x + j * NTH;
        int r, c;
        if (t < BX) {
            r = 0;
            c = HX + t;
        } else if (t < 2 * BX) {
            r = H1 - 1;
            c = HX + (t - BX);
        } else {
            const int u = min(t - 2 * BX, 2 * BY - 1);
            r = 1 + (u >> 1);
            c = (u & 1) ? HX + BX : HX - 1;
        }
        hval[j] = t < NH;
        hidx[j] = r * W + c;
        const int x = X0 - HX + c, y = Y0 - 1 + r;
        hin[j] = x >= 1 && x <= nx - 2 && y >= 1 && y <= ny - 2;
    }

    // T1 of plane q from the T stages of planes q-1, q, q+1 and the Ci stage of plane q:
    // own nodes (returned) and ring values, into the T1 tile Wq
    auto t1_plane = [&](int sm, int sc, int sp, int cq, int wq, int q) -> V {
        const E *Tm = sT + sm * TS, *Tc = sT + sc * TS, *Tp = sT + sp * TS;
        const E *Cq = sC + cq * CS;
        E *Wq = sW + wq * CS;
        const bool zin = q >= 1 && q <= nz - 2;
        const int o = (r1 + 1) * W + c0;  // own centre in a T box
        const V c = *(const V *)(Tc + o);
        const V up = *(const V *)(Tc + o - W), dn = *(const V *)(Tc + o + W);
        const V zm = *(const V *)(Tm + o), zp = *(const V *)(Tp + o);
        const E l = Tc[o - 1], r = Tc[o + PX];
        const V ci = *(const V *)(Cq + r1 * W + c0);
        V out;
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            const E ce = z2get<V, E>(c, i);
            E v = ce;
            if (zin && in[i])
                v = z2_node<E>(ce, i == 0 ? l : z2get<V, E>(c, i - 1),
                               i == PX - 1 ? r : z2get<V, E>(c, i + 1), z2get<V, E>(up, i),
                               z2get<V, E>(dn, i), z2get<V, E>(zm, i), z2get<V, E>(zp, i),
                               z2get<V, E>(ci, i), p);
            z2set<V, E>(out, i, v);
        }
        *(V *)(Wq + r1 * W + c0) = out;
#pragma unroll
        for (int j = 0; j < NHT; ++j) {
            if (!hval[j]) continue;
            const int ob = hidx[j] + W;  // the same node in a T box
            const E ce = Tc[ob];
            E v = ce;
            if (zin && hin[j])
                v = z2_node<E>(ce, Tc[ob - 1], Tc[ob + 1], Tc[ob - W], Tc[ob + W], Tm[ob], Tp[ob],
                               Cq[hidx[j]], p);
            Wq[hidx[j]] = v;
        }
        return out;
    };

    // ---- prologue: T1 own values of plane k0-1, T1 tile of plane k0 (tile 0)
    // (T planes k0-2 .. k0+1 are in stages 0 .. 3, Ci planes k0-1, k0 in 0, 1)
    bool ok = waitT(0);
    ok = waitT(1) && ok;
    ok = waitT(2) && ok;
    ok = waitC(0) && ok;
    // plane k0-1's tile values go to tile 1, which plane k0+1 overwrites after the barrier
    V t1m = t1_plane(0, 1, 2, 0, 1, k0 - 1);
    ok = waitT(3) && ok;
    ok = waitC(1) && ok;
    V t1c = t1_plane(1, 2, 3, 1, 0, k0);
    if (!ok) {
        s_abort = 1;
        atomicOr(err, 1u);
    }
    __syncthreads();
    if (s_abort) {
        drain(min(k0 - 3 + NT, qTmax), min(k0 - 2 + NC, qCmax));
        return;
    }
    if (threadIdx.x == 0) {  // T planes k0-2, k0-1 and Ci plane k0-1 are no longer read
        if (k0 - 2 + NT <= qTmax) issueT(0, k0 - 2 + NT);
        if (k0 - 1 + NT <= qTmax) issueT(1, k0 - 1 + NT);
        if (k0 - 1 + NC <= qCmax) issueC(0, k0 - 1 + NC);
    }

    const bool all_x = gx0 >= 1 && gx0 + PX - 1 <= nx - 2;
    int tz = 2 % NT;  // T stage of plane z
    int cz = 1;       // Ci stage of plane z
    int wz = 0;       // T1 tile of plane z
    for (int z = k0; z < k1; ++z) {
        // T1 of plane z+1 (T planes z .. z+2, Ci plane z+1) into the other tile
        const int t1 = nT(tz), t2 = nT(t1), c1 = nC(cz);
        ok = waitT(t2);
        ok = waitC(c1) && ok;
        const V t1p = t1_plane(tz, t1, t2, c1, wz ^ 1, z + 1);
        if (!ok) {
            s_abort = 1;
            atomicOr(err, 1u);
        }
        // T2 of plane z (T1 tile z is complete since the previous barrier)
        if ((kStates ? gy <= ny - 1 : yin) && ok) {
            const E *Wz = sW + wz * CS;
            const int o = r1 * W + c0;
            const V up = *(const V *)(Wz + o - W), dn = *(const V *)(Wz + o + W);
            const E l = Wz[o - 1], r = Wz[o + PX];
            const V ci = *(const V *)(sC + cz * CS + o);
            V out;
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                const E ce = z2get<V, E>(t1c, i);
                z2set<V, E>(out, i,
                            z2_node<E>(ce, i == 0 ? l : z2get<V, E>(t1c, i - 1),
                                       i == PX - 1 ? r : z2get<V, E>(t1c, i + 1), z2get<V, E>(up, i),
                                       z2get<V, E>(dn, i), z2get<V, E>(t1m, i), z2get<V, E>(t1p, i),
                                       z2get<V, E>(ci, i), p));
            }
            const int64_t base = (int64_t)gx0 + p.pitch * ((int64_t)gy + p.ny * (int64_t)z);
            if constexpr (kStates) {
                // T1 of plane z and T2 at every node of the row: T's value (held in T1's
                // non-interior entries) where the node is not interior
#pragma unroll
                for (int i = 0; i < PX; ++i)
                    if (!in[i]) z2set<V, E>(out, i, z2get<V, E>(t1c, i));
                if (gx0 + PX - 1 <= nx - 1) {
                    *(V *)(T1o + base) = t1c;
                    *(V *)(T2 + base) = out;
                } else {
#pragma unroll
                    for (int i = 0; i < PX; ++i)
                        if (gx0 + i <= nx - 1) {
                            T1o[base + i] = z2get<V, E>(t1c, i);
                            T2[base + i] = z2get<V, E>(out, i);
                        }
                }
            } else if (all_x) {
                *(V *)(T2 + base) = out;
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i)
                    if (in[i]) T2[base + i] = z2get<V, E>(out, i);
            }
        }
        // tile z+1 complete; tile z, T plane z and Ci plane z are no longer read
        __syncthreads();
        if (s_abort) {
            drain(min(z - 1 + NT, qTmax), min(z - 1 + NC, qCmax));
            return;
        }
        if (threadIdx.x == 0) {
            if (z + NT <= qTmax) issueT(tz, z + NT);  // into T plane z's stage
            if (z + NC <= qCmax) issueC(cz, z + NC);  // into Ci plane z's stage
        }
        t1m = t1c;
        t1c = t1p;
        tz = t1;
        cz = c1;
        wz ^= 1;
    }
}

}  // namespace psd

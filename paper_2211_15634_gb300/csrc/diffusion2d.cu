// 2-D form of the step (Fig. 1's step! with the z term dropped) as a warp-level
// y-march.
//
// Warp w owns a strip of 32*PX columns (PX nodes per lane: two 16-byte accesses when
// the rows allow them - eight FP32 or four FP64 nodes - else PX = 1) and a chunk of
// interior rows [j0, j1).  Each
// lane keeps its own values of rows j-1, j, j+1 and Ci of row j in registers and
// loads row j+2 and Ci of row j+1 while it computes row j: plain coalesced loads,
// no shared memory and no barriers - the x-neighbours come from the neighbouring
// lanes by warp shuffles and, at the strip's two edges, from one extra load each.
// Every T value is read from HBM once (the strip-edge columns and the rows shared
// by consecutive chunks hit in L2).  The per-node arithmetic is the 3-D step's
// (node.cuh, emu64.cuh) with the z-neighbours set to the centre value: the z
// difference is then exactly zero.
#include <algorithm>

#include "emu64.cuh"
#include "internal.h"
#include "node.cuh"
#include "zmarch.h"

namespace psd {

struct P2D {
    int64_t nx, ny;
    int chunk, nstrips;
    float fdtlam, fax, fay;
    EmuCoef ek;
};

template <int MODE>
struct M2D;  // element type per mode
template <>
struct M2D<Z_F32> {
    using E = float;
};
template <>
struct M2D<Z_F64_SCALED> {
    using E = double;
};
template <>
struct M2D<Z_F64_EMU_ISO_DMUL> {
    using E = double;
};
template <>
struct M2D<Z_F64_NATIVE> {
    using E = double;
};

template <int MODE, typename E>
__device__ __forceinline__ E node2d(E c, E xm, E xp, E ym, E yp, E ci, const P2D &p) {
    if constexpr (MODE == Z_F32) {
        return f32_node(c, xm, xp, ym, yp, c, c, ci, p.fdtlam, p.fax, p.fay, 0.f);
    } else if constexpr (MODE == Z_F64_SCALED) {
        return f64s_node(c, xm, xp, ym, yp, c, c, ci);
    } else if constexpr (MODE == Z_F64_EMU_ISO_DMUL) {
        return emu_step_node<true, true>(dbits(c), dbits(xm), dbits(xp), dbits(ym), dbits(yp), dbits(c),
                                         dbits(c), ci, p.ek);
    } else {
        const double d2x = (xp - c) - (c - xm), d2y = (yp - c) - (c - ym);
        return c + p.ek.dtlam * (ci * (d2x * p.ek.ax + d2y * p.ek.ay));
    }
}

// PX values of row r starting at column x (x % PX == 0); columns >= nx read as 0
template <typename E, int PX>
__device__ __forceinline__ void load_row(E (&v)[PX], const E *__restrict__ A, int64_t r, int64_t nx,
                                         int64_t x) {
    const E *q = A + r * nx + x;
    if constexpr (PX * sizeof(E) == 32) {  // two 16-byte loads
        if (x + PX <= nx) {
            if constexpr (sizeof(E) == 8) {
                const double2 a = __ldg((const double2 *)q), b = __ldg((const double2 *)q + 1);
                v[0] = a.x;
                v[1] = a.y;
                v[2] = b.x;
                v[3] = b.y;
            } else {
                const float4 a = __ldg((const float4 *)q), b = __ldg((const float4 *)q + 1);
                v[0] = a.x;
                v[1] = a.y;
                v[2] = a.z;
                v[3] = a.w;
                v[4] = b.x;
                v[5] = b.y;
                v[6] = b.z;
                v[7] = b.w;
            }
            return;
        }
    }
    if constexpr (PX * sizeof(E) == 16) {
        if (x + PX <= nx) {
            if constexpr (sizeof(E) == 8) {
                const double2 t = __ldg((const double2 *)q);
                v[0] = t.x;
                v[1] = t.y;
            } else {
                const float4 t = __ldg((const float4 *)q);
                v[0] = t.x;
                v[1] = t.y;
                v[2] = t.z;
                v[3] = t.w;
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < PX; ++i) v[i] = x + i < nx ? __ldg(q + i) : E(0);
}

// MINB CTAs of 8 warps per SM: 3 for two FP64 / eight FP32 nodes per lane and the
// scalar forms (the FP64 emulated modes spill at 4, measured 4% slower there); 2 for four
// FP64 nodes per lane (111 registers, no spill)
template <int MODE, int PX, int MINB = 3>
__global__ void __launch_bounds__(256, MINB)
k_ymarch2d(typename M2D<MODE>::E *__restrict__ T2, const typename M2D<MODE>::E *__restrict__ T,
           const typename M2D<MODE>::E *__restrict__ Ci, const P2D p) {
    using E = typename M2D<MODE>::E;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t strip = warp % p.nstrips, chunk = warp / p.nstrips;
    const int64_t nx = p.nx, ny = p.ny;
    const int64_t j0 = 1 + chunk * p.chunk, j1 = min(j0 + p.chunk, ny - 1);  // rows [j0, j1)
    if (j0 >= j1) return;  // warp-uniform
    const int64_t x0 = strip * 32 * PX, gx0 = x0 + lane * PX;
    const bool has_l = lane == 0 && x0 >= 1, has_r = lane == 31 && x0 + 32 * PX < nx;
    bool wr[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) wr[i] = gx0 + i >= 1 && gx0 + i <= nx - 2;
    const bool all_w = gx0 >= 1 && gx0 + PX - 1 <= nx - 2;

    E up[PX], c[PX], dn[PX], ci[PX], nxt[PX], cin[PX];
    load_row<E, PX>(up, T, j0 - 1, nx, gx0);
    load_row<E, PX>(c, T, j0, nx, gx0);
    load_row<E, PX>(dn, T, j0 + 1, nx, gx0);
    load_row<E, PX>(ci, Ci, j0, nx, gx0);
    E hl = has_l ? __ldg(T + j0 * nx + x0 - 1) : E(0), hr = has_r ? __ldg(T + j0 * nx + x0 + 32 * PX) : E(0);
    for (int64_t j = j0; j < j1; ++j) {
        // row j+2 (the next "down" row) and Ci of row j+1, and the strip-edge values of
        // row j+1, are in flight while row j is computed
        const bool more = j + 1 < j1;
        if (more) {
            load_row<E, PX>(nxt, T, j + 2, nx, gx0);
            load_row<E, PX>(cin, Ci, j + 1, nx, gx0);
        }
        const E hl1 = (more && has_l) ? __ldg(T + (j + 1) * nx + x0 - 1) : E(0);
        const E hr1 = (more && has_r) ? __ldg(T + (j + 1) * nx + x0 + 32 * PX) : E(0);
        // x-neighbours across lanes
        E left = __shfl_up_sync(0xffffffffu, c[PX - 1], 1);
        E right = __shfl_down_sync(0xffffffffu, c[0], 1);
        if (lane == 0) left = hl;
        if (lane == 31) right = hr;
        E out[PX];
        bool warp_fast = false;
        if constexpr (MODE == Z_F64_SCALED || MODE == Z_F64_EMU_ISO_DMUL) {
            // one same-binade check over this lane's distinct values (words of nodes that
            // are not written replaced by the reference, so they cannot force the general
            // path); the whole warp takes the short path together when all lanes pass
            bool any_wr = false;
#pragma unroll
            for (int i = 0; i < PX; ++i) any_wr = any_wr || wr[i];
            // a lane that writes none of its nodes (past the grid) votes for the fast path:
            // its reference is 1.0's word (its outputs are never stored)
            const unsigned hc = any_wr ? (unsigned)(dbits(c[0]) >> 32) : 0x3ff00000u;
            unsigned hw[3 * PX + 1];
            hw[0] = wr[0] ? (unsigned)(dbits(left) >> 32) : hc;
            hw[1] = wr[PX - 1] ? (unsigned)(dbits(right) >> 32) : hc;
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                hw[2 + 2 * i] = wr[i] ? (unsigned)(dbits(up[i]) >> 32) : hc;
                hw[3 + 2 * i] = wr[i] ? (unsigned)(dbits(dn[i]) >> 32) : hc;
            }
#pragma unroll
            for (int i = 1; i < PX; ++i) {
                const bool need = wr[i] || wr[i - 1] || (i + 1 < PX && wr[i + 1]);
                hw[1 + 2 * PX + i] = need ? (unsigned)(dbits(c[i]) >> 32) : hc;
            }
            warp_fast = __all_sync(0xffffffffu, emu_same_binade_hi(hw, hc));
        }
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            const E xm = i == 0 ? left : c[i - 1], xp = i == PX - 1 ? right : c[i + 1];
            if constexpr (MODE == Z_F64_SCALED) {
                if (warp_fast) {
                    out[i] = emu_fast_node_scaled(dbits(c[i]), dbits(xm), dbits(xp), dbits(up[i]), dbits(dn[i]),
                                                  dbits(c[i]), dbits(c[i]), ci[i]);
                    continue;
                }
            } else if constexpr (MODE == Z_F64_EMU_ISO_DMUL) {
                if (warp_fast) {
                    out[i] = emu_fast_node<true, true>(dbits(c[i]), dbits(xm), dbits(xp), dbits(up[i]),
                                                       dbits(dn[i]), dbits(c[i]), dbits(c[i]), ci[i], p.ek);
                    continue;
                }
            }
            out[i] = node2d<MODE, E>(c[i], xm, xp, up[i], dn[i], ci[i], p);
        }
        E *q = T2 + j * nx + gx0;
        if constexpr (PX * sizeof(E) == 32) {
            if (all_w) {
                if constexpr (sizeof(E) == 8) {
                    ((double2 *)q)[0] = make_double2(out[0], out[1]);
                    ((double2 *)q)[1] = make_double2(out[2], out[3]);
                } else {
                    ((float4 *)q)[0] = make_float4(out[0], out[1], out[2], out[3]);
                    ((float4 *)q)[1] = make_float4(out[4], out[5], out[6], out[7]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i)
                    if (wr[i]) q[i] = out[i];
            }
        } else if constexpr (PX * sizeof(E) == 16) {
            if (all_w) {
                if constexpr (sizeof(E) == 8)
                    *(double2 *)q = make_double2(out[0], out[1]);
                else
                    *(float4 *)q = make_float4(out[0], out[1], out[2], out[3]);
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i)
                    if (wr[i]) q[i] = out[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < PX; ++i)
                if (wr[i]) q[i] = out[i];
        }
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            up[i] = c[i];
            c[i] = dn[i];
            dn[i] = nxt[i];
            ci[i] = cin[i];
        }
        hl = hl1;
        hr = hr1;
    }
}

// Edges of a 2-D field: T2 = T on rows 0, ny-1 and columns 0, nx-1 (Fig. 1's
// T2 = copy(T) as far as the boundary is concerned).
template <typename E>
__global__ void k_copy_edges2d(E *__restrict__ T2, const E *__restrict__ T, int64_t nx, int64_t ny) {
    const int64_t n_edge = 2 * nx + 2 * (ny - 2);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_edge;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t p;
        if (t < nx) p = t;
        else if (t < 2 * nx) p = (ny - 1) * nx + (t - nx);
        else {
            const int64_t u = t - 2 * nx, r = 1 + u / 2;
            p = r * nx + ((u & 1) ? nx - 1 : 0);
        }
        T2[p] = T[p];
    }
}

template <int MODE, int PX, int MINB = 3>
static cudaError_t launch_2d_t(void *T2, const void *T, const void *Ci, P2D p, int64_t nx, int64_t ny,
                               cudaStream_t s) {
    using E = typename M2D<MODE>::E;
    p.nx = nx;
    p.ny = ny;
    p.nstrips = (int)((nx + 32 * PX - 1) / (32 * PX));
    // chunks of 16-256 rows, about eight waves of resident warps (48 per SM)
    int chunk = launch_override(PS_OVERRIDE_CHUNK2D);
    if (chunk <= 0) {
        const int64_t target = 8LL * 48 * sm_count();
        const int64_t c = (ny - 2) * (int64_t)p.nstrips / target;
        chunk = (int)(c < 16 ? 16 : (c > 256 ? 256 : c));
    }
    p.chunk = chunk;
    const int64_t nch = (ny - 2 + chunk - 1) / chunk, warps = nch * p.nstrips, blocks = (warps + 7) / 8;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_ymarch2d<MODE, PX, MINB><<<(unsigned)blocks, 256, 0, s>>>((E *)T2, (const E *)T, (const E *)Ci, p);
    return cudaGetLastError();
}

// mode: Z_F32, Z_F64_SCALED (Ci holds dt*lam*_dx^2*Ci, equal spacings), Z_F64_EMU_ISO_DMUL
// (equal spacings, positive coefficient) or Z_F64_NATIVE (anything else in FP64)
cudaError_t launch_step2d(int mode, void *T2, const void *T, const void *Ci, StepCoef c, int64_t nx,
                          int64_t ny, cudaStream_t s) {
    P2D p{};
    p.fdtlam = (float)c.dtlam;
    p.fax = (float)c.ax;
    p.fay = (float)c.ay;
    p.ek = EmuCoef{emu_const(c.dtlam * c.ax), emu_const(c.dtlam * c.ay), emu_const(c.dtlam * c.ax),
                   c.dtlam, c.ax, c.ay, 0.0, c.dtlam * c.ax};
    const int esz = mode == Z_F32 ? 4 : 8;
    const bool vec = ((nx * esz) % 16 == 0) && ((((uintptr_t)T2 | (uintptr_t)T | (uintptr_t)Ci) & 15u) == 0);
    switch (mode) {
        case Z_F32:
            // eight nodes per lane (two 16-byte accesses): measured 7-9% faster than four at
            // 16384^2 and 32768^2
            return vec ? launch_2d_t<Z_F32, 8>(T2, T, Ci, p, nx, ny, s) : launch_2d_t<Z_F32, 1>(T2, T, Ci, p, nx, ny, s);
        // FP64: four nodes per lane (two 16-byte accesses) at two CTAs per SM, measured 8%
        // faster than two per lane at three CTAs per SM at 16384^2 (6% at 8192^2); four per
        // lane at three CTAs per SM spilled and ran 25% slower
        case Z_F64_SCALED:
            return vec ? launch_2d_t<Z_F64_SCALED, 4, 2>(T2, T, Ci, p, nx, ny, s)
                       : launch_2d_t<Z_F64_SCALED, 1>(T2, T, Ci, p, nx, ny, s);
        case Z_F64_EMU_ISO_DMUL:
            return vec ? launch_2d_t<Z_F64_EMU_ISO_DMUL, 4, 2>(T2, T, Ci, p, nx, ny, s)
                       : launch_2d_t<Z_F64_EMU_ISO_DMUL, 1>(T2, T, Ci, p, nx, ny, s);
        default:
            return vec ? launch_2d_t<Z_F64_NATIVE, 4, 2>(T2, T, Ci, p, nx, ny, s)
                       : launch_2d_t<Z_F64_NATIVE, 1>(T2, T, Ci, p, nx, ny, s);
    }
}

cudaError_t launch_copy_edges2d(void *T2, const void *T, int64_t nx, int64_t ny, int esz, cudaStream_t s) {
    const int64_t n = 2 * nx + 2 * (ny - 2);
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    if (esz == 8)
        k_copy_edges2d<unsigned long long><<<blocks, 256, 0, s>>>((unsigned long long *)T2,
                                                                 (const unsigned long long *)T, nx, ny);
    else
        k_copy_edges2d<unsigned><<<blocks, 256, 0, s>>>((unsigned *)T2, (const unsigned *)T, nx, ny);
    return cudaGetLastError();
}

}  // namespace psd

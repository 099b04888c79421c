// FP64 transposed step (adjoint) on Ci as given, as a TMA-fed z-march.
//
// For ybar = dL/dT_{t+1} and the state T = T_t the forward step read:
//   w[q]      = Ci[q]*ybar[q] at interior q, 0 elsewhere (and outside the grid),
//   Tbar[p]   = ybar[p] + dt*lam * sum_d (w[p-e_d] - 2 w[p] + w[p+e_d]) * _d^2   (every p),
//   Cibar[q] += dt*lam * ybar[q] * Lap(T)[q]                                    (interior q).
//
// A CTA owns an x-y tile (one warp per row, PX nodes per thread) and a chunk of
// z-planes over the whole grid [0, nz) (Tbar is written on the boundary too).
// For every plane one thread issues three TMA boxes - T, ybar and Ci, each
// with the x/y halo - into one stage of a ring, all tracked by one mbarrier.
// w is computed once per tile value (with halo) into a shared tile one plane
// ahead of the output plane (three tiles rotate, so a tile is only rewritten
// after every thread has passed the barrier that follows its last read).
// Cibar is read and written with plain 16-byte accesses (no halo).
//
// FP64 arithmetic (see emu64.cuh): every w-stencil sum is formed exactly in
// fixed point at the largest exponent of its seven values (w changes sign and
// is zero on the boundary, so the bit-pattern fast path rarely applies), then
// Tbar = fma(dt*lam*_d^2, S, ybar).  The T-Laplacian of the Cibar term takes the
// same-binade fast path.  About four FP64 instructions per node in all.
#include <cudaTypedefs.h>


#include "emu64.cuh"
#include "internal.h"
#include "pdl.cuh"
#include "tma.cuh"
#include "zmarch.h"

namespace psd {

__device__ unsigned g_adj_error;

struct AdjParams {
    int64_t nx, ny, nz;
    int kchunk, ntx;
    double Kx, Ky, Kz;  // dt*lam*_d^2
};

template <typename E>
struct ATraits;
template <>
struct ATraits<double> {
    using V = double2;
    static constexpr int PX = 2;
};

template <typename V, typename E>
__device__ __forceinline__ E aget(const V &v, int i) {
    return reinterpret_cast<const E *>(&v)[i];
}

template <typename E, bool kIso, int BY, int NST>
__global__ void __launch_bounds__(32 * BY, 3)
k_adjoint_zmarch(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmY,
                 const __grid_constant__ CUtensorMap tmC, E *__restrict__ Tbar,
                 E *__restrict__ Cibar, const AdjParams p) {
    using V = typename ATraits<E>::V;
    static_assert(sizeof(E) == 8, "FP64 only (the FP32 transposed step is k_adjoint_f32)");
    // w tiles hold w in 64-bit fixed point at a CTA-uniform scale
    using WT = long long;
    using WV = longlong2;
    constexpr int PX = ATraits<E>::PX, HX = PX, BX = 32 * PX, W = BX + 2 * HX, H = BY + 2;
    constexpr int NTH = 32 * BY, NV = (W * H + NTH - 1) / NTH;  // tile values per thread
    constexpr unsigned TB = W * H * sizeof(E);
    constexpr unsigned TBA = (TB + 127) / 128 * 128, SS = TBA / sizeof(E);  // box stride in elements
    extern __shared__ __align__(128) unsigned char smem[];
    E *ring = (E *)smem;                          // NST stages x {T, ybar, Ci}
    WT *wtile = (WT *)(smem + 3 * NST * TBA);     // 3 rotating w tiles
    uint64_t *bar = (uint64_t *)(smem + 3 * NST * TBA + 3 * TBA);
    __shared__ int s_abort;
    __shared__ int s_emax[BY];
    grid_dep_wait();  // the previous launch's writes (and its reads of Tbar) are complete
    grid_dep_launch();
    // FP64: biased exponent of the fixed-point scale (value = X * 2^(Esc-1079)); it only grows,
    // and every stored value is at most 2^57 in magnitude.  0x7ff marks a non-finite w.
    int Esc = 1;

    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int X0 = (int)(blockIdx.x % p.ntx) * BX, Y0 = (int)(blockIdx.x / p.ntx) * BY;
    const int k0 = (int)blockIdx.y * p.kchunk;
    const int k1 = (int)min((int64_t)k0 + p.kchunk, p.nz);  // output planes [k0, k1)
    const int nx = (int)p.nx, ny = (int)p.ny, nz = (int)p.nz;

    auto issue = [&](int s, int q) {  // T, ybar, Ci planes q into stage s
        mbar_expect_tx(&bar[s], 3 * TB);
        tma_load_3d(ring + (3 * s + 0) * SS, &tmT, &bar[s], X0 - HX, Y0 - 1, q);
        tma_load_3d(ring + (3 * s + 1) * SS, &tmY, &bar[s], X0 - HX, Y0 - 1, q);
        tma_load_3d(ring + (3 * s + 2) * SS, &tmC, &bar[s], X0 - HX, Y0 - 1, q);
    };
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < NST; ++s)
            if (k0 - 1 + s <= k1) issue(s, k0 - 1 + s);  // planes k0-1 .. (k1 may be nz: zero fill)

    unsigned par = 0u;
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
    // w of tile position (r, c) of plane q, from a stage
    auto wval = [&](const E *Ys, const E *Cs, int r, int c, int q) -> E {
        const int x = X0 - HX + c, y = Y0 - 1 + r;
        const bool in = x >= 1 && x <= nx - 2 && y >= 1 && y <= ny - 2 && q >= 1 && q <= nz - 2;
        return in ? Cs[r * W + c] * Ys[r * W + c] : E(0);
    };
    // this thread's share (indices threadIdx.x + v*NTH) of a plane's w tile; returns the
    // largest biased exponent among them (FP64)
    auto w_values = [&](E (&wv)[NV], const E *Ys, const E *Cs, int q) -> int {
        int em = 0;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int idx = threadIdx.x + v * NTH;
            if (idx < W * H) {
                const int r = idx / W, c = idx - r * W;
                wv[v] = wval(Ys, Cs, r, c, q);
                em = max(em, emu_exp(dbits(wv[v])));
            }
        }
        return em;
    };
    auto w_store = [&](WT *wt, const E (&wv)[NV]) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int idx = threadIdx.x + v * NTH;
            if (idx < W * H) {
                wt[idx] = emu_fixed(dbits(wv[v]), Esc);
            }
        }
    };
    // agree on the CTA's scale (contains a __syncthreads); entries this thread
    // stored earlier and its register queue are shifted down when the scale grows
    auto agree = [&](int em_local, WT *older, WT (&wreg)[PX]) {
        const unsigned m = __reduce_max_sync(0xffffffffu, (unsigned)em_local);
        if (lane == 0) s_emax[ty] = (int)m;
        __syncthreads();
        int e = Esc;
#pragma unroll
        for (int w = 0; w < BY; ++w) e = max(e, s_emax[w]);
        if (e > Esc) {
            const int d = e - Esc;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const int idx = threadIdx.x + v * NTH;
                if (idx < W * H) older[idx] = d >= 64 ? 0 : (older[idx] >> d);
            }
#pragma unroll
            for (int i = 0; i < PX; ++i) wreg[i] = d >= 64 ? 0 : (wreg[i] >> d);
            Esc = e;
        }
    };

    const int row = ty + 1, col = HX + lane * PX;
    // prologue: plane k0-1 (own T and w centres), plane k0 (own T centre, w tile)
    int s_m = 0;            // stage of plane k0-1
    int s_c = nexts(s_m);   // stage of plane k
    bool ok = acquire(s_m);
    V tm = *(const V *)(ring + (3 * s_m) * SS + row * W + col);
    E wm0[PX];
    int em0 = 0;
#pragma unroll
    for (int i = 0; i < PX; ++i) {
        wm0[i] = wval(ring + (3 * s_m + 1) * SS, ring + (3 * s_m + 2) * SS, row, col + i, k0 - 1);
        em0 = max(em0, emu_exp(dbits(wm0[i])));
    }
    ok = acquire(s_c) && ok;
    V tc = *(const V *)(ring + (3 * s_c) * SS + row * W + col);
    int wcur = 0;
    WT wm[PX];
    {
        E wv[NV];
        em0 = max(em0, w_values(wv, ring + (3 * s_c + 1) * SS, ring + (3 * s_c + 2) * SS, k0));
#pragma unroll
        for (int i = 0; i < PX; ++i) wm[i] = WT(0);
        agree(em0, wtile + wcur * SS, wm);  // nothing stored yet: only sets the scale
        w_store(wtile + wcur * SS, wv);
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            wm[i] = emu_fixed(dbits(wm0[i]), Esc);
        }
    }
    if (!ok) {
        s_abort = 1;
        atomicOr(&g_adj_error, 1u);
    }

    const int gy = Y0 + ty;
    const int gx0 = X0 + lane * PX;
    const bool row_out = gy <= ny - 1;                    // Tbar rows written
    const bool row_in = gy >= 1 && gy <= ny - 2;          // rows with interior nodes
    const bool all_x = gx0 + PX - 1 <= nx - 1;            // every node of the thread exists
    const bool all_in = gx0 >= 1 && gx0 + PX - 1 <= nx - 2;

    for (int k = k0; k < k1; ++k) {
        const int s_n = nexts(s_c);  // stage of plane k+1
        ok = acquire(s_n) && ok;
        const int wnxt = wcur == 2 ? 0 : wcur + 1;
        {
            E wv[NV];
            const int em = w_values(wv, ring + (3 * s_n + 1) * SS, ring + (3 * s_n + 2) * SS, k + 1);
            agree(em, wtile + wcur * SS, wm);
            w_store(wtile + wnxt * SS, wv);
        }
        if (!ok) {
            s_abort = 1;
            atomicOr(&g_adj_error, 1u);
        }
        __syncthreads();  // w tile k+1 complete; every thread has left iteration k-1
        if (s_abort) {  // planes up to k-2+NST (at most k1) have been issued
            drain(min(k - 2 + NST, k1));
            return;
        }
        if (threadIdx.x == 0 && k - 1 + NST <= k1) issue(s_m, k - 1 + NST);  // plane k-1's stage

        const E *Tk = ring + (3 * s_c) * SS;
        const E *Yk = ring + (3 * s_c + 1) * SS;
        const WT *wk = wtile + wcur * SS;
        const V tp = *(const V *)(ring + (3 * s_n) * SS + row * W + col);
        const V yc = *(const V *)(Yk + row * W + col);
        const WV wc = *(const WV *)(wk + row * W + col);
        const WV wu = *(const WV *)(wk + (row - 1) * W + col);
        const WV wd = *(const WV *)(wk + (row + 1) * W + col);
        const WV wp = *(const WV *)(wtile + wnxt * SS + row * W + col);
        const WT wl = wk[row * W + col - 1], wr = wk[row * W + col + PX];
        const V tu = *(const V *)(Tk + (row - 1) * W + col);
        const V td = *(const V *)(Tk + (row + 1) * W + col);
        const E tl = Tk[row * W + col - 1], tr = Tk[row * W + col + PX];
        const bool plane_in = k >= 1 && k <= nz - 2;

        if (row_out) {
            const int64_t base = (int64_t)gx0 + p.nx * ((int64_t)gy + p.ny * (int64_t)k);
            V tb, cb{};
            const bool do_ci = row_in && plane_in;
            if (do_ci) {
                if (all_in) {
                    cb = *(const V *)(Cibar + base);
                } else {
#pragma unroll
                    for (int i = 0; i < PX; ++i) {
                        const int gx = gx0 + i;
                        reinterpret_cast<E *>(&cb)[i] = (gx >= 1 && gx <= nx - 2) ? Cibar[base + i] : E(0);
                    }
                }
            }
            // ---- Tbar: exact fixed-point w-stencil sums, one DFMA per coefficient
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                const long long c2 = 2 * aget<WV, WT>(wc, i);
                const long long xm = i == 0 ? wl : aget<WV, WT>(wc, i - 1);
                const long long xp = i == PX - 1 ? wr : aget<WV, WT>(wc, i + 1);
                const long long sx = xm + xp - c2;
                const long long sy = aget<WV, WT>(wu, i) + aget<WV, WT>(wd, i) - c2;
                const long long sz = wm[i] + aget<WV, WT>(wp, i) - c2;
                const double yb = aget<V, E>(yc, i);
                // a non-finite w anywhere in this CTA's march: report NaN, not garbage
                reinterpret_cast<E *>(&tb)[i] =
                    Esc == 0x7ff ? __longlong_as_double(0x7ff8000000000000ll)
                                 : emu_axpy3<kIso>(yb, sx, sy, sz, Esc - 1079, p.Kx, p.Ky, p.Kz);
            }
            // ---- Cibar: T-Laplacian, same-binade fast path when the whole warp allows it
            if (do_ci) {
                unsigned long long c[PX], xm[PX], xp[PX], ym[PX], yp[PX], zm[PX], zp[PX];
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    c[i] = dbits(aget<V, E>(tc, i));
                    xm[i] = dbits(i == 0 ? tl : aget<V, E>(tc, i - 1));
                    xp[i] = dbits(i == PX - 1 ? tr : aget<V, E>(tc, i + 1));
                    ym[i] = dbits(aget<V, E>(tu, i));
                    yp[i] = dbits(aget<V, E>(td, i));
                    zm[i] = dbits(aget<V, E>(tm, i));
                    zp[i] = dbits(aget<V, E>(tp, i));
                }
                unsigned hc = (unsigned)(c[0] >> 32);
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
                bool use[PX];
#pragma unroll
                for (int i = 0; i < PX; ++i) use[i] = gx0 + i >= 1 && gx0 + i <= nx - 2;
                if (!all_in) {  // unstored edge nodes must not force the general path
                    bool any_use = false;
#pragma unroll
                    for (int i = 0; i < PX; ++i) any_use = any_use || use[i];
                    // a lane that stores none of its nodes (past the grid: zeros) votes for the
                    // fast path: its reference is 1.0's word (its outputs are never stored)
                    if (!any_use) hc = 0x3ff00000u;
                    if (!use[0]) hw[0] = hc;
                    if (!use[PX - 1]) hw[1] = hc;
#pragma unroll
                    for (int i = 0; i < PX; ++i)
                        if (!use[i]) hw[2 + 4 * i] = hw[3 + 4 * i] = hw[4 + 4 * i] = hw[5 + 4 * i] = hc;
#pragma unroll
                    for (int i = 1; i < PX; ++i)
                        if (!(use[i] || use[i - 1] || (i + 1 < PX && use[i + 1]))) hw[1 + 4 * PX + i] = hc;
                }
                const bool fast = emu_same_binade_hi(hw, hc);
                const bool wfast = __all_sync(0xffffffffu, fast);
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    long long sx, sy, sz;
                    int sc;
                    double L;
                    if (wfast || fast) {
                        const unsigned long long c2 = c[i] + c[i];
                        sx = (long long)(xm[i] + xp[i] - c2);
                        sy = (long long)(ym[i] + yp[i] - c2);
                        sz = (long long)(zm[i] + zp[i] - c2);
                        if (c[i] >> 63) {
                            sx = -sx;
                            sy = -sy;
                            sz = -sz;
                        }
                        const int e = emu_exp(c[i]);
                        sc = (e ? e : 1) - 1075;
                        L = emu_axpy3<kIso>(0.0, sx, sy, sz, sc, p.Kx, p.Ky, p.Kz);
                    } else if (emu_sums_general(c[i], xm[i], xp[i], ym[i], yp[i], zm[i], zp[i],
                                                sx, sy, sz, sc)) {
                        L = emu_axpy3<kIso>(0.0, sx, sy, sz, sc, p.Kx, p.Ky, p.Kz);
                    } else {
                        const double cc = bitsd(c[i]);
                        L = (p.Kx * ((bitsd(xm[i]) - cc) - (cc - bitsd(xp[i]))) +
                             p.Ky * ((bitsd(ym[i]) - cc) - (cc - bitsd(yp[i])))) +
                            p.Kz * ((bitsd(zm[i]) - cc) - (cc - bitsd(zp[i])));
                    }
                    reinterpret_cast<E *>(&cb)[i] = fma(aget<V, E>(yc, i), L, aget<V, E>(cb, i));
                }
            }
            if (all_x) {
                *(V *)(Tbar + base) = tb;
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i)
                    if (gx0 + i <= nx - 1) Tbar[base + i] = aget<V, E>(tb, i);
            }
            if (do_ci) {
                if (all_in) {
                    *(V *)(Cibar + base) = cb;
                } else {
#pragma unroll
                    for (int i = 0; i < PX; ++i) {
                        const int gx = gx0 + i;
                        if (gx >= 1 && gx <= nx - 2) Cibar[base + i] = aget<V, E>(cb, i);
                    }
                }
            }
        }
        // rotate: plane k's values become the "minus" neighbours
#pragma unroll
        for (int i = 0; i < PX; ++i) wm[i] = aget<WV, WT>(wc, i);
        tm = tc;
        tc = tp;
        s_m = s_c;
        s_c = s_n;
        wcur = wnxt;
    }
}

template <typename E, bool kIso, int BY, int NST>
static cudaError_t launch_adj_t(E *Tbar, E *Cibar, const E *ybar, const E *T, const E *Ci, Grid3 g,
                                AdjParams p, int kchunk, cudaStream_t s) {
    constexpr int PX = ATraits<E>::PX, BX = 32 * PX, W = BX + 2 * PX, H = BY + 2;
    constexpr unsigned TBA = (W * H * sizeof(E) + 127) / 128 * 128;
    constexpr size_t smem = 3 * NST * TBA + 3 * TBA + NST * 8;
    static unsigned attr_gen[64] = {0};
    cudaError_t ae;
    if (!set_smem_attr_once((const void *)k_adjoint_zmarch<E, kIso, BY, NST>, (int)smem, attr_gen, &ae)) return ae;
    CUtensorMap mT, mY, mC;
    if (!make_tensor_map_3d(&mT, T, sizeof(E), g, W, H) || !make_tensor_map_3d(&mY, ybar, sizeof(E), g, W, H) ||
        !make_tensor_map_3d(&mC, Ci, sizeof(E), g, W, H))
        return cudaErrorInvalidValue;
    const int64_t ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY, tiles = ntx * nty;
    if (kchunk <= 0) {
        // long z-chunks amortise the two prologue planes; keep at least ~3 waves of CTAs
        const int64_t waves = 3LL * 3 * sm_count();
        const int64_t kc = g.nz * tiles / waves;
        kchunk = (int)(kc < 4 ? 4 : (kc > 16 ? 16 : kc));
    }
    const int64_t gz = (g.nz + kchunk - 1) / kchunk;
    if (tiles > 0x7fffffffLL || gz > 65535) return cudaErrorInvalidConfiguration;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.ntx = (int)ntx;
    p.kchunk = kchunk;
    return launch_pdl(k_adjoint_zmarch<E, kIso, BY, NST>, dim3((unsigned)tiles, (unsigned)gz, 1), dim3(32 * BY), smem,
                      s, mT, mY, mC, Tbar, Cibar, p);
}

bool adjoint_zmarch_supported(Grid3 g, int esz, const void *const *ptrs, int nptr) {
    uintptr_t acc = 0;
    for (int i = 0; i < nptr; ++i) acc |= (uintptr_t)ptrs[i];
    if (acc & 15u) return false;
    if ((g.nx * esz) % 16 != 0) return false;
    if (g.nx > (1LL << 31) - 256 || g.ny > (1LL << 31) - 64 || g.nz > (1LL << 31) - 2) return false;
    return zmarch_supported(g, esz, ptrs[0], ptrs[0], ptrs[0]);
}

template <typename E>
cudaError_t launch_adjoint_zmarch(E *Tbar, E *Cibar, const E *ybar, const E *T, const E *Ci,
                                  StepCoef c, Grid3 g, cudaStream_t s) {
    AdjParams p{};
    p.Kx = c.dtlam * c.ax;
    p.Ky = c.dtlam * c.ay;
    p.Kz = c.dtlam * c.az;
    const int kchunk = launch_override(PS_OVERRIDE_ADJ_KCHUNK);
    const bool iso = c.ax == c.ay && c.ay == c.az;
    if (iso) return launch_adj_t<E, true, 8, 3>(Tbar, Cibar, ybar, T, Ci, g, p, kchunk, s);
    return launch_adj_t<E, false, 8, 3>(Tbar, Cibar, ybar, T, Ci, g, p, kchunk, s);
}

template cudaError_t launch_adjoint_zmarch<double>(double *, double *, const double *, const double *,
                                                   const double *, StepCoef, Grid3, cudaStream_t);

unsigned adjoint_device_error(bool clear) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_adj_error, sizeof(v));
    if (clear) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_adj_error, &z, sizeof(z));
    }
    return v;
}

}  // namespace psd

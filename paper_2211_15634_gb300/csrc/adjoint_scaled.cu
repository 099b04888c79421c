// Transposed step on the pre-scaled coefficient (FP64, equal spacings).
//
// With Cs = dt*lam*_d^2*Ci the forward step reads T2 = T + Cs*L(T) at interior
// nodes, L(A) = sum of the six neighbours of A minus six times the centre.
// Its transpose, for ybar = dL/dT2 and the state T the step read:
//   w[q]      = Cs[q]*ybar[q] at interior q, 0 elsewhere (and outside the grid),
//   Tbar[p]   = ybar[p] + L(w)[p]                      (every node p),
//   Csbar[q] += ybar[q]*L(T)[q]                         (interior q),
// and dL/dCi = dt*lam*_d^2 * Csbar (applied once by the caller).
//
// Layout as in the other z-march kernels: a CTA owns a 64 x BY x-y tile (one
// warp per row, two nodes per thread) and a chunk of z-planes of the whole
// grid.  For every plane one thread issues three TMA boxes (T, ybar, Cs with a
// one-node y halo and a 16-byte x halo) into one ring stage tracked by one
// mbarrier.  w of plane k+1 is built into one of three rotating shared tiles
// as 64-bit fixed point at a CTA-uniform, non-decreasing scale 2^(Esc-1079)
// (|value| < 2^57 units): each thread converts its own two nodes, and 144
// threads one halo node each.  A conversion that would not fit the current
// scale is flagged through the plane's single __syncthreads_or; only then does
// the CTA agree on a larger scale and shift what it already holds.
//
// Per node: Tbar = ybar + pack(S_w) with S_w the exact integer sum (one DADD);
// Csbar = fma(ybar, pack(S_T), Csbar) with S_T the exact bit-pattern sum of
// the same-binade fast path (one DFMA); w = Cs*ybar costs one DMUL per tile
// value.  Csbar of plane k is loaded at the top of iteration k so that its
// latency hides behind the w tile work.
#include <cudaTypedefs.h>


#include "emu64.cuh"
#include "internal.h"
#include "pdl.cuh"
#include "tma.cuh"
#include "zmarch.h"

namespace psd {

__device__ unsigned g_adjs_error;  // set when an mbarrier wait times out

struct AdjSParams {
    int64_t nx, ny, nz;
    int kchunk, ntx;
};

// Fixed-point value of FP64 bits v at scale 2^(E-1079) (E >= the exponent of v).
__device__ __forceinline__ long long adjs_fixed(unsigned long long v, int E) {
    return emu_fixed(v, E);
}

// Exact-when-possible FP64 of the integer S at scale 2^sc.
__device__ __forceinline__ double adjs_pack(long long S, int sc) { return emu_pack(S, sc); }

// The same for a scale at which every packed sum is normal (or zero): |S| < 2^61 at
// scale 2^(E-1079) has an exponent between E - 57 and E + 3, so for E in [57, 2042] the
// range checks can go (the CTA-uniform scale picks this form for the whole plane).
__device__ __forceinline__ double adjs_pack_normal(long long S, int sc) {
    unsigned long long sg;
    const unsigned long long a = emu_abs(S, &sg);
    return bitsd(emu_pack_mag_normal(a, sc) | sg);
}

static __device__ __noinline__ double adjs_lap_general(unsigned long long c, unsigned long long xm,
                                                       unsigned long long xp, unsigned long long ym,
                                                       unsigned long long yp, unsigned long long zm,
                                                       unsigned long long zp) {
    long long sx, sy, sz;
    int sc;
    if (emu_sums_general(c, xm, xp, ym, yp, zm, zp, sx, sy, sz, sc)) return emu_pack(sx + sy + sz, sc);
    const double cc = bitsd(c);  // Inf / NaN: plain FP64 propagates it
    return (((bitsd(xm) + bitsd(xp)) + (bitsd(ym) + bitsd(yp))) + (bitsd(zm) + bitsd(zp))) - 6.0 * cc;
}

template <int BY, int NST>
__global__ void __launch_bounds__(32 * BY, 3)
k_adjoint_scaled(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmY,
                 const __grid_constant__ CUtensorMap tmC, double *__restrict__ Tbar,
                 double *__restrict__ Csbar, const AdjSParams p) {
    constexpr int PX = 2, HX = 2, BX = 64, W = BX + 2 * HX, H = BY + 2;
    constexpr int NHALO = 2 * BX + 2 * BY;  // y-halo rows and x-halo columns (no corners)
    static_assert(NHALO <= 32 * BY, "one halo value per thread at most");
    constexpr unsigned TB = W * H * 8;
    constexpr unsigned TBA = (TB + 127) / 128 * 128, SS = TBA / 8;  // box stride in elements
    extern __shared__ __align__(128) unsigned char smem[];
    double *ring = (double *)smem;                       // NST stages x {T, ybar, Cs}
    long long *wtile = (long long *)(smem + 3 * NST * TBA);  // 3 rotating w tiles
    uint64_t *bar = (uint64_t *)(smem + 3 * NST * TBA + 3 * TBA);
    __shared__ int s_abort, s_E;
    grid_dep_wait();  // the previous launch's writes (and its reads of Tbar) are complete
    grid_dep_launch();

    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int X0 = (int)(blockIdx.x % p.ntx) * BX, Y0 = (int)(blockIdx.x / p.ntx) * BY;
    const int k0 = (int)blockIdx.y * p.kchunk;
    const int k1 = (int)min((int64_t)k0 + p.kchunk, p.nz);  // output planes [k0, k1)
    const int nx = (int)p.nx, ny = (int)p.ny, nz = (int)p.nz;

    auto issue = [&](int s, int q) {
        mbar_expect_tx(&bar[s], 3 * TB);
        tma_load_3d(ring + (3 * s + 0) * SS, &tmT, &bar[s], X0 - HX, Y0 - 1, q);
        tma_load_3d(ring + (3 * s + 1) * SS, &tmY, &bar[s], X0 - HX, Y0 - 1, q);
        tma_load_3d(ring + (3 * s + 2) * SS, &tmC, &bar[s], X0 - HX, Y0 - 1, q);
    };
    if (threadIdx.x == 0) {
        s_abort = 0;
        s_E = 1;
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < NST; ++s)
            if (k0 - 1 + s <= k1) issue(s, k0 - 1 + s);  // planes k0-1 .. (-1 and nz read zeros)

    unsigned par = 0u;
    auto nexts = [](int s) { return s + 1 == NST ? 0 : s + 1; };
    // After a timed-out wait: bounded waits for the copies of the last NST planes
    // issued (up to plane q_iss), so that no TMA write lands after the CTA exits.
    auto drain = [&](int q_iss) {
        for (int q = max(k0 - 1, q_iss - NST + 1); q <= q_iss; ++q) {
            const int i = q - (k0 - 1);
            mbar_wait(&bar[i % NST], (unsigned)(i / NST) & 1u);
        }
    };
    auto acquire = [&](int s) -> bool {
        const unsigned ph = (par >> s) & 1u;
        par ^= 1u << s;
        return mbar_wait(&bar[s], ph);
    };

    // this thread's own nodes (row, col .. col+1 of the tile) and halo node
    const int row = ty + 1, col = HX + lane * PX;
    const int gy = Y0 + ty, gx0 = X0 + lane * PX;
    const bool iny = gy >= 1 && gy <= ny - 2;
    const bool m0 = iny && gx0 >= 1 && gx0 <= nx - 2;
    const bool m1 = iny && gx0 + 1 >= 1 && gx0 + 1 <= nx - 2;
    const int t = threadIdx.x;
    const bool has_h = t < NHALO;
    int hr, hc;
    if (t < 2 * BX) {
        hr = t < BX ? 0 : H - 1;
        hc = HX + (t & (BX - 1));
    } else {
        const int u = t - 2 * BX;
        hr = 1 + (u >> 1);
        hc = (u & 1) ? HX + BX : HX - 1;
    }
    const int hidx = has_h ? hr * W + hc : 0;
    const int hx = X0 - HX + hc, hy = Y0 - 1 + hr;
    const bool hm = has_h && hx >= 1 && hx <= nx - 2 && hy >= 1 && hy <= ny - 2;

    // w of plane q from a stage: own two nodes and the halo node, as doubles
    double w0, w1, wh;
    double2 ynext;  // ybar at the own nodes of plane q (the next iteration's centre)
    auto w_compute = [&](int s, int q) -> int {
        const double *Ys = ring + (3 * s + 1) * SS, *Cs = ring + (3 * s + 2) * SS;
        const bool zin = q >= 1 && q <= nz - 2;
        ynext = *(const double2 *)(Ys + row * W + col);
        const double2 c2 = *(const double2 *)(Cs + row * W + col);
        w0 = (zin && m0) ? c2.x * ynext.x : 0.0;
        w1 = (zin && m1) ? c2.y * ynext.y : 0.0;
        wh = (zin && hm) ? Cs[hidx] * Ys[hidx] : 0.0;
        return max(max(emu_exp(dbits(w0)), emu_exp(dbits(w1))), emu_exp(dbits(wh)));
    };
    auto w_store = [&](long long *wt, int E, long long &f0, long long &f1) {
        f0 = adjs_fixed(dbits(w0), E);
        f1 = adjs_fixed(dbits(w1), E);
        *(longlong2 *)(wt + row * W + col) = make_longlong2(f0, f1);
        if (has_h) wt[hidx] = adjs_fixed(dbits(wh), E);
    };

    // ---- prologue: planes k0-1 (own w, T centre) and k0 (w tile, T and ybar centres)
    int s_m = 0, s_c = 1 % NST;
    bool ok = acquire(s_m);
    ok = acquire(s_c) && ok;
    double2 tm = *(const double2 *)(ring + (3 * s_m) * SS + row * W + col);
    double2 tc = *(const double2 *)(ring + (3 * s_c) * SS + row * W + col);
    int em = w_compute(s_m, k0 - 1);  // includes both own w of plane k0-1
    const double wm0d = w0, wm1d = w1;  // (its halo value is not needed)
    em = max(em, w_compute(s_c, k0));
    double2 yc = ynext;
    em = (int)__reduce_max_sync(0xffffffffu, (unsigned)em);
    if (lane == 0) atomicMax(&s_E, em);
    if (!ok) {
        s_abort = 1;
        atomicOr(&g_adjs_error, 1u);
    }
    __syncthreads();
    if (s_abort) {
        drain(min(k0 + 1, k1));
        return;
    }
    int Esc = s_E;  // CTA-uniform
    int wcur = 0;
    long long wc0, wc1;
    w_store(wtile, Esc, wc0, wc1);
    long long wm0 = adjs_fixed(dbits(wm0d), Esc), wm1 = adjs_fixed(dbits(wm1d), Esc);

    const bool row_out = gy <= ny - 1;
    const bool all_x = gx0 + PX - 1 <= nx - 1;
    const bool all_in = m0 && m1;

    for (int k = k0; k < k1; ++k) {
        const int s_n = nexts(s_c);  // stage of plane k+1
        const bool plane_in = k >= 1 && k <= nz - 2;
        const bool do_ci = iny && plane_in;
        const int64_t base = (int64_t)gx0 + p.nx * ((int64_t)gy + p.ny * (int64_t)k);
        // Csbar of plane k: issued early, used at the end of the iteration
        double2 cb = make_double2(0.0, 0.0);
        if (do_ci) {
            if (all_in) {
                cb = *(const double2 *)(Csbar + base);
            } else {
                if (m0) cb.x = Csbar[base];
                if (m1) cb.y = Csbar[base + 1];
            }
        }
        ok = acquire(s_n);
        const int wnxt = wcur == 2 ? 0 : wcur + 1;
        const int emn = w_compute(s_n, k + 1);
        long long wp0, wp1;
        w_store(wtile + wnxt * SS, Esc, wp0, wp1);
        if (!ok) {
            s_abort = 1;
            atomicOr(&g_adjs_error, 1u);
        }
        // tile k+1 complete; every thread has left iteration k-1 (its stage is free)
        if (__syncthreads_or(emn > Esc || !ok)) {
            if (s_abort) {
                drain(min(k + 1, k1));
                return;
            }
            // a w of plane k+1 needs a larger scale: agree on it, shift what is held
            const int e = (int)__reduce_max_sync(0xffffffffu, (unsigned)emn);
            if (lane == 0) atomicMax(&s_E, e);
            __syncthreads();
            const int E2 = s_E;
            const int d = E2 - Esc;  // > 0
            long long *wk = wtile + wcur * SS;
            auto shr = [d](long long v) { return d >= 64 ? 0ll : (v >> d); };
            wc0 = shr(wc0);
            wc1 = shr(wc1);
            wm0 = shr(wm0);
            wm1 = shr(wm1);
            *(longlong2 *)(wk + row * W + col) = make_longlong2(wc0, wc1);
            if (has_h) wk[hidx] = shr(wk[hidx]);
            Esc = E2;
            w_store(wtile + wnxt * SS, Esc, wp0, wp1);
            __syncthreads();
        }
        if (threadIdx.x == 0 && k - 1 + NST <= k1) issue(s_m, k - 1 + NST);  // plane k-1's stage

        if (row_out) {
            // ---- Tbar = ybar + L(w), exact integer sums, one DADD per node
            const long long *wk = wtile + wcur * SS;
            const long long wl = wk[row * W + col - 1], wr = wk[row * W + col + PX];
            const longlong2 wu = *(const longlong2 *)(wk + (row - 1) * W + col);
            const longlong2 wd = *(const longlong2 *)(wk + (row + 1) * W + col);
            const long long S0 = ((wl + wc1) + (wu.x + wd.x)) + (wm0 + wp0) - 6 * wc0;
            const long long S1 = ((wc0 + wr) + (wu.y + wd.y)) + (wm1 + wp1) - 6 * wc1;
            const int sc = Esc - 1079;
            double2 tb;
            if (Esc >= 57 && Esc <= 2042) {  // CTA-uniform: the packed sums are normal
                tb.x = yc.x + adjs_pack_normal(S0, sc);
                tb.y = yc.y + adjs_pack_normal(S1, sc);
            } else if (Esc == 0x7ff) {  // a non-finite w in this CTA's march: report NaN
                tb.x = tb.y = __longlong_as_double(0x7ff8000000000000ll);
            } else {
                tb.x = yc.x + adjs_pack(S0, sc);
                tb.y = yc.y + adjs_pack(S1, sc);
            }
            if (all_x) {
                *(double2 *)(Tbar + base) = tb;
            } else {
                if (gx0 <= nx - 1) Tbar[base] = tb.x;
                if (gx0 + 1 <= nx - 1) Tbar[base + 1] = tb.y;
            }

            // ---- Csbar += ybar * L(T), bit-pattern sums on the same-binade fast path
            if (do_ci) {
                const double *Tk = ring + (3 * s_c) * SS;
                const double2 tp = *(const double2 *)(ring + (3 * s_n) * SS + row * W + col);
                const double2 tu = *(const double2 *)(Tk + (row - 1) * W + col);
                const double2 td = *(const double2 *)(Tk + (row + 1) * W + col);
                const double tl = Tk[row * W + col - 1], tr = Tk[row * W + col + PX];
                const unsigned long long c0 = dbits(tc.x), c1 = dbits(tc.y);
                const unsigned long long xl = dbits(tl), xr = dbits(tr);
                const unsigned long long u0 = dbits(tu.x), u1 = dbits(tu.y), d0 = dbits(td.x),
                                         d1 = dbits(td.y), m0b = dbits(tm.x), m1b = dbits(tm.y),
                                         p0 = dbits(tp.x), p1 = dbits(tp.y);
                unsigned hc0 = (unsigned)(c0 >> 32);
                unsigned hw[11] = {(unsigned)(xl >> 32), (unsigned)(xr >> 32), (unsigned)(u0 >> 32),
                                   (unsigned)(d0 >> 32), (unsigned)(m0b >> 32), (unsigned)(p0 >> 32),
                                   (unsigned)(u1 >> 32), (unsigned)(d1 >> 32), (unsigned)(m1b >> 32),
                                   (unsigned)(p1 >> 32), (unsigned)(c1 >> 32)};
                if (!all_in) {  // values of unstored nodes must not force the general path
                    // a lane that stores neither node (past the grid: zeros) votes for the fast
                    // path: its reference is 1.0's word (its outputs are never stored)
                    if (!m0 && !m1) hc0 = 0x3ff00000u;
                    if (!m0) hw[0] = hw[2] = hw[3] = hw[4] = hw[5] = hc0;
                    if (!m1) hw[1] = hw[6] = hw[7] = hw[8] = hw[9] = hc0;
                    if (!m0 && !m1) hw[10] = hc0;
                }
                const bool fast = emu_same_binade_hi(hw, hc0);
                double L0, L1;
                if (__all_sync(0xffffffffu, fast)) {
                    const long long S0t = (long long)(((xl + c1) + (u0 + d0)) + (m0b + p0) - 6ull * c0);
                    const long long S1t = (long long)(((c0 + xr) + (u1 + d1)) + (m1b + p1) - 6ull * c1);
                    const int e = emu_exp(c0);
                    const int sct = (e ? e : 1) - 1075;
                    const unsigned long long flip = c0 & 0x8000000000000000ull;  // negative: minus
                    unsigned long long g0, g1;
                    const unsigned long long a0 = emu_abs(S0t, &g0), a1 = emu_abs(S1t, &g1);
                    L0 = bitsd(emu_pack_mag_normal(a0, sct) | (g0 ^ flip));
                    L1 = bitsd(emu_pack_mag_normal(a1, sct) | (g1 ^ flip));
                } else {
                    L0 = m0 ? adjs_lap_general(c0, xl, c1, u0, d0, m0b, p0) : 0.0;
                    L1 = m1 ? adjs_lap_general(c1, c0, xr, u1, d1, m1b, p1) : 0.0;
                }
                cb.x = fma(yc.x, L0, cb.x);
                cb.y = fma(yc.y, L1, cb.y);
                if (all_in) {
                    *(double2 *)(Csbar + base) = cb;
                } else {
                    if (m0) Csbar[base] = cb.x;
                    if (m1) Csbar[base + 1] = cb.y;
                }
            }
        }
        // rotate: plane k becomes the minus neighbour, plane k+1 the centre
        tm = tc;
        tc = *(const double2 *)(ring + (3 * s_n) * SS + row * W + col);
        yc = ynext;
        wm0 = wc0;
        wm1 = wc1;
        wc0 = wp0;
        wc1 = wp1;
        s_m = s_c;
        s_c = s_n;
        wcur = wnxt;
    }
}

cudaError_t launch_adjoint_scaled(double *Tbar, double *Csbar, const double *ybar, const double *T,
                                  const double *Cs, Grid3 g, cudaStream_t s) {
    constexpr int BY = 8, NST = 3, PX = 2, BX = 32 * PX, W = BX + 2 * PX, H = BY + 2;
    constexpr unsigned TBA = (W * H * 8 + 127) / 128 * 128;
    constexpr size_t smem = 3 * NST * TBA + 3 * TBA + NST * 8;
    static unsigned attr_gen[64] = {0};
    cudaError_t ae;
    if (!set_smem_attr_once((const void *)k_adjoint_scaled<BY, NST>, (int)smem, attr_gen, &ae)) return ae;
    CUtensorMap mT, mY, mC;
    if (!make_tensor_map_3d(&mT, T, 8, g, W, H) || !make_tensor_map_3d(&mY, ybar, 8, g, W, H) ||
        !make_tensor_map_3d(&mC, Cs, 8, g, W, H))
        return cudaErrorInvalidValue;
    const int64_t ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY, tiles = ntx * nty;
    int kchunk = launch_override(PS_OVERRIDE_ADJ_KCHUNK);
    if (kchunk <= 0) {
        // long z-chunks amortise the two prologue planes; keep at least ~3 waves of CTAs
        // (3 per SM).  Where chunks of 16 planes or more keep that many, take the chunk
        // of 16-24 planes whose last wave is fullest: measured 256^3 at 19 planes
        // (3.93 waves) 0.1734 ms against 0.1777 at 16 (4.49 waves); 512^3 at 22-24
        // planes 1.5% ahead of 16.
        const int64_t slots = 3LL * sm_count();
        const int64_t kc = g.nz * tiles / (3 * slots);
        if (kc < 16) {
            kchunk = (int)(kc < 4 ? 4 : kc);
        } else {
            kchunk = 16;
            int64_t best = -1;
            for (int c = 16; c <= 24; ++c) {
                const int64_t ctas = tiles * ((g.nz + c - 1) / c);
                const int64_t last = ctas % slots == 0 ? slots : ctas % slots;  // CTAs in the last wave
                if (last > best) {
                    best = last;
                    kchunk = c;
                }
            }
        }
    }
    const int64_t gz = (g.nz + kchunk - 1) / kchunk;
    if (tiles > 0x7fffffffLL || gz > 65535) return cudaErrorInvalidConfiguration;
    AdjSParams p{g.nx, g.ny, g.nz, kchunk, (int)ntx};
    return launch_pdl(k_adjoint_scaled<BY, NST>, dim3((unsigned)tiles, (unsigned)gz, 1), dim3(32 * BY), smem, s,
                      mT, mY, mC, Tbar, Csbar, p);
}

unsigned adjoint_scaled_device_error(bool clear) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_adjs_error, sizeof(v));
    if (clear) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_adjs_error, &z, sizeof(z));
    }
    return v;
}

}  // namespace psd

// Reverse sweep of the pre-scaled FP64 step with the adjoint state in 64-bit fixed
// point (FP64, equal spacings).
//
// The transposed step on Cs = dt*lam*_d^2*Ci (see adjoint_scaled.cu) is, for
// ybar = dL/dT_{t+1} and the state T = T_t the forward step read,
//   w[q]      = Cs[q]*ybar[q] at interior q, 0 elsewhere (and outside the grid),
//   ybar'[p]  = ybar[p] + L(w)[p]                     (every node p),
//   Csbar[q] += ybar[q]*L(T)[q]                        (interior q),
// with L(A) = (sum of the six neighbours of A) - 6 A.  Over a whole sweep ybar
// is only ever multiplied by Cs and summed, so it is kept here as an integer
// field Y with ybar = Y * 2^sigma, one scale sigma for the whole grid:
//   w[q]      = Cs[q]*Y[q] rounded toward zero to an integer (64 x 53-bit
//               integer product, no FP64 instruction),
//   Y'[p]     = Y[p] + L(w)[p]                         (exact integer sum),
//   Csbar[q] += (Y[q]*2^sigma) * L(T)[q]               (one I2F, one DFMA),
// where L(T) is the exact bit-pattern sum of emu64.cuh's same-binade path (the
// fixed-point general path otherwise).  Per node that is two FP64-pipe
// instructions (the sweep with an FP64 ybar needs 3.3) and no pack of L(w).
// Every step keeps |Y| below 2^62; a step records max|Y'| in a small device
// state, and the next step rescales what it reads by a power of two whenever
// that maximum leaves [2^50, 2^60) (it never does on smooth problems), so the
// largest values always carry 50-60 significant bits - more than FP64's 53 at
// the top of the range, fixed absolute resolution 2^sigma below it.
//
// Layout and pipeline as in adjoint_scaled.cu: a CTA owns a 64 x 8 tile of the
// x-y plane (two nodes per thread) and a chunk of z-planes of the whole grid;
// per plane one thread issues three TMA boxes (T, Y, Cs with a one-node y halo
// and a 16-byte x halo) into one ring stage tracked by one mbarrier; w of plane
// k+1 is built into one of three rotating shared tiles (own nodes plus 144 halo
// values), one barrier per plane.
#include <cudaTypedefs.h>

#include "emu64.cuh"
#include "internal.h"
#include "tma.cuh"
#include "zmarch.h"

namespace psd {

__device__ unsigned g_adjfx_error;  // set when an mbarrier wait times out

// One slot of the sweep's scale state (three rotate: see the launch).
struct FxSlot {
    unsigned long long amax;  // max |Y| of the field at this slot's scale
    int sigma;                // ybar = Y * 2^sigma
    int bad;                  // a non-finite input or an out-of-range coefficient was met
};
static_assert(sizeof(FxSlot) == 16, "state layout");
constexpr int kFxSlots = 3;

struct AdjFxParams {
    int64_t nx, ny, nz;
    int kchunk, ntx;
    int slot_in, slot_out, slot_clear;
};

// Number of significant bits of v (0 for v == 0).
__device__ __forceinline__ int bitlen64(unsigned long long v) { return 64 - __clzll((long long)v); }

// Shift applied to an input field of maximum magnitude amax so that its maximum
// lands in [2^58, 2^59) whenever it left [2^50, 2^60): > 0 shifts right.
__device__ __forceinline__ int fx_rescale(unsigned long long amax) {
    const int b = bitlen64(amax);
    if (b > 60) return b - 59;
    if (b > 0 && b < 51) return b - 59;
    return 0;
}

__device__ __forceinline__ long long fx_shift(long long v, int k) {
    return k > 0 ? (v >> k) : (long long)((unsigned long long)v << (-k));
}

// Cs*Y rounded toward zero to an integer; sets *bad for a non-finite Cs or for
// |Cs| >= 1/4.  |Y| < 2^60, so |w| < 2^58 otherwise.
__device__ __forceinline__ long long fx_mul(unsigned long long cs_bits, long long Y, int *bad) {
    const int e = (int)((cs_bits >> 52) & 0x7ff);
    const unsigned long long m = (cs_bits & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
    const int s = 1075 - (e ? e : 1);  // Cs = m * 2^-s
    const unsigned long long neg = (unsigned long long)(Y >> 63);
    const unsigned long long a = ((unsigned long long)Y ^ neg) - neg;  // |Y|
    const unsigned long long lo = a * m, hi = __umul64hi(a, m);
    unsigned long long q;
    if (s >= 64) {
        q = s >= 128 ? 0ull : (hi >> (s - 64));
    } else {
        // s <= 54: |Cs| >= 1/4 (a stable step has Cs <= 1/6.1), where Y + L(w) could
        // leave 63 bits; also Inf / NaN
        if (s <= 54 || e == 0x7ff) *bad = 1;
        q = (lo >> (s & 63)) | (s > 0 ? (hi << ((64 - s) & 63)) : 0ull);
    }
    const unsigned long long sg = neg ^ (unsigned long long)((long long)cs_bits >> 63);
    return (long long)((q ^ sg) - sg);
}

static __device__ __noinline__ double fx_lap_general(unsigned long long c, unsigned long long xm,
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
k_adjoint_fx(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmY,
             const __grid_constant__ CUtensorMap tmC, long long *__restrict__ Yout,
             double *__restrict__ Csbar, FxSlot *__restrict__ state, const AdjFxParams p) {
    constexpr int PX = 2, HX = 2, BX = 64, W = BX + 2 * HX, H = BY + 2;
    constexpr int NHALO = 2 * BX + 2 * BY;  // y-halo rows and x-halo columns (no corners)
    static_assert(NHALO <= 32 * BY, "one halo value per thread at most");
    constexpr unsigned TB = W * H * 8;
    constexpr unsigned TBA = (TB + 127) / 128 * 128, SS = TBA / 8;  // box stride in elements
    extern __shared__ __align__(128) unsigned char smem[];
    double *ring = (double *)smem;                           // NST stages x {T, Y, Cs}
    long long *wtile = (long long *)(smem + 3 * NST * TBA);  // 3 rotating w tiles
    uint64_t *bar = (uint64_t *)(smem + 3 * NST * TBA + 3 * TBA);
    __shared__ int s_abort;

    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int X0 = (int)(blockIdx.x % p.ntx) * BX, Y0 = (int)(blockIdx.x / p.ntx) * BY;
    const int k0 = (int)blockIdx.y * p.kchunk;
    const int k1 = (int)min((int64_t)k0 + p.kchunk, p.nz);  // output planes [k0, k1)
    const int nx = (int)p.nx, ny = (int)p.ny, nz = (int)p.nz;

    // scale of the input, the rescale this step applies, and the slots' upkeep
    const FxSlot in = state[p.slot_in];
    const int kres = fx_rescale(in.amax);
    const int sig = in.sigma + kres;       // ybar = Y * 2^sig for what this step reads and writes
    const double sgm = ldexp(1.0, sig);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        state[p.slot_out].sigma = sig;    // every CTA would write the same value
        state[p.slot_clear].amax = 0ull;  // the slot the next step reports into
        state[p.slot_clear].bad = 0;
        if (in.bad) atomicOr(&state[p.slot_out].bad, 1);
    }

    auto issue = [&](int s, int q) {
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

    int bad = 0;
    auto rd = [&](long long v) { return kres ? fx_shift(v, kres) : v; };
    // w of plane q from a stage into tile wt: own two nodes (returned) and the halo node
    longlong2 ynext;  // Y at the own nodes of plane q (the next iteration's centre)
    auto w_build = [&](int s, int q, long long *wt, long long &f0, long long &f1) {
        const long long *Ys = (const long long *)(ring + (3 * s + 1) * SS);
        const unsigned long long *Cb = (const unsigned long long *)(ring + (3 * s + 2) * SS);
        const bool zin = q >= 1 && q <= nz - 2;
        const longlong2 y2 = *(const longlong2 *)(Ys + row * W + col);
        ynext = make_longlong2(rd(y2.x), rd(y2.y));
        const ulonglong2 c2 = *(const ulonglong2 *)(Cb + row * W + col);
        f0 = (zin && m0) ? fx_mul(c2.x, ynext.x, &bad) : 0ll;
        f1 = (zin && m1) ? fx_mul(c2.y, ynext.y, &bad) : 0ll;
        *(longlong2 *)(wt + row * W + col) = make_longlong2(f0, f1);
        if (has_h) wt[hidx] = (zin && hm) ? fx_mul(Cb[hidx], rd(Ys[hidx]), &bad) : 0ll;
    };

    // ---- prologue: planes k0-1 (own w, T centre) and k0 (w tile, T and Y centres)
    int s_m = 0, s_c = 1 % NST;
    bool ok = acquire(s_m);
    ok = acquire(s_c) && ok;
    if (!ok) {
        s_abort = 1;
        atomicOr(&g_adjfx_error, 1u);
    }
    double2 tm = *(const double2 *)(ring + (3 * s_m) * SS + row * W + col);
    double2 tc = *(const double2 *)(ring + (3 * s_c) * SS + row * W + col);
    long long wm0, wm1, wc0, wc1;
    int wcur = 0;
    // plane k0-1: only its own w is needed (the tile slot is overwritten just below)
    w_build(s_m, k0 - 1, wtile + 2 * SS, wm0, wm1);
    w_build(s_c, k0, wtile, wc0, wc1);
    longlong2 yc = ynext;
    __syncthreads();
    if (s_abort) {
        drain(min(k0 + 1, k1));
        return;
    }

    const bool row_out = gy <= ny - 1;
    const bool all_x = gx0 + PX - 1 <= nx - 1;
    const bool all_in = m0 && m1;
    unsigned long long amax = 0ull;

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
        long long wp0, wp1;
        w_build(s_n, k + 1, wtile + wnxt * SS, wp0, wp1);
        if (!ok) {
            s_abort = 1;
            atomicOr(&g_adjfx_error, 1u);
        }
        __syncthreads();  // tile k+1 complete; every thread has left iteration k-1
        if (s_abort) {
            drain(min(k + 1, k1));
            return;
        }
        if (threadIdx.x == 0 && k - 1 + NST <= k1) issue(s_m, k - 1 + NST);  // plane k-1's stage

        if (row_out) {
            // ---- Y' = Y + L(w), exact integer sums
            const long long *wk = wtile + wcur * SS;
            const long long wl = wk[row * W + col - 1], wr = wk[row * W + col + PX];
            const longlong2 wu = *(const longlong2 *)(wk + (row - 1) * W + col);
            const longlong2 wd = *(const longlong2 *)(wk + (row + 1) * W + col);
            const long long y0 = yc.x + (((wl + wc1) + (wu.x + wd.x)) + (wm0 + wp0) - 6 * wc0);
            const long long y1 = yc.y + (((wc0 + wr) + (wu.y + wd.y)) + (wm1 + wp1) - 6 * wc1);
            if (all_x) {
                *(longlong2 *)(Yout + base) = make_longlong2(y0, y1);
                amax = max(amax, max((unsigned long long)llabs(y0), (unsigned long long)llabs(y1)));
            } else {
                if (gx0 <= nx - 1) {
                    Yout[base] = y0;
                    amax = max(amax, (unsigned long long)llabs(y0));
                }
                if (gx0 + 1 <= nx - 1) {
                    Yout[base + 1] = y1;
                    amax = max(amax, (unsigned long long)llabs(y1));
                }
            }

            // ---- Csbar += (Y * 2^sigma) * L(T): L(T) on the same-binade fast path
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
                const unsigned hc0 = (unsigned)(c0 >> 32);
                unsigned hw[11] = {(unsigned)(xl >> 32), (unsigned)(xr >> 32), (unsigned)(u0 >> 32),
                                   (unsigned)(d0 >> 32), (unsigned)(m0b >> 32), (unsigned)(p0 >> 32),
                                   (unsigned)(u1 >> 32), (unsigned)(d1 >> 32), (unsigned)(m1b >> 32),
                                   (unsigned)(p1 >> 32), (unsigned)(c1 >> 32)};
                if (!all_in) {  // values of unstored nodes must not force the general path
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
                    L0 = bitsd(emu_pack_mag(a0, sct + sig) | (g0 ^ flip));
                    L1 = bitsd(emu_pack_mag(a1, sct + sig) | (g1 ^ flip));
                } else {
                    L0 = m0 ? fx_lap_general(c0, xl, c1, u0, d0, m0b, p0) * sgm : 0.0;
                    L1 = m1 ? fx_lap_general(c1, c0, xr, u1, d1, m1b, p1) * sgm : 0.0;
                }
                // ybar = Y * 2^sigma: the power of two goes into L's exponent, the
                // integer into one I2F
                cb.x = fma(__ll2double_rn(yc.x), L0, cb.x);
                cb.y = fma(__ll2double_rn(yc.y), L1, cb.y);
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
    // one report per warp of the largest |Y'| written and of a bad coefficient
    for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const int anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        atomicMax(&state[p.slot_out].amax, amax);
        if (anybad) atomicOr(&state[p.slot_out].bad, 1);
    }
}

// Reductions and conversions at the two ends of the sweep.
__global__ void k_fx_absmax(const double *__restrict__ ybar, int64_t n, FxSlot *__restrict__ state) {
    unsigned long long m = 0ull;
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long b = dbits(ybar[i]) & 0x7fffffffffffffffull;  // |ybar| bits
        if (b >= 0x7ff0000000000000ull) bad = 1;
        m = max(m, b);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&state[0].amax, m);  // bit patterns of non-negative doubles order like values
        if (bad) atomicOr(&state[0].bad, 1);
    }
}

// Y = ybar * 2^-sigma rounded to nearest, sigma such that max|ybar| * 2^-sigma is in
// [2^58, 2^59] (k_fx_set_scale then records sigma and that bound in slot 0).
__global__ void k_fx_from_double(long long *__restrict__ Y, const double *__restrict__ ybar, int64_t n,
                                 FxSlot *__restrict__ state) {
    const unsigned long long ab = state[0].amax;  // |max| bits
    const int e = (int)(ab >> 52);                 // biased exponent of max|ybar|
    const int sigma = ab == 0ull ? 0 : (e ? e : 1) - 1023 - 58;
    const double scale = ldexp(1.0, -sigma);
    const int bad = state[0].bad;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        Y[i] = bad ? 0ll : __double2ll_rn(ybar[i] * scale);
}

__global__ void k_fx_set_scale(FxSlot *__restrict__ state) {
    const unsigned long long ab = state[0].amax;
    const int e = (int)(ab >> 52);
    state[0].sigma = ab == 0ull ? 0 : (e ? e : 1) - 1023 - 58;
    state[0].amax = ab == 0ull ? 0ull : (1ull << 59);
    state[1].amax = 0ull;
    state[1].bad = 0;
    state[2].amax = 0ull;
    state[2].bad = 0;
}

// ybar = Y * 2^sigma (one rounding to 53 bits); NaN everywhere if the sweep met a
// non-finite value or an out-of-range coefficient.
__global__ void k_fx_to_double(double *__restrict__ ybar, const long long *__restrict__ Y, int64_t n,
                               const FxSlot *__restrict__ state, int slot) {
    const FxSlot st = state[slot];
    const double s = ldexp(1.0, st.sigma);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        ybar[i] = st.bad ? nan : __ll2double_rn(Y[i]) * s;
}

static unsigned fx_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = 8LL * sm_count();
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

cudaError_t launch_adjoint_fx_begin(long long *Y, const double *ybar, int64_t n, void *state,
                                    cudaStream_t s) {
    FxSlot *st = (FxSlot *)state;
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(FxSlot) * kFxSlots, s);
    if (e != cudaSuccess) return e;
    k_fx_absmax<<<fx_blocks(n), 256, 0, s>>>(ybar, n, st);
    k_fx_from_double<<<fx_blocks(n), 256, 0, s>>>(Y, ybar, n, st);
    k_fx_set_scale<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_fx_end(double *ybar, const long long *Y, int64_t n, const void *state, int step,
                                  cudaStream_t s) {
    k_fx_to_double<<<fx_blocks(n), 256, 0, s>>>(ybar, Y, n, (const FxSlot *)state, step % kFxSlots);
    return cudaGetLastError();
}

bool adjoint_fx_supported(Grid3 g, const void *const *ptrs, int nptr) {
    for (int i = 0; i < nptr; ++i)
        if ((uintptr_t)ptrs[i] & 15u) return false;
    return zmarch_supported(g, 8, ptrs[0], ptrs[0], ptrs[0]);
}

cudaError_t launch_adjoint_fx(long long *Yout, double *Csbar, const long long *Yin, const double *T,
                              const double *Cs, Grid3 g, void *state, int step, cudaStream_t s) {
    constexpr int BY = 8, NST = 3, PX = 2, BX = 32 * PX, W = BX + 2 * PX, H = BY + 2;
    constexpr unsigned TBA = (W * H * 8 + 127) / 128 * 128;
    constexpr size_t smem = 3 * NST * TBA + 3 * TBA + NST * 8;
    static unsigned attr_gen[64] = {0};
    cudaError_t ae;
    if (!set_smem_attr_once((const void *)k_adjoint_fx<BY, NST>, (int)smem, attr_gen, &ae)) return ae;
    CUtensorMap mT, mY, mC;
    if (!make_tensor_map_3d(&mT, T, 8, g, W, H) || !make_tensor_map_3d(&mY, Yin, 8, g, W, H) ||
        !make_tensor_map_3d(&mC, Cs, 8, g, W, H))
        return cudaErrorInvalidValue;
    const int64_t ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY, tiles = ntx * nty;
    int kchunk = launch_override(PS_OVERRIDE_ADJ_KCHUNK);
    if (kchunk <= 0) {
        // as the FP64 transposed step: ~3 waves of CTAs (3 per SM), else the chunk of
        // 16-24 planes whose last wave is fullest
        const int64_t slots = 3LL * sm_count();
        const int64_t kc = g.nz * tiles / (3 * slots);
        if (kc < 16) {
            kchunk = (int)(kc < 4 ? 4 : kc);
        } else {
            kchunk = 16;
            int64_t best = -1;
            for (int c = 16; c <= 24; ++c) {
                const int64_t ctas = tiles * ((g.nz + c - 1) / c);
                const int64_t last = ctas % slots == 0 ? slots : ctas % slots;
                if (last > best) {
                    best = last;
                    kchunk = c;
                }
            }
        }
    }
    const int64_t gz = (g.nz + kchunk - 1) / kchunk;
    if (tiles > 0x7fffffffLL || gz > 65535) return cudaErrorInvalidConfiguration;
    AdjFxParams p{g.nx, g.ny, g.nz, kchunk, (int)ntx, step % kFxSlots, (step + 1) % kFxSlots,
                  (step + 2) % kFxSlots};
    k_adjoint_fx<BY, NST><<<dim3((unsigned)tiles, (unsigned)gz, 1), 32 * BY, smem, s>>>(
        mT, mY, mC, Yout, Csbar, (FxSlot *)state, p);
    return cudaGetLastError();
}

unsigned adjoint_fx_device_error(bool clear) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_adjfx_error, sizeof(v));
    if (clear) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_adjfx_error, &z, sizeof(z));
    }
    return v;
}

}  // namespace psd

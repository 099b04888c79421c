// FP64 step arithmetic with one (or two) FP64 instructions per node.
//
// The GB300 runs FP64 instructions (DFMA, DADD and every FP64<->FP32/INT
// conversion) at about 1/58 of the FP32 rate, so a plain FP64 evaluation of
// Fig. 1's step (about nine FP64 instructions per node) is bound by the FP64
// pipe at roughly a quarter of the HBM rate.  These routines compute the
// same update with integer instructions plus a single DFMA:
//
//   T2 = fma(Ci, L, T),   L = K * S * 2^sc,
//
// where S is the sum of the six neighbours minus six times the centre (or one
// such sum per axis), formed EXACTLY in 64-bit integer arithmetic, K =
// dt*lam*_d^2 is a host constant, and the product K*S is formed with a 64x64
// bit high multiply and packed into an FP64 bit pattern with integer ops.
// The kDmul variant instead packs S exactly and spends a second FP64
// instruction on Ci*K:  T2 = fma(Ci*K, S*2^sc, T).
//
//  * Fast path: when all seven values share sign and exponent, the
//    difference of two FP64 bit patterns is the difference of the values in
//    units of the common ulp, so S needs no conversion at all (for negative
//    values the bit difference is minus the value difference; the sign of
//    the packed result is flipped instead).
//  * General path (other nodes): every value is converted to fixed point at
//    the largest exponent among the seven (57-bit magnitudes), then summed.
//    Per node it is a separate, non-inlined function reached by a branch, so
//    nodes on the fast path never execute it; the z-march tiles instead take
//    emu_lane_general (the same arithmetic, inlined) for all nodes of every lane
//    of a warp at once, so the warp does not diverge.
//  * Inf/NaN inputs fall back to the plain FP64 expression.
//
// Error: the fast path forms S exactly.  The general path keeps each value's
// bits down to 2^-56 of the largest of the seven (a value more than four binades
// below it loses low-order bits, one 57 or more binades below loses all of them),
// so S is exact when the seven span at most five binades and otherwise within
// 7 * 2^-56 of the largest value.  K*S keeps >= 60 bits before one
// round-to-nearest into 53 bits; the DFMA rounds once more.  Per step this stays
// within a few units in the last place of the stencil's largest value.
#pragma once

#include <cstdint>
#include <cstring>

namespace psd {

// K = m * 2^e with m in [2^62, 2^63).
struct EmuK {
    unsigned long long m;
    int e;
};

__host__ __device__ inline EmuK emu_const(double K) {
    // K > 0 normal: K = (2^52 + f) * 2^(k-52) = ((2^52 + f) << 10) * 2^(k-62)
    unsigned long long b;
    memcpy(&b, &K, 8);
    const int k = (int)((b >> 52) & 0x7ff) - 1023;
    const unsigned long long man = (b & 0xfffffffffffffull) | (1ull << 52);
    return EmuK{man << 10, k - 62};
}

struct EmuCoef {
    EmuK kx, ky, kz;  // dt*lam*_d^2 per axis as integer mantissa and exponent
    double dtlam, ax, ay, az;
    double Kx;        // dt*lam*_dx^2 (the kDmul variant, iso grids)
};

__device__ __forceinline__ unsigned long long dbits(double d) {
    return (unsigned long long)__double_as_longlong(d);
}
__device__ __forceinline__ double bitsd(unsigned long long b) {
    return __longlong_as_double((long long)b);
}
__device__ __forceinline__ int emu_exp(unsigned long long v) { return (int)((v >> 52) & 0x7ff); }

// FP64 bit pattern nearest to K * |S| * 2^sc, S an exact signed integer
// (sign bit not set; the caller applies the sign).  Zero for S == 0; below the
// normal range the subnormal nearest to the kept product bits (gradual underflow);
// Inf from 2^1024 up.
__device__ __forceinline__ unsigned long long emu_scaled_mag(unsigned long long a, int sc, EmuK K) {
    const int lz = __clzll((long long)a);  // 64 when a == 0
    a <<= (lz & 63);
    const unsigned long long P = __umul64hi(a, K.m);  // [2^61, 2^63) unless a == 0
    const int top = (int)(P >> 62);
    // top: P in [2^62, 2^63) -> 53-bit mantissa P >> 10; else (2P) >> 10 = P >> 9
    const int sh = 9 + top;
    const unsigned long long M = (P + (1ull << (sh - 1))) >> sh;  // [2^52, 2^53], rounded
    const int be = 125 + top + K.e + sc - lz + 1022;            // biased exponent - 1
    if ((unsigned)be >= 0x7feu) {  // outside the normal range (one compare on the common path)
        if (be > 0) return a == 0ull ? 0ull : 0x7ff0000000000000ull;  // |value| >= 2^1024: Inf
        // subnormal: the mantissa in units of 2^-1074 is P * 2^(be - sh), rounded to nearest
        // (a carry into bit 52 gives the smallest normal, as it should)
        const int s2 = sh - be;
        return s2 >= 64 ? 0ull : (P + (1ull << (s2 - 1))) >> s2;
    }
    const unsigned long long bits = ((unsigned long long)(long long)be << 52) + M;
    return a == 0ull ? 0ull : bits;
}

// The FP64 bit pattern of |S| * 2^sc for a result known to be normal or zero (rounded to
// nearest when |S| >= 2^53): the fast paths, whose common binade lies in the exponent range
// that emu_same_binade_hi admits, so no range check is spent on them.
__device__ __forceinline__ unsigned long long emu_pack_mag_normal(unsigned long long a, int sc) {
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << (lz & 63);              // leading one at bit 63
    const unsigned long long M = (n + 0x400ull) >> 11;        // [2^52, 2^53]
    const int be = 63 - lz + sc + 1022;
    const unsigned long long bits = ((unsigned long long)(long long)be << 52) + M;
    return a == 0ull ? 0ull : bits;
}

// Exact FP64 bit pattern of |S| * 2^sc (rounded to nearest when |S| >= 2^53; Inf from
// 2^1024 up).  Below the normal range it is the subnormal |S| * 2^(sc + 1074) in units of
// 2^-1074, exact: every
// sum these routines pack is a whole multiple of 2^-1074 (sc >= -1074 on the fast and
// window paths; on the general path at sc = emax' - 1079 < -1074 the sum is a multiple
// of 2^(5 - emax') units, since no value of exponent >= 1 loses bits there).
__device__ __forceinline__ unsigned long long emu_pack_mag(unsigned long long a, int sc) {
    const int lz = __clzll((long long)a);
    const int be = 63 - lz + sc + 1022;
    if ((unsigned)be >= 0x7feu) {  // outside the normal range (one compare on the common path)
        if (be > 0) return 0x7ff0000000000000ull;  // |value| >= 2^1024: Inf (a != 0 here)
        const int t = sc + 1074;
        return t >= 0 ? (a << t) : (a >> -t);
    }
    const unsigned long long n = a << (lz & 63);              // leading one at bit 63
    const unsigned long long M = (n + 0x400ull) >> 11;        // [2^52, 2^53]
    const unsigned long long bits = ((unsigned long long)(long long)be << 52) + M;
    return a == 0ull ? 0ull : bits;
}

__device__ __forceinline__ unsigned long long emu_abs(long long S, unsigned long long *sign) {
    const unsigned long long neg = (unsigned long long)(S >> 63);
    *sign = neg & 0x8000000000000000ull;
    return ((unsigned long long)S ^ neg) - neg;
}

// d | (a ^ c) and (a ^ c) | (b ^ c) as single 3-input logic instructions.
__device__ __forceinline__ unsigned lop_or_xor(unsigned d, unsigned a, unsigned c) {
    unsigned r;
    asm("lop3.b32 %0, %1, %2, %3, 0xF6;" : "=r"(r) : "r"(d), "r"(a), "r"(c));
    return r;
}
__device__ __forceinline__ unsigned lop_xor_or(unsigned a, unsigned b, unsigned c) {
    unsigned r;
    asm("lop3.b32 %0, %1, %2, %3, 0x7E;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// Biased exponents of the binades the fast paths take: a sum of seven values of one
// binade e, packed at scale 2^(e - 1075), is then a normal double (or zero) - its
// exponent lies between e - 53 and e + 3 - so the fast packs need no range check.
// Values outside (below 2^-970 or from 2^1020) take the general path.
__device__ __forceinline__ bool emu_fast_exponent(unsigned hc) {
    return ((hc >> 20) & 0x7ffu) - 53u <= 2042u - 53u;
}

// True when every high word in h shares the sign and exponent field (top 12
// bits) with hc and hc's exponent is in the fast range (emu_fast_exponent, which
// leaves out Inf/NaN): then the FP64 values they belong to lie in one binade and
// their bit patterns differ by whole ulps.
template <int N>
__device__ __forceinline__ bool emu_same_binade_hi(const unsigned (&h)[N], unsigned hc) {
    unsigned d = lop_xor_or(h[0], h[1], hc);
#pragma unroll
    for (int i = 2; i < N; ++i) d = lop_or_xor(d, h[i], hc);
    return (d & 0xfff00000u) == 0u && emu_fast_exponent(hc);
}

// True when the six neighbours share sign and exponent with the centre and that
// exponent is in the fast range (emu_fast_exponent).
__device__ __forceinline__ bool emu_same_binade(unsigned long long c, unsigned long long xm,
                                                unsigned long long xp, unsigned long long ym,
                                                unsigned long long yp, unsigned long long zm,
                                                unsigned long long zp) {
    const unsigned hc = (unsigned)(c >> 32);
    const unsigned d = ((unsigned)(xm >> 32) ^ hc) | ((unsigned)(xp >> 32) ^ hc) |
                       ((unsigned)(ym >> 32) ^ hc) | ((unsigned)(yp >> 32) ^ hc) |
                       ((unsigned)(zm >> 32) ^ hc) | ((unsigned)(zp >> 32) ^ hc);
    return ((d & 0xfff00000u) == 0u) && emu_fast_exponent(hc);
}

// L (as FP64 bits, with sign) from exact per-axis sums at scale 2^sc.
template <bool kIso>
__device__ __forceinline__ double emu_L(long long sx, long long sy, long long sz, int sc,
                                        unsigned long long flip, const EmuCoef &k) {
    unsigned long long sg;
    if (kIso) {
        const unsigned long long a = emu_abs(sx + sy + sz, &sg);
        return bitsd(emu_scaled_mag(a, sc, k.kx) | (sg ^ flip));
    } else {
        unsigned long long s1, s2, s3;
        const unsigned long long ax = emu_abs(sx, &s1), ay = emu_abs(sy, &s2), az = emu_abs(sz, &s3);
        const double L = (bitsd(emu_scaled_mag(ax, sc, k.kx) | s1) +
                          bitsd(emu_scaled_mag(ay, sc, k.ky) | s2)) +
                         bitsd(emu_scaled_mag(az, sc, k.kz) | s3);
        return bitsd(dbits(L) ^ flip);
    }
}

// Fast path (caller checked emu_same_binade).
template <bool kIso, bool kDmul>
__device__ __forceinline__ double emu_fast_node(unsigned long long c, unsigned long long xm,
                                                unsigned long long xp, unsigned long long ym,
                                                unsigned long long yp, unsigned long long zm,
                                                unsigned long long zp, double ci,
                                                const EmuCoef &k) {
    // bit-pattern differences = value differences in ulps of the common binade
    const unsigned long long c2 = c + c;
    const long long sx = (long long)(xm + xp - c2);
    const long long sy = (long long)(ym + yp - c2);
    const long long sz = (long long)(zm + zp - c2);
    const int e = emu_exp(c);
    const int sc = (e ? e : 1) - 1075;
    const unsigned long long flip = c & 0x8000000000000000ull;  // negative values: minus
    if (kDmul && kIso) {
        unsigned long long sg;
        const unsigned long long a = emu_abs(sx + sy + sz, &sg);
        const double Sd = bitsd(emu_pack_mag_normal(a, sc) | (sg ^ flip));
        return fma(ci * k.Kx, Sd, bitsd(c));
    }
    return fma(ci, emu_L<kIso>(sx, sy, sz, sc, flip, k), bitsd(c));
}

// Signed fixed-point value of FP64 bits v at scale 2^(Emax' - 1079), where
// Emax' = max(Emax, 1) is the largest biased exponent of the group (57-bit
// magnitudes: a value more than 4 binades below Emax' loses low-order bits, one
// 57 or more below becomes 0).
__device__ __forceinline__ long long emu_fixed(unsigned long long v, int emax1) {
    const int e = (int)((v >> 52) & 0x7ff);
    const unsigned long long man = (v & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
    const int r = emax1 - (e ? e : 1);
    const unsigned long long x = r < 64 ? ((man << 4) >> r) : 0ull;
    return (v >> 63) ? -(long long)x : (long long)x;
}

// General path: any signs and exponents (rare for smooth fields).
template <bool kIso>
__device__ __noinline__ double emu_general_node(unsigned long long c, unsigned long long xm,
                                                unsigned long long xp, unsigned long long ym,
                                                unsigned long long yp, unsigned long long zm,
                                                unsigned long long zp, double ci,
                                                const EmuCoef k) {
    int em = emu_exp(c);
    em = max(em, max(emu_exp(xm), emu_exp(xp)));
    em = max(em, max(emu_exp(ym), emu_exp(yp)));
    em = max(em, max(emu_exp(zm), emu_exp(zp)));
    if (em == 0x7ff) {  // Inf / NaN somewhere: plain FP64 propagates it
        const double cc = bitsd(c);
        const double d2x = (bitsd(xp) - cc) - (cc - bitsd(xm));
        const double d2y = (bitsd(yp) - cc) - (cc - bitsd(ym));
        const double d2z = (bitsd(zp) - cc) - (cc - bitsd(zm));
        return cc + k.dtlam * (ci * ((d2x * k.ax + d2y * k.ay) + d2z * k.az));
    }
    const int em1 = em ? em : 1;
    const long long fc2 = 2 * emu_fixed(c, em1);
    const long long sx = emu_fixed(xm, em1) + emu_fixed(xp, em1) - fc2;
    const long long sy = emu_fixed(ym, em1) + emu_fixed(yp, em1) - fc2;
    const long long sz = emu_fixed(zm, em1) + emu_fixed(zp, em1) - fc2;
    return fma(ci, emu_L<kIso>(sx, sy, sz, em1 - 1079, 0ull, k), bitsd(c));
}

// Exact per-axis second-difference sums of seven arbitrary finite FP64 values
// (bit patterns) in fixed point at the largest exponent of the seven:
// value(S_d) = S_d * 2^sc.  Returns false if any value is Inf/NaN.
__device__ __forceinline__ bool emu_sums_general(unsigned long long c, unsigned long long xm,
                                                 unsigned long long xp, unsigned long long ym,
                                                 unsigned long long yp, unsigned long long zm,
                                                 unsigned long long zp, long long &sx,
                                                 long long &sy, long long &sz, int &sc) {
    int em = emu_exp(c);
    em = max(em, max(emu_exp(xm), emu_exp(xp)));
    em = max(em, max(emu_exp(ym), emu_exp(yp)));
    em = max(em, max(emu_exp(zm), emu_exp(zp)));
    if (em == 0x7ff) return false;
    const int em1 = em ? em : 1;
    const long long fc2 = 2 * emu_fixed(c, em1);
    sx = emu_fixed(xm, em1) + emu_fixed(xp, em1) - fc2;
    sy = emu_fixed(ym, em1) + emu_fixed(yp, em1) - fc2;
    sz = emu_fixed(zm, em1) + emu_fixed(zp, em1) - fc2;
    sc = em1 - 1079;
    return true;
}

// Exact FP64 of S * 2^sc (signed), via emu_pack_mag.
__device__ __forceinline__ double emu_pack(long long S, int sc) {
    unsigned long long sg;
    const unsigned long long a = emu_abs(S, &sg);
    return bitsd(emu_pack_mag(a, sc) | sg);
}

// base + sum_d K_d * S_d * 2^sc with one DFMA per distinct coefficient
// (one in total when the grid is isotropic).  Kx/Ky/Kz are FP64 constants.
template <bool kIso>
__device__ __forceinline__ double emu_axpy3(double base, long long sx, long long sy, long long sz,
                                            int sc, double Kx, double Ky, double Kz) {
    if (kIso) return fma(Kx, emu_pack(sx + sy + sz, sc), base);
    return fma(Kz, emu_pack(sz, sc), fma(Ky, emu_pack(sy, sc), fma(Kx, emu_pack(sx, sc), base)));
}

// Pre-scaled coefficient (isotropic grids): cs = dt*lam*_d^2*Ci, so the node is
// T2 = fma(cs, S*2^sc, T) with S the exact sum of the six neighbours minus six
// times the centre: one FP64 instruction per node.
__device__ __forceinline__ double emu_fast_node_scaled(unsigned long long c, unsigned long long xm,
                                                       unsigned long long xp, unsigned long long ym,
                                                       unsigned long long yp, unsigned long long zm,
                                                       unsigned long long zp, double cs) {
    const unsigned long long c6 = 6ull * c;
    const long long S = (long long)(((xm + xp) + (ym + yp)) + (zm + zp) - c6);
    const int e = emu_exp(c);
    const unsigned long long flip = c & 0x8000000000000000ull;  // negative values: minus
    unsigned long long sg;
    const unsigned long long a = emu_abs(S, &sg);
    return fma(cs, bitsd(emu_pack_mag_normal(a, e - 1075) | (sg ^ flip)), bitsd(c));
}

static __device__ __noinline__ double emu_general_node_scaled(unsigned long long c, unsigned long long xm,
                                                       unsigned long long xp, unsigned long long ym,
                                                       unsigned long long yp, unsigned long long zm,
                                                       unsigned long long zp, double cs) {
    long long sx, sy, sz;
    int sc;
    if (!emu_sums_general(c, xm, xp, ym, yp, zm, zp, sx, sy, sz, sc)) {
        const double cc = bitsd(c);  // Inf / NaN: plain FP64 propagates it
        return cc + cs * ((((bitsd(xm) + bitsd(xp)) + (bitsd(ym) + bitsd(yp))) +
                           (bitsd(zm) + bitsd(zp))) - 6.0 * cc);
    }
    return fma(cs, emu_pack(sx + sy + sz, sc), bitsd(c));
}

__device__ __forceinline__ double emu_step_node_scaled(unsigned long long c, unsigned long long xm,
                                                       unsigned long long xp, unsigned long long ym,
                                                       unsigned long long yp, unsigned long long zm,
                                                       unsigned long long zp, double cs) {
    if (emu_same_binade(c, xm, xp, ym, yp, zm, zp))
        return emu_fast_node_scaled(c, xm, xp, ym, yp, zm, zp, cs);
    return emu_general_node_scaled(c, xm, xp, ym, yp, zm, zp, cs);
}

// General path for the PX stencils of one thread at once (a warp whose lanes do
// not all pass the same-binade check takes it for every lane, so the warp does not
// diverge, and nothing is called).  Node by node it is the arithmetic of
// emu_general_node(_scaled): the node's seven values in 57-bit fixed point at the
// largest of their exponents, exact integer sums, one pack - so its results are
// bit for bit those of the per-node general path that the fused-pair and column
// kernels take.  Inf/NaN among a node's values: plain FP64, which propagates it.
//   kScaled: out = fma(cs, S*2^sc, c) with ci = cs (pre-scaled coefficient);
//   else:    out = fma(ci, L, c), L = emu_L<kIso>(per-axis sums).
template <int PX, bool kScaled, bool kIso>
__device__ __forceinline__ void emu_lane_general(const unsigned long long (&c)[PX], unsigned long long xl,
                                                 unsigned long long xr, const unsigned long long (&ym)[PX],
                                                 const unsigned long long (&yp)[PX],
                                                 const unsigned long long (&zm)[PX],
                                                 const unsigned long long (&zp)[PX], const double (&ci)[PX],
                                                 const EmuCoef &k, double (&out)[PX]) {
#pragma unroll
    for (int i = 0; i < PX; ++i) {
        const unsigned long long xm = i == 0 ? xl : c[i - 1], xp = i == PX - 1 ? xr : c[i + 1];
        long long sx, sy, sz;
        int sc;
        if (emu_sums_general(c[i], xm, xp, ym[i], yp[i], zm[i], zp[i], sx, sy, sz, sc)) {
            if (kScaled)
                out[i] = fma(ci[i], emu_pack(sx + sy + sz, sc), bitsd(c[i]));
            else
                out[i] = fma(ci[i], emu_L<kIso>(sx, sy, sz, sc, 0ull, k), bitsd(c[i]));
        } else {  // Inf / NaN
            const double cc = bitsd(c[i]);
            if (kScaled) {
                out[i] = cc + ci[i] * ((((bitsd(xm) + bitsd(xp)) + (bitsd(ym[i]) + bitsd(yp[i]))) +
                                        (bitsd(zm[i]) + bitsd(zp[i]))) - 6.0 * cc);
            } else {
                const double d2x = (bitsd(xp) - cc) - (cc - bitsd(xm));
                const double d2y = (bitsd(yp[i]) - cc) - (cc - bitsd(ym[i]));
                const double d2z = (bitsd(zp[i]) - cc) - (cc - bitsd(zm[i]));
                out[i] = cc + k.dtlam * (ci[i] * ((d2x * k.ax + d2y * k.ay) + d2z * k.az));
            }
        }
    }
}

// True when every high word in h and hc has the sign of hc and a biased exponent in
// [e, e + 4] for one e in [53, 2038] (no zero, subnormal, Inf or NaN): the values lie,
// with one sign, in a window of five adjacent binades - where the general path's 57-bit
// fixed point is exact too, so both give the same sums - and their sums (below 2^61
// units of 2^(e-1075)) pack to normal doubles without range checks.  With one sign the
// words order as their magnitudes, so the smallest and largest word give the lowest and
// highest exponent.  *ewin = the top 12 bits (sign and exponent e) of the smallest word.
template <int N>
__device__ __forceinline__ bool emu_window_hi(const unsigned (&h)[N], unsigned hc, unsigned *ewin) {
    unsigned lo = hc, hi = hc, sg = 0u;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        lo = min(lo, h[i]);
        hi = max(hi, h[i]);
        sg = lop_or_xor(sg, h[i], hc);
    }
    const unsigned el = (lo >> 20) & 0x7ffu;
    *ewin = lo >> 20;
    return (sg & 0x80000000u) == 0u && (hi >> 20) - (lo >> 20) <= 4u && el - 53u <= 2038u - 53u;
}

// |v| in units of the ulp of binade e, for v of the window's sign and a biased exponent
// in [e, e + 4] (ewin = sign and e as emu_window_hi gives them): the 53-bit significand
// shifted left by the exponent difference (< 2^57).  Exact.
__device__ __forceinline__ long long emu_window_units(unsigned long long v, unsigned ewin) {
    const unsigned hi = (unsigned)(v >> 32);
    const int d = (int)((hi >> 20) & 0x7ffu) - (int)(ewin & 0x7ffu);
    const unsigned long long m = ((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | (unsigned)v;
    return (long long)(m << d);
}

// The PX stencils of one thread when all their values lie, with one sign, in a
// window of five binades (emu_window_hi; ewin: their sign and lowest exponent): each
// value becomes an exact integer in units of the lowest binade's ulp with a few integer
// instructions (|value| < 2^57 units, so the sums of seven stay below 2^61), the sums
// are exact, and the node finishes as on the general path (same real sum, same rounding: bit for
// bit emu_lane_general's result) at about half its cost.  flip: the values' sign.
template <int PX, bool kScaled, bool kIso>
__device__ __forceinline__ void emu_lane_window(const unsigned long long (&c)[PX], unsigned long long xl,
                                                unsigned long long xr, const unsigned long long (&ym)[PX],
                                                const unsigned long long (&yp)[PX],
                                                const unsigned long long (&zm)[PX],
                                                const unsigned long long (&zp)[PX], const double (&ci)[PX],
                                                const EmuCoef &k, unsigned ewin, double (&out)[PX]) {
    const unsigned long long flip = c[0] & 0x8000000000000000ull;
    const int sc = (int)(ewin & 0x7ffu) - 1075;
    long long uc[PX];
#pragma unroll
    for (int i = 0; i < PX; ++i) uc[i] = emu_window_units(c[i], ewin);
    const long long ul = emu_window_units(xl, ewin), ur = emu_window_units(xr, ewin);
#pragma unroll
    for (int i = 0; i < PX; ++i) {
        const long long uxm = i == 0 ? ul : uc[i - 1], uxp = i == PX - 1 ? ur : uc[i + 1];
        const long long c2 = 2 * uc[i];
        const long long sx = uxm + uxp - c2;
        const long long sy = emu_window_units(ym[i], ewin) + emu_window_units(yp[i], ewin) - c2;
        const long long sz = emu_window_units(zm[i], ewin) + emu_window_units(zp[i], ewin) - c2;
        if (kScaled) {
            unsigned long long sg;
            const unsigned long long a = emu_abs(sx + sy + sz, &sg);
            out[i] = fma(ci[i], bitsd(emu_pack_mag_normal(a, sc) | (sg ^ flip)), bitsd(c[i]));
        } else {
            out[i] = fma(ci[i], emu_L<kIso>(sx, sy, sz, sc, flip, k), bitsd(c[i]));
        }
    }
}

// One node, either path (per-lane branch).
template <bool kIso, bool kDmul>
__device__ __forceinline__ double emu_step_node(unsigned long long c, unsigned long long xm,
                                                unsigned long long xp, unsigned long long ym,
                                                unsigned long long yp, unsigned long long zm,
                                                unsigned long long zp, double ci,
                                                const EmuCoef &k) {
    if (emu_same_binade(c, xm, xp, ym, yp, zm, zp))
        return emu_fast_node<kIso, kDmul>(c, xm, xp, ym, yp, zm, zp, ci, k);
    return emu_general_node<kIso>(c, xm, xp, ym, yp, zm, zp, ci, k);
}

}  // namespace psd

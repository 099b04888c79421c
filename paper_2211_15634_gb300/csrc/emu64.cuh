// FP64 step arithmetic with one FP64 instruction per node.
//
// The GB300 runs FP64 instructions (DFMA, DADD and every FP64<->FP32/INT
// conversion) at about 1/58 of the FP32 rate, so a plain FP64 evaluation of
// Fig. 1's step (about nine FP64 instructions per node) is bound by the FP64
// pipe at roughly a quarter of the HBM rate.  These routines compute the
// same update with integer and FP32-pipe instructions plus a single DFMA:
//
//   T2 = fma(Ci, L, T),   L = K * S * 2^sc,
//
// where S is the sum of the six neighbours minus six times the centre (or one
// such sum per axis), formed EXACTLY in 64-bit integer arithmetic, K =
// dt*lam*_d^2 is a host constant, and the product K*S is formed with a 64x64
// bit high multiply and packed into an FP64 bit pattern with integer ops.
//
//  * Fast path: when all seven values share sign and exponent, the
//    difference of two FP64 bit patterns is the difference of the values in
//    units of the common ulp, so S needs no conversion at all.
//  * General path (other nodes): every value is converted to fixed point at
//    the largest exponent among the seven (57-bit magnitudes), then summed.
//  * Inf/NaN inputs fall back to the plain FP64 expression.
//
// Error: S is exact (the general path truncates values more than 57 binades
// below the largest of the seven); K*S keeps >= 60 bits before one
// round-to-nearest into 53 bits; the DFMA rounds once more.  Per step this
// stays within a few units in the last place of T.
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

__device__ __forceinline__ unsigned long long dbits(double d) {
    return (unsigned long long)__double_as_longlong(d);
}
__device__ __forceinline__ double bitsd(unsigned long long b) {
    return __longlong_as_double((long long)b);
}

// FP64 nearest to K * S * 2^sc for an exact signed integer S.
__device__ __forceinline__ double emu_scaled(long long S, int sc, EmuK K) {
    const unsigned long long neg = (unsigned long long)(S >> 63);
    unsigned long long a = ((unsigned long long)S ^ neg) - neg;  // |S|
    const int lz = __clzll((long long)a);                        // 64 when S == 0
    a <<= (lz & 63);
    unsigned long long P = __umul64hi(a, K.m);                   // [2^61, 2^63) unless S == 0
    const int top = (int)(P >> 62);
    P = top ? P : (P << 1);
    const int be = 125 + top + K.e + sc - lz + 1022;             // biased exponent - 1
    const unsigned long long M = (P + 0x200ull) >> 10;           // [2^52, 2^53], rounded
    unsigned long long bits = ((unsigned long long)(long long)be << 52) + M;
    bits |= neg & 0x8000000000000000ull;
    bits = (a == 0ull || be < 0) ? 0ull : bits;                   // zero, or underflow -> 0
    return bitsd(bits);
}

// Signed fixed-point value of FP64 bits v at scale 2^(Emax' - 1079), where
// Emax' = max(Emax, 1) is the largest biased exponent of the group (57-bit
// magnitudes; values 64+ binades below Emax' become 0).
__device__ __forceinline__ long long emu_fixed(unsigned long long v, int emax1) {
    const int e = (int)((v >> 52) & 0x7ff);
    const unsigned long long man = (v & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
    const int r = emax1 - (e ? e : 1);
    const unsigned long long x = r < 64 ? ((man << 4) >> r) : 0ull;
    return (v >> 63) ? -(long long)x : (long long)x;
}

__device__ __forceinline__ int emu_exp(unsigned long long v) { return (int)((v >> 52) & 0x7ff); }

// True when the six neighbours share sign and exponent with the centre and the
// centre is finite.
__device__ __forceinline__ bool emu_same_binade(unsigned long long c, unsigned long long xm,
                                                unsigned long long xp, unsigned long long ym,
                                                unsigned long long yp, unsigned long long zm,
                                                unsigned long long zp) {
    const unsigned hc = (unsigned)(c >> 32);
    const unsigned d = ((unsigned)(xm >> 32) ^ hc) | ((unsigned)(xp >> 32) ^ hc) |
                       ((unsigned)(ym >> 32) ^ hc) | ((unsigned)(yp >> 32) ^ hc) |
                       ((unsigned)(zm >> 32) ^ hc) | ((unsigned)(zp >> 32) ^ hc);
    return ((d & 0xfff00000u) == 0u) && ((hc & 0x7ff00000u) != 0x7ff00000u);
}

struct EmuCoef {
    EmuK kx, ky, kz;  // dt*lam*_d^2 per axis
    double dtlam, ax, ay, az;
};

// One node of Fig. 1's step: returns T2 for centre c, neighbours, and Ci.
// kIso: the three axis coefficients are equal (one product instead of three).
template <bool kIso>
__device__ __forceinline__ double emu_step_node(unsigned long long c, unsigned long long xm,
                                                unsigned long long xp, unsigned long long ym,
                                                unsigned long long yp, unsigned long long zm,
                                                unsigned long long zp, double ci,
                                                const EmuCoef &k) {
    long long sx, sy, sz;
    int sc;
    if (emu_same_binade(c, xm, xp, ym, yp, zm, zp)) {
        // bit-pattern differences = value differences in ulps of the common binade
        const unsigned long long c2 = c << 1;
        sx = (long long)(xm + xp - c2);
        sy = (long long)(ym + yp - c2);
        sz = (long long)(zm + zp - c2);
        if (c >> 63) {
            sx = -sx;
            sy = -sy;
            sz = -sz;
        }
        const int e = emu_exp(c);
        sc = (e ? e : 1) - 1075;
    } else {
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
        sx = emu_fixed(xm, em1) + emu_fixed(xp, em1) - fc2;
        sy = emu_fixed(ym, em1) + emu_fixed(yp, em1) - fc2;
        sz = emu_fixed(zm, em1) + emu_fixed(zp, em1) - fc2;
        sc = em1 - 1079;
    }
    double L;
    if (kIso) {
        L = emu_scaled(sx + sy + sz, sc, k.kx);
    } else {
        L = (emu_scaled(sx, sc, k.kx) + emu_scaled(sy, sc, k.ky)) + emu_scaled(sz, sc, k.kz);
    }
    return fma(ci, L, bitsd(c));
}

}  // namespace psd

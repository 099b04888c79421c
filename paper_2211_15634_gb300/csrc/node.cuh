// Per-node update of Fig. 1's step shared by the one-step and the two-step
// z-march kernels, so that two fused steps give bit for bit the result of two
// single steps.
#pragma once

#include "emu64.cuh"

namespace psd {

// FP32: T2 = T + dt*lam*(Ci*((d2x*_dx^2 + d2y*_dy^2) + d2z*_dz^2)), with the
// roundings fixed by explicit intrinsics (no compiler-chosen contraction).
__device__ __forceinline__ float f32_node(float c, float xm, float xp, float ym, float yp, float zm,
                                          float zp, float ci, float dtlam, float ax, float ay,
                                          float az) {
    const float d2x = __fsub_rn(__fsub_rn(xp, c), __fsub_rn(c, xm));
    const float d2y = __fsub_rn(__fsub_rn(yp, c), __fsub_rn(c, ym));
    const float d2z = __fsub_rn(__fsub_rn(zp, c), __fsub_rn(c, zm));
    const float lap = __fmaf_rn(d2z, az, __fmaf_rn(d2y, ay, __fmul_rn(d2x, ax)));
    return __fmaf_rn(dtlam, __fmul_rn(ci, lap), c);
}

// FP32 three-axis Laplacian term of f32_node: (d2x*_dx^2 + d2y*_dy^2) + d2z*_dz^2.
__device__ __forceinline__ float f32_lap(float c, float xm, float xp, float ym, float yp, float zm,
                                         float zp, float ax, float ay, float az) {
    const float d2x = __fsub_rn(__fsub_rn(xp, c), __fsub_rn(c, xm));
    const float d2y = __fsub_rn(__fsub_rn(yp, c), __fsub_rn(c, ym));
    const float d2z = __fsub_rn(__fsub_rn(zp, c), __fsub_rn(c, zm));
    return __fmaf_rn(d2z, az, __fmaf_rn(d2y, ay, __fmul_rn(d2x, ax)));
}

// Compensated FP32 step on a two-float state: the value of a node is the unevaluated
// sum D + E of its FP32 value D and a small FP32 correction E (|E| <= ulp(D)/2 after
// a step).  The update of Fig. 1's step! is taken on the whole state,
//   delta = dt*lam*(Ci*(lap(D) + lap(E))),
// and added exactly: s = E + delta, then D2 + E2 = D + s by Knuth's TwoSum (six
// roundings, exact for any magnitudes), so the addition to the state loses nothing
// and only delta's own FP32 roundings remain.  e* are the E values at the stencil.
__device__ __forceinline__ float comp32_node(float c, float xm, float xp, float ym, float yp, float zm,
                                             float zp, float ec, float exl, float exr, float eyl,
                                             float eyr, float ezl, float ezr, float ci, float dtlam,
                                             float ax, float ay, float az, float *e_out) {
    const float lapD = f32_lap(c, xm, xp, ym, yp, zm, zp, ax, ay, az);
    const float lapE = f32_lap(ec, exl, exr, eyl, eyr, ezl, ezr, ax, ay, az);
    const float delta = __fmul_rn(dtlam, __fmul_rn(ci, __fadd_rn(lapD, lapE)));
    const float s = __fadd_rn(ec, delta);
    const float t = __fadd_rn(c, s);
    const float bp = __fsub_rn(t, c);
    const float ap = __fsub_rn(t, bp);
    *e_out = __fadd_rn(__fsub_rn(c, ap), __fsub_rn(s, bp));
    return t;
}

// FP64 on the pre-scaled coefficient cs = dt*lam*_d^2*Ci (equal spacings):
// T2 = T + cs*(sum of the six neighbours - 6 T), the sum formed exactly
// (emu64.cuh), one DFMA.
__device__ __forceinline__ double f64s_node(double c, double xm, double xp, double ym, double yp,
                                            double zm, double zp, double cs) {
    return emu_step_node_scaled(dbits(c), dbits(xm), dbits(xp), dbits(ym), dbits(yp), dbits(zm),
                                dbits(zp), cs);
}

}  // namespace psd

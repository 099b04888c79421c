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

// FP64 on the pre-scaled coefficient cs = dt*lam*_d^2*Ci (equal spacings):
// T2 = T + cs*(sum of the six neighbours - 6 T), the sum formed exactly
// (emu64.cuh), one DFMA.
__device__ __forceinline__ double f64s_node(double c, double xm, double xp, double ym, double yp,
                                            double zm, double zp, double cs) {
    return emu_step_node_scaled(dbits(c), dbits(xm), dbits(xp), dbits(ym), dbits(yp), dbits(zm),
                                dbits(zp), cs);
}

}  // namespace psd

// Per-node arithmetic of the FP32 transposed step, shared by the one-step and the
// two-step kernels (adjoint_f32.cu) so that a fused pair gives bit for bit the
// result of two single steps.  Roundings are fixed by explicit intrinsics (no
// compiler-chosen contraction).
//
// For ybar = dL/dT_{t+1}, state S = T_t, coefficient C and K_d = dt*lam*_d^2:
//   w        = C*ybar at interior nodes, 0 elsewhere,
//   Tbar     = ybar + sum_d K_d * ((w[+d] - w) - (w - w[-d]))          (every node),
//   Cibar   += ybar * sum_d K_d * ((S[+d] - S) - (S - S[-d]))          (interior nodes).
#pragma once

namespace psd {

__device__ __forceinline__ float a32_w(float c, float y, bool interior) {
    return interior ? __fmul_rn(c, y) : 0.f;
}

// sum_d K_d * second difference of the seven values (x, y, z order)
__device__ __forceinline__ float a32_lap(float c, float xm, float xp, float ym, float yp, float zm,
                                         float zp, float Kx, float Ky, float Kz) {
    const float d2x = __fsub_rn(__fsub_rn(xp, c), __fsub_rn(c, xm));
    const float d2y = __fsub_rn(__fsub_rn(yp, c), __fsub_rn(c, ym));
    const float d2z = __fsub_rn(__fsub_rn(zp, c), __fsub_rn(c, zm));
    return __fmaf_rn(d2z, Kz, __fmaf_rn(d2y, Ky, __fmul_rn(d2x, Kx)));
}

__device__ __forceinline__ float a32_tbar(float y, float lap_w) { return __fadd_rn(y, lap_w); }

__device__ __forceinline__ float a32_cibar(float cb, float y, float lap_s) { return __fmaf_rn(y, lap_s, cb); }

}  // namespace psd

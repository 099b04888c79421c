// FP32 forward step dispatch (deviation storage D = T - T_ref): TMA z-march
// when nx is a multiple of 4, else the plain column march.
#include "internal.h"
#include "stencil_basic.cuh"
#include "zmarch.h"

namespace psd {

static CoefT<float> coef_f32(StepCoef c) {
    return CoefT<float>{(float)c.dtlam, (float)c.ax, (float)c.ay, (float)c.az};
}

cudaError_t launch_step_f32(float *T2, const float *T, const float *Ci, StepCoef c, Grid3 g,
                            cudaStream_t s, bool write_bnd) {
    if (step_tma_ok(g, 4, T2, T, Ci))
        return launch_zmarch(Z_F32, T2, T, nullptr, nullptr, Ci, c, g, s, write_bnd);
    return launch_step_basic<float, false>(T2, T, nullptr, nullptr, Ci, coef_f32(c), g.nx, g.ny, g.nz,
                                           sm_count(), s);
}

// Two-float state (D, E) -> (D2, E2): the TMA z-march stages E like T.
cudaError_t launch_step_f32_comp(float *T2, const float *T, float *E2, const float *E, const float *Ci,
                                 StepCoef c, Grid3 g, cudaStream_t s) {
    if (step_tma_ok(g, 4, T2, T, Ci) && step_tma_ok(g, 4, E2, E, Ci))
        return launch_zmarch(Z_F32_COMP, T2, T, E2, E, Ci, c, g, s);
    return launch_step_basic<float, true>(T2, T, E2, E, Ci, coef_f32(c), g.nx, g.ny, g.nz,
                                          sm_count(), s);
}

const char *step_f32_kernel_name(Grid3 g, const void *T2, const void *T, const void *Ci) {
    return step_tma_ok(g, 4, T2, T, Ci) ? "k_zmarch<F32>" : "k_step_basic<float>";
}

}  // namespace psd

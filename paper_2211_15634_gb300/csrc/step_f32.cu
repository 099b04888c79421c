// FP32 forward step kernels (deviation storage D = T - T_ref).
#include "internal.h"
#include "stencil_basic.cuh"

namespace psd {

static CoefT<float> coef_f32(StepCoef c) {
    return CoefT<float>{(float)c.dtlam, (float)c.ax, (float)c.ay, (float)c.az};
}

cudaError_t launch_step_f32(float *T2, const float *T, const float *Ci, StepCoef c, Grid3 g,
                            cudaStream_t s) {
    return launch_step_basic<float, false>(T2, T, nullptr, Ci, coef_f32(c), g.nx, g.ny, g.nz,
                                           sm_count(), s);
}

cudaError_t launch_step_f32_comp(float *T2, const float *T, float *comp, const float *Ci,
                                 StepCoef c, Grid3 g, cudaStream_t s) {
    return launch_step_basic<float, true>(T2, T, comp, Ci, coef_f32(c), g.nx, g.ny, g.nz,
                                          sm_count(), s);
}

}  // namespace psd

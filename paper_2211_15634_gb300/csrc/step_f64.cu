// FP64 forward step kernels.
#include "internal.h"
#include "stencil_basic.cuh"

namespace psd {

static CoefT<double> coef_f64(StepCoef c) { return CoefT<double>{c.dtlam, c.ax, c.ay, c.az}; }

cudaError_t launch_step_f64_native(double *T2, const double *T, const double *Ci, StepCoef c,
                                   Grid3 g, cudaStream_t s) {
    return launch_step_basic<double, false>(T2, T, nullptr, Ci, coef_f64(c), g.nx, g.ny, g.nz,
                                            sm_count(), s);
}

cudaError_t launch_step_f64_fast(double *T2, const double *T, const double *Ci, StepCoef c,
                                 Grid3 g, cudaStream_t s) {
    return launch_step_f64_native(T2, T, Ci, c, g, s);
}

}  // namespace psd

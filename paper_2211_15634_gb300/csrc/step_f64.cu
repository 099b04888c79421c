// FP64 forward step dispatch.
//   fast:   TMA z-march with one-DFMA emulated arithmetic (even nx), else the
//           plain column march with the same arithmetic;
//   native: plain column march with ordinary FP64 instructions.
#include "internal.h"
#include "stencil_basic.cuh"
#include "zmarch.h"

namespace psd {

static CoefT<double> coef_f64(StepCoef c) { return CoefT<double>{c.dtlam, c.ax, c.ay, c.az}; }

cudaError_t launch_step_f64_native(double *T2, const double *T, const double *Ci, StepCoef c,
                                   Grid3 g, cudaStream_t s) {
    return launch_step_basic<double, false>(T2, T, nullptr, nullptr, Ci, coef_f64(c), g.nx, g.ny, g.nz,
                                            sm_count(), s);
}

static bool emu_ok(StepCoef c) {
    const double k[3] = {c.dtlam * c.ax, c.dtlam * c.ay, c.dtlam * c.az};
    for (double v : k)
        if (!(v > 2.2250738585072014e-308 && v < 1e300)) return false;  // positive normal
    return true;
}

cudaError_t launch_step_f64_fast(double *T2, const double *T, const double *Ci, StepCoef c,
                                 Grid3 g, cudaStream_t s, bool write_bnd) {
    if (!emu_ok(c)) return launch_step_f64_native(T2, T, Ci, c, g, s);
    const bool iso = c.ax == c.ay && c.ay == c.az;
    if (step_tma_ok(g, 8, T2, T, Ci))
        return launch_zmarch(iso ? Z_F64_EMU_ISO : Z_F64_EMU_ANISO, T2, T, nullptr, nullptr, Ci, c, g, s,
                             write_bnd);
    const EmuCoef ek{emu_const(c.dtlam * c.ax), emu_const(c.dtlam * c.ay), emu_const(c.dtlam * c.az),
                     c.dtlam, c.ax, c.ay, c.az, c.dtlam * c.ax};
    return launch_step_basic_emu(T2, T, Ci, ek, iso, g.nx, g.ny, g.nz, sm_count(), s);
}

// Ci already scaled to dt*lam*_dx^2*Ci (isotropic grids): one DFMA per node.
cudaError_t launch_step_f64_scaled(double *T2, const double *T, const double *Cs, Grid3 g,
                                   cudaStream_t s, bool write_bnd) {
    const StepCoef dummy{1.0, 1.0, 1.0, 1.0};
    if (step_tma_ok(g, 8, T2, T, Cs))
        return launch_zmarch(Z_F64_SCALED, T2, T, nullptr, nullptr, Cs, dummy, g, s, write_bnd);
    const EmuCoef ek{};
    return launch_step_basic_emu(T2, T, Cs, ek, true, g.nx, g.ny, g.nz, sm_count(), s, true);
}

bool step_writes_xy_boundary(int dtype, bool scaled, bool native, StepCoef c, Grid3 g, const void *T2,
                             const void *T, const void *Ci) {
    if (dtype != PS_F64) return step_tma_ok(g, 4, T2, T, Ci);  // launch_step_f32
    if (scaled) return step_tma_ok(g, 8, T2, T, Ci);           // launch_step_f64_scaled
    if (native || !emu_ok(c)) return false;                     // the plain column kernel
    return step_tma_ok(g, 8, T2, T, Ci);                        // launch_step_f64_fast
}

const char *step_f64_kernel_name(Grid3 g, const void *T2, const void *T, const void *Ci, StepCoef c,
                                 bool scaled) {
    if (scaled) {
        if (!step_tma_ok(g, 8, T2, T, Ci)) return "k_step_basic_emu";
        return f64_scaled_wide(g, T2, T, Ci) ? "k_zmarch<F64_SCALED4>" : "k_zmarch<F64_SCALED>";
    }
    if (!emu_ok(c)) return "k_step_basic<double>";
    const bool iso = c.ax == c.ay && c.ay == c.az;
    if (step_tma_ok(g, 8, T2, T, Ci)) return iso ? "k_zmarch<F64_EMU_ISO>" : "k_zmarch<F64_EMU_ANISO>";
    return "k_step_basic_emu";
}

}  // namespace psd

// Declarations of the TMA-fed z-march step kernels (zmarch.cu).
#pragma once

#include <cuda.h>

#include "emu64.cuh"
#include "internal.h"

namespace psd {

enum ZMode {
    Z_F64_EMU_ISO = 0,       // one DFMA per node, 64x64 high multiply by K
    Z_F64_EMU_ANISO = 1,     // as above, one product per axis
    Z_F64_NATIVE = 2,        // plain FP64 instructions
    Z_F32 = 3,
    Z_F32_COMP = 4,
    Z_F64_EMU_ISO_DMUL = 5,  // two FP64 ops per node: fma(Ci*K, S, T)
    Z_F64_SCALED = 6,        // Ci already holds dt*lam*_d^2*Ci: fma(Cs, S, T)
    Z_F64_SCALED4 = 7,       // as Z_F64_SCALED, four nodes per thread (32-byte accesses)
};

struct ZParams {
    int64_t nx, ny, nz;
    int64_t pitch;  // elements between consecutive rows (nx for a contiguous grid)
    int kchunk, ntx;
    EmuCoef ek;
    float fdtlam, fax, fay, faz;
};

// True when the TMA path can serve this grid and these pointers.
bool zmarch_supported(Grid3 g, int esz, const void *a, const void *b, const void *c);
// The same for one forward step, unless PS_OVERRIDE_STEP_PLAIN asks for the plain kernel.
bool step_tma_ok(Grid3 g, int esz, const void *a, const void *b, const void *c);
// 3-D tiled tensor map over a (nz, ny, nx) field with a bx x by x 1 box.
bool make_tensor_map_3d(CUtensorMap *m, const void *ptr, int esz, Grid3 g, unsigned bx, unsigned by);
// The same over a grid whose rows are `pitch` elements apart (pitch*esz a multiple of 16).
bool make_tensor_map_3d_pitch(CUtensorMap *m, const void *ptr, int esz, Grid3 g, int64_t pitch,
                              unsigned bx, unsigned by);
// True when the driver's tensor-map encoder could be loaded (a GPU driver is present).
bool tma_encoder_available();
// Whether the pre-scaled FP64 step takes the four-nodes-per-thread kernel (rows of a
// multiple of 32 bytes, 32-byte aligned fields; PS_F64_VARIANT=px2 turns it off).
bool f64_scaled_wide(Grid3 g, const void *T2, const void *T, const void *Ci);
// Step parameters of the z-march kernels for coefficients c on grid g with row pitch `pitch`.
ZParams zparams_for(StepCoef c, Grid3 g, int64_t pitch);

// TMA-fed transposed step (adjoint_zmarch.cu).
bool adjoint_zmarch_supported(Grid3 g, int esz, const void *const *ptrs, int nptr);
template <typename E>
cudaError_t launch_adjoint_zmarch(E *Tbar, E *Cibar, const E *ybar, const E *T, const E *Ci,
                                  StepCoef c, Grid3 g, cudaStream_t s);
unsigned adjoint_device_error(bool clear);
// TMA-fed transposed step on the pre-scaled coefficient (adjoint_scaled.cu).
cudaError_t launch_adjoint_scaled(double *Tbar, double *Csbar, const double *ybar, const double *T,
                                  const double *Cs, Grid3 g, cudaStream_t s);
// One step of the TMA z-march in `mode`; E2 / Ein: the correction fields of the
// two-float state (Z_F32_COMP only, else unused).  write_bnd: also store the x and y
// boundary nodes of planes 1 .. nz-2 as copies of T's (not with Z_F32_COMP).
cudaError_t launch_zmarch(int mode, void *T2, const void *T, void *E2, const void *Ein, const void *Ci,
                          StepCoef c, Grid3 g, cudaStream_t s, bool write_bnd = false);
unsigned zmarch_device_error(bool clear);

}  // namespace psd

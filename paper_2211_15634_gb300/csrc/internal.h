// Internal declarations shared by the library's translation units (host side).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "ps_diffusion3d.h"

namespace psd {

// Coefficients of one step, precomputed on the host in FP64 from the
// paper's arguments: dtlam = dt*lam and a_d = _d*_d (Fig. 1's _dx^2 ...).
struct StepCoef {
    double dtlam, ax, ay, az;
};

inline StepCoef make_coef(double lam, double dt, double _dx, double _dy, double _dz) {
    return StepCoef{dt * lam, _dx * _dx, _dy * _dy, _dz * _dz};
}

struct Grid3 {
    int64_t nx, ny, nz;
    int64_t n() const { return nx * ny * nz; }
};

// Number of SMs of the current device (cached per device).
int sm_count();
int current_device();

// Generation of the current device's context (grows after cudaDeviceReset), and a
// once-per-context cudaFuncSetAttribute(MaxDynamicSharedMemorySize) keyed on it:
// done_gen is a launcher's array of 64 generations; false (with *err) on failure.
unsigned context_generation();
bool set_smem_attr_once(const void *func, int smem, unsigned *done_gen, cudaError_t *err);

// Launch-shape override set through ps_set_launch_override (PS_OVERRIDE_*); 0 when
// unset, which leaves the choice to the library's own rule (abi.cu).
int launch_override(int which);

// Record a message for ps_last_error() and return the status (abi.cu).
int api_fail(int status, const char *msg);
int api_cuda_fail(cudaError_t e, const char *where);

// ---- forward step kernels (step_f64.cu, step_f32.cu) ----
// write_bnd: where the TMA z-march serves the step, it also stores the x and y boundary
// nodes of planes 1 .. nz-2 as copies of T's (step_writes_xy_boundary tells where).
cudaError_t launch_step_f64_native(double *T2, const double *T, const double *Ci, StepCoef c,
                                   Grid3 g, cudaStream_t s);
cudaError_t launch_step_f64_fast(double *T2, const double *T, const double *Ci, StepCoef c,
                                 Grid3 g, cudaStream_t s, bool write_bnd = false);
cudaError_t launch_step_f32(float *T2, const float *T, const float *Ci, StepCoef c, Grid3 g,
                            cudaStream_t s, bool write_bnd = false);
// True when the one-step launcher for these arguments takes the TMA z-march, so that
// write_bnd is honoured (FP64: scaled = PS_RUN_CI_SCALED, native = PS_RUN_NATIVE_F64).
bool step_writes_xy_boundary(int dtype, bool scaled, bool native, StepCoef c, Grid3 g, const void *T2,
                             const void *T, const void *Ci);
// compensated FP32 step on the two-float state (T, E) -> (T2, E2)
cudaError_t launch_step_f32_comp(float *T2, const float *T, float *E2, const float *E, const float *Ci,
                                 StepCoef c, Grid3 g, cudaStream_t s);
cudaError_t launch_step_f64_scaled(double *T2, const double *T, const double *Cs, Grid3 g,
                                   cudaStream_t s, bool write_bnd = false);
cudaError_t launch_scale_ci(double *Cs, const double *Ci, double K, int64_t n, cudaStream_t s);
// two steps per pass (zmarch2.cu): T2 = step(step(T)); the caller checks zmarch2_supported
// (the same preconditions as the one-step TMA kernel)
bool zmarch2_supported(Grid3 g, int esz, const void *a, const void *b, const void *c);
cudaError_t launch_step2_f32(float *T2, const float *T, const float *Ci, StepCoef c, Grid3 g,
                             cudaStream_t s);
cudaError_t launch_step2_f64_scaled(double *T2, const double *T, const double *Cs, Grid3 g,
                                    cudaStream_t s);
// A fused FP32 pair that keeps both states: T1 = step(T) to T1o, T2 = step(T1), both
// written at every node of planes 1 .. nz-2 (x and y faces as copies of T's).
cudaError_t launch_step2_states_f32(float *T1o, float *T2, const float *T, const float *Ci, StepCoef c,
                                    Grid3 g, cudaStream_t s);
unsigned zmarch2_device_error(bool clear);
const char *step_f64_kernel_name(Grid3 g, const void *T2, const void *T, const void *Ci, StepCoef c,
                                 bool scaled);
const char *step_f32_kernel_name(Grid3 g, const void *T2, const void *T, const void *Ci);
unsigned zmarch_device_error(bool clear);
cudaError_t launch_selftest_wait(unsigned polls, unsigned ns, cudaStream_t s);
unsigned adjoint_device_error(bool clear);
unsigned adjoint_scaled_device_error(bool clear);
// FP32 transposed step, every read staged by TMA (adjoint_f32.cu).
bool adjoint_f32_supported(Grid3 g, const void *const *ptrs, int nptr);
cudaError_t launch_adjoint_f32_tma(float *Tbar, float *Cibar, const float *ybar, const float *T,
                                   const float *Ci, StepCoef c, Grid3 g, cudaStream_t s);
unsigned adjoint_f32_device_error(bool clear);
// 2-D form of the step (diffusion2d.cu); mode is a ZMode: Z_F32, Z_F64_SCALED,
// Z_F64_EMU_ISO_DMUL or Z_F64_NATIVE
cudaError_t launch_step2d(int mode, void *T2, const void *T, const void *Ci, StepCoef c, int64_t nx,
                          int64_t ny, cudaStream_t s);
cudaError_t launch_copy_edges2d(void *T2, const void *T, int64_t nx, int64_t ny, int esz, cudaStream_t s);
// two FP32 transposed steps per pass (states S1 then S0), every read staged by TMA
cudaError_t launch_adjoint2_f32(float *Tbar, float *Cibar, const float *ybar, const float *S1,
                                const float *S0, const float *Ci, StepCoef c, Grid3 g, cudaStream_t s);

// ---- helpers (misc.cu) ----
cudaError_t launch_copy_boundary(void *T2, const void *T, Grid3 g, int elem_bytes, cudaStream_t s);
cudaError_t launch_copy_boundary_many(void *dst, int64_t count, int64_t gstride, const void *T,
                                      Grid3 g, int elem_bytes, cudaStream_t s, bool z_faces_only = false);
cudaError_t launch_to_deviation(float *D, const double *T, double t_ref, int64_t n, cudaStream_t s);
cudaError_t launch_from_deviation(double *T, const float *D, double t_ref, int64_t n,
                                  cudaStream_t s);
cudaError_t launch_to_deviation_pair(float *D, float *E, const double *T, double t_ref, int64_t n,
                                     cudaStream_t s);
cudaError_t launch_from_deviation_pair(double *T, const float *D, const float *E, double t_ref, int64_t n,
                                       cudaStream_t s);

// ---- adjoint (adjoint.cu) ----
cudaError_t launch_adjoint_f64(double *Tbar, double *Cibar, const double *ybar, const double *T,
                               const double *Ci, StepCoef c, Grid3 g, cudaStream_t s);
cudaError_t launch_adjoint_f64_scaled(double *Tbar, double *Csbar, const double *ybar,
                                      const double *T, const double *Cs, Grid3 g, cudaStream_t s);
cudaError_t launch_adjoint_f32(float *Tbar, float *Cibar, const float *ybar, const float *T,
                               const float *Ci, StepCoef c, Grid3 g, cudaStream_t s);

// ---- reductions (reduce.cu) ----
constexpr int kReduceBlocks = 1024;           // fixed partition => deterministic sums
constexpr size_t kWorkspaceBytes = 16384;     // >= kReduceBlocks doubles + one key
cudaError_t launch_maximum(double *out_dev, const void *A, int64_t n, int dtype, void *ws,
                           cudaStream_t s);
cudaError_t launch_dot(double *out_dev, const void *A, const void *B, int64_t n, int dtype,
                       void *ws, cudaStream_t s);
cudaError_t launch_half_sq_dist(double *out_dev, void *R, const void *A, const void *B, int64_t n,
                                int dtype, void *ws, cudaStream_t s);

// ---- batch (batch.cu) ----
struct BatchHeader {
    int64_t nprob, nitems;
    int32_t dtype, tile_x, tile_y, tile_z;
    int64_t problems_offset, items_offset;  // byte offsets from the table start
    // kernel 0: column march (batch.cu); 1: TMA z-march (batch_tma.cu) in step mode
    // zmode, with a ZParams record and three tensor maps per problem at these offsets
    int32_t kernel, zmode;
    int64_t zparams_offset, maps_offset;
    // z-march tables built for fused step pairs (PS_BATCH_TEMPORAL2): a second work list
    // of two-steps-per-pass items and a Z2Params record per problem (else nitems2 = 0)
    int64_t nitems2, items2_offset, z2params_offset;
};
struct BatchProblem {
    void *T;
    void *T2;
    const void *Ci;
    double dtlam, ax, ay, az;
    int64_t nx, ny, nz;
    int64_t pitch;  // elements between consecutive rows; planes are pitch*ny apart
    // one-DFMA-class emulated arithmetic constants (FP64): K_d = dtlam*a_d as
    // integer mantissa/exponent, and whether the three axes share one K
    unsigned long long kxm, kym, kzm;
    int32_t kxe, kye, kze, iso;
};
struct BatchItem {
    int32_t prob;
    int32_t i0, j0, k0;      // first interior node of the work item
    int16_t ni, nj, nk;       // extents (clipped to the interior; z-march: ni = nj = 0)
    int16_t kind;             // z-march: 0 a wide tile (one warp per row), 1 a narrow one
};
cudaError_t launch_batch_step(const void *dev_table, int parity, int dtype, cudaStream_t s);
unsigned batch_device_error(bool clear);
// TMA z-march batch (batch_tma.cu): tile width per dtype, tile height, the per-problem
// records (ZParams and three tensor maps), the launch (grid = one CTA per item)
// x-y tiles of the z-march over an nx x ny plane: (x0, y0, kind) into out[i].i0/.j0/.kind
// when out is not null; returns their number
int64_t batch_zmarch_xy_tiles(int dtype, int64_t nx, int64_t ny, BatchItem *out);
// fused-pair tiles (one width, 8 rows), kind 2; returns their number
int64_t batch_zmarch2_xy_tiles(int dtype, int64_t nx, int64_t ny, BatchItem *out);
constexpr int kBatchZmarchMaps = 9;  // tensor maps per problem (wide, narrow, fused pair)
bool batch_zmarch_fill(void *zparams_dst, void *z2params_dst, void *maps_dst, const BatchProblem &r,
                       StepCoef c, int dtype);
size_t batch_z2params_bytes();
cudaError_t launch_batch_zmarch2(const void *dev_table, int64_t nitems2, int dtype, int parity,
                                 cudaStream_t s);
cudaError_t launch_batch_zmarch(const void *dev_table, int64_t nitems, int zmode, int parity,
                                cudaStream_t s);
unsigned batch_zmarch_device_error(bool clear);
bool tma_encoder_available();
void batch_prepare(int dtype);
int batch_default_tile(int dtype, int *tx, int *ty, int *tz);

}  // namespace psd

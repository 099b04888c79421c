/*
 * ps_diffusion3d.h - C ABI of the GB300 (sm_103a) 3-D heat diffusion stencil.
 *
 * The operation is the explicit time step of the 3-D variable-coefficient
 * heat diffusion solver in Omlin & Raess, "High-performance xPU Stencil
 * Computations in Julia" (arXiv 2211.15634), Fig. 1:
 *
 *   step!(T2, T, Ci, lam, dt, _dx, _dy, _dz):
 *     @inn(T2) = @inn(T) + dt*(lam*@inn(Ci)*(@d2_xi(T)*_dx^2
 *                                          + @d2_yi(T)*_dy^2 + @d2_zi(T)*_dz^2))
 *
 * with @d2_di the three-point second difference along axis d at interior
 * nodes, iterated nt times with the two buffers swapped after every step
 * (Fig. 1 time loop) and the stable step dt = min(dx^2,dy^2,dz^2)/lam/
 * maximum(Ci)/6.1 (Fig. 1).  Boundary nodes are never written: they keep
 * their initial values in both buffers (Dirichlet), which is what
 * "T2 = copy(T)" in Fig. 1 sets up.
 *
 * ----------------------------------------------------------------------
 * Conventions that hold for every entry point
 * ----------------------------------------------------------------------
 * Layout   A field is one contiguous array of nx*ny*nz elements; node
 *          (i,j,k) is at offset i + nx*(j + ny*k) (x fastest, Julia's
 *          column-major T[i,j,k]).  Base pointers must be 16-byte aligned
 *          (any size works; rows need not be aligned).
 * Dtypes   PS_F64: every field is double.
 *          PS_F32: every field is float.  Temperature fields hold the
 *          deviation D = T - T_ref from a constant reference (the solver
 *          is exact under this shift because the second difference of a
 *          constant is zero and the boundary is fixed); ps_to_deviation /
 *          ps_from_deviation convert.
 * Memory   All field pointers are DEVICE pointers allocated and owned by
 *          the caller.  The library allocates no device memory on these
 *          calls.  Entry points that need scratch take a caller-owned
 *          device workspace of at least ps_workspace_bytes() bytes.  The
 *          two calls that return a host result (ps_maximum,
 *          ps_diffusion3d_stable_dt) keep a 64-byte pinned host slot per
 *          concurrent caller, allocated on first use and reused for the
 *          life of the context.
 * Streams  `stream` is a cudaStream_t (NULL = legacy default stream).
 *          Every call only enqueues work on it and returns; none
 *          synchronizes, except where a host result is returned
 *          (ps_maximum, ps_diffusion3d_stable_dt), which synchronize
 *          `stream` before returning.  The step and transposed-step
 *          kernels use programmatic dependent launch: one may be
 *          scheduled while the launch before it on the stream still
 *          runs, but it touches no memory until that launch has
 *          completed, so stream order holds as for any other launch.
 * Errors   Every entry point returns a ps_status.  Arguments are checked
 *          on the host before anything is launched; a failed check
 *          launches nothing.  PS_ERR_CUDA reports a CUDA error seen at
 *          launch.  ps_last_error() gives a message for the last non-OK
 *          status of the calling thread.  Nothing traps on the device.
 */
#ifndef PS_DIFFUSION3D_H
#define PS_DIFFUSION3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { PS_F32 = 0, PS_F64 = 1 } ps_dtype;

typedef enum {
    PS_OK = 0,
    PS_ERR_ARG = -1,         /* null pointer, size < 3, bad dtype, nt < 0, ... */
    PS_ERR_ALIAS = -2,       /* an output overlaps an input it must not overlap */
    PS_ERR_ALIGN = -3,       /* a base pointer is not 16-byte aligned */
    PS_ERR_CUDA = -4,        /* a CUDA call or launch failed */
    PS_ERR_UNSUPPORTED = -5  /* valid request this build cannot serve */
} ps_status;

/* Flags of ps_diffusion3d_run_ex. */
#define PS_RUN_GRAPH 1u       /* capture the nt launches into a CUDA graph once, replay it */
#define PS_RUN_COMPENSATED 2u /* PS_F32 only: compensated step on the two-float state,
                                 needs `comp` (see ps_diffusion3d_step_comp_f32) */
#define PS_RUN_NATIVE_F64 4u  /* PS_F64 only: force the plain FP64-instruction kernel */
#define PS_RUN_CI_SCALED 8u   /* PS_F64, equal spacings: Ci holds dt*lam*_dx^2*Ci (see
                                 ps_diffusion3d_scale_ci); lam, dt are then only checked */
#define PS_RUN_TEMPORAL2 16u  /* run only: two steps per pass (temporal blocking of depth
                                 2), bit for bit the same result; needs PS_F32 without
                                 PS_RUN_COMPENSATED, or PS_F64 with PS_RUN_CI_SCALED (else
                                 PS_ERR_UNSUPPORTED); grids the TMA kernels cannot serve
                                 (nx*sizeof not a multiple of 16) run single steps */

/* Library version (major*10000 + minor*100 + patch). */
int ps_version(void);

/* Message for the last non-OK status returned to the calling thread
 * ("" if none).  The pointer stays valid until the thread's next call. */
const char *ps_last_error(void);

/* Bytes of device workspace the reduction entry points need.  A reduction
 * reads and writes its workspace on its stream until it completes: one
 * workspace must not serve two reductions that may run at the same time (on
 * different streams); give each stream its own. */
size_t ps_workspace_bytes(void);

/* Device-side error flags of the current device, to *out_host (host
 * unsigned): bit 0 = a pipelined kernel gave up waiting for a shared-memory
 * stage (bounded wait) and left without writing its remaining output; bit 1 =
 * the column-march batch kernel was given a z-march table.  With
 * clear != 0 the flags are reset.  Synchronizes the device. */
int ps_device_error(unsigned *out_host, int clear);

/* Failure-path self-test (no fault): launches one CTA that waits on an
 * mbarrier nothing ever arrives on; the bounded wait gives up after `polls`
 * polls (1 .. 2^24) of at most `suspend_ns` ns each (1 .. 10^6) and sets bit
 * 0 of ps_device_error - the path a pipelined kernel takes when a shared-
 * memory stage never lands.  Asynchronous on `stream`. */
int ps_selftest_bounded_wait(unsigned polls, unsigned suspend_ns, void *stream);

/* Name of the kernel ps_diffusion3d_step_ex would launch for these arguments
 * and flags (for profiles and reports; no validation, launches nothing). */
const char *ps_diffusion3d_step_kernel(const void *T2, const void *T, const void *Ci, double lam,
                                       double dt, double _dx, double _dy, double _dz, int64_t nx,
                                       int64_t ny, int64_t nz, int dtype, unsigned flags);

/* ---------------------------------------------------------------------
 * Time step (Fig. 1, step!).  Writes the interior nodes of T2 from T and
 * Ci; T2's boundary is left untouched.  T2 must not overlap T or Ci.
 * lam, dt, _dx, _dy, _dz are the paper's arguments (_d = 1/d-spacing);
 * the kernel uses _d*_d.  nx, ny, nz >= 3.
 * dtype PS_F64: results match the FP64 definition to within a few units
 * in the last place per step (FMA contraction and association differ).
 * ------------------------------------------------------------------- */
int ps_diffusion3d_step(void *T2, const void *T, const void *Ci, double lam, double dt,
                        double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz,
                        int dtype, void *stream);

/* As ps_diffusion3d_step with flags: PS_RUN_CI_SCALED (Ci is the pre-scaled
 * field of ps_diffusion3d_scale_ci; PS_F64 and equal spacings, else
 * PS_ERR_UNSUPPORTED) or PS_RUN_NATIVE_F64. */
int ps_diffusion3d_step_ex(void *T2, const void *T, const void *Ci, double lam, double dt,
                           double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz,
                           int dtype, unsigned flags, void *stream);

/* Pre-scaled coefficient field for repeated FP64 steps on a grid with equal
 * spacings: Cs[p] = (dt*lam*_dx^2) * Ci[p] for p < n (FP64, device arrays;
 * Cs may be Ci itself, else must not overlap it).  With it the step is
 * T2 = T + Cs * (sum of the six neighbours - 6 T) - Fig. 1's step! with the
 * constant factors folded once per run - and needs one FP64 multiply-add per
 * node. */
int ps_diffusion3d_scale_ci(double *Cs, const double *Ci, double lam, double dt, double _dx,
                            int64_t n, void *stream);

/* Compensated FP32 step (the compensated-update variant of the FP32 form).
 * The state is a two-float pair: the value of node p is the unevaluated sum
 * T[p] + E[p] of the FP32 deviation T and a small FP32 correction E (start E
 * at 0, or at the residual ps_to_deviation_pair leaves).  The step is Fig. 1's
 * step! on that value: delta = dt*lam*Ci*(lap(T) + lap(E)) in FP32 (lap: the
 * three second differences times _d^2, Fig. 1's order), then the pair
 * (T2, E2) holds T + (E + delta) exactly (TwoSum), so rounding the state to
 * FP32 loses nothing from step to step; only delta's own FP32 roundings
 * remain.  Reads T, E (with their x/y/z neighbours) and Ci, writes the
 * interior of T2 and E2 (5 fields per step).  E2's boundary must equal E's
 * and T2's T's (ps_diffusion3d_run_ex with PS_RUN_COMPENSATED sets both).  E2
 * must not overlap T, T2, E or Ci; E must not overlap T2. */
int ps_diffusion3d_step_comp_f32(float *T2, const float *T, float *E2, const float *E, const float *Ci,
                                 double lam, double dt, double _dx, double _dy, double _dz,
                                 int64_t nx, int64_t ny, int64_t nz, void *stream);

/* Copy the six boundary faces of T into T2 (so that T2 = copy(T) holds on
 * the boundary, Fig. 1), leaving T2's interior untouched. */
int ps_diffusion3d_copy_boundary(void *T2, const void *T, int64_t nx, int64_t ny, int64_t nz,
                                 int dtype, void *stream);

/* The same for `count` grids stored one after another from dst, grid i at
 * dst + i*grid_stride elements (grid_stride >= nx*ny*nz and a multiple of 16
 * bytes, so that every grid keeps the 16-byte alignment the other calls
 * need), in one launch: state buffers that all keep T's boundary.  T must not
 * overlap them. */
int ps_diffusion3d_copy_boundary_many(void *dst, int64_t count, int64_t grid_stride,
                                      const void *T, int64_t nx, int64_t ny, int64_t nz, int dtype,
                                      void *stream);

/* ---------------------------------------------------------------------
 * Time loop (Fig. 1): copy T's boundary into T2, then nt steps, swapping
 * the roles of T and T2 after each.  On return *result_in_T2 (host int,
 * may be NULL) is 1 when the final state is in T2 (nt odd) and 0 when it is
 * in T.  T's interior is overwritten when nt >= 2.
 * ------------------------------------------------------------------- */
int ps_diffusion3d_run(void *T, void *T2, const void *Ci, double lam, double dt, double _dx,
                       double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz, int nt,
                       int dtype, void *stream, int *result_in_T2);

/* As ps_diffusion3d_run with flags (PS_RUN_*).  With PS_RUN_COMPENSATED
 * `comp` holds TWO float fields of nx*ny*nz values one after the other: the
 * correction E paired with T at comp[0 .. n) (the caller sets it: zeros, or the
 * E of ps_to_deviation_pair) and the one paired with T2 at comp[n .. 2n) (its
 * boundary is set from the first at the start); the final correction is in
 * the half paired with the buffer that holds the result.  Else `comp` is NULL.
 * With PS_RUN_GRAPH the nt launches are captured into a CUDA graph on the
 * first call for a given argument set and replayed afterwards (the graph
 * is cached inside the library until ps_clear_graph_cache()). */
int ps_diffusion3d_run_ex(void *T, void *T2, void *comp, const void *Ci, double lam, double dt,
                          double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz,
                          int nt, int dtype, unsigned flags, void *stream, int *result_in_T2);

/* Time loop that keeps states (the forward pass of a reverse sweep).  Runs
 * nt steps from T0 (not modified).  The state after step t goes to grid slot
 * t/every - 1 when every divides t, else to one of two work grids (slots
 * nt/every and nt/every + 1; none when every == 1), never the grid the step
 * reads.  Grid slot i is states + i*grid_stride elements (grid_stride >=
 * nx*ny*nz, a multiple of 16 bytes).  The call sets the boundary of every
 * grid it may write (the nt/every slots and the work grids) to T0's: where
 * the TMA z-march serves the steps, they store the x and y faces themselves
 * and only the two z faces are copied; else the whole boundary is copied
 * (the caller need not prepare the grids).  *final_slot = the slot holding
 * T(nt): >= 0 a state slot, -1 / -2 work grid 0 / 1, -3 T0 itself (nt = 0).
 * Flags: PS_RUN_CI_SCALED, PS_RUN_NATIVE_F64 as for ps_diffusion3d_step_ex;
 * PS_RUN_GRAPH captures the boundary copy and the nt launches into a CUDA
 * graph on the first call for this argument set (pointers, stride, every,
 * coefficients, sizes) and replays it afterwards.  Else one launch per step
 * from a host loop in the library.  PS_RUN_TEMPORAL2 (PS_F32, else
 * PS_ERR_UNSUPPORTED): the steps run as fused pairs, bit for bit the same
 * states - with every = 1 pairs that write both states (one pass over HBM per
 * two states: read the state and Ci, write two states); with every > 1 pairs
 * that never step over a kept state (a single step where one would).  Grids
 * the fused-pair kernel cannot serve run single steps.  Which work grid holds
 * T(nt) can differ from the single-step loop's (*final_slot says). */
int ps_diffusion3d_run_states(const void *T0, void *states, int64_t grid_stride, int every,
                              const void *Ci, double lam, double dt, double _dx, double _dy,
                              double _dz, int64_t nx, int64_t ny, int64_t nz, int nt, int dtype,
                              unsigned flags, void *stream, int *final_slot);

/* Destroy every cached CUDA graph.  The cache (PS_RUN_GRAPH of the 3-D and 2-D time
 * loops and the batch run) holds at most 256 graphs, keyed by the call's device,
 * pointers, coefficients, sizes and flags; beyond that the least recently replayed
 * one is destroyed (a graph still running is freed when it completes). */
int ps_clear_graph_cache(void);
/* Number of graphs in the cache. */
size_t ps_graph_cache_size(void);

/* ---------------------------------------------------------------------
 * Launch-shape overrides (no counterpart in the paper): for tests that
 * compare launch shapes bit for bit and for a tuner that times them.  Each
 * value is process-wide and read on the host at launch; 0 (the initial
 * value) leaves the choice to the library's own rule.  Chunk values are
 * planes (or rows) per CTA, 1 .. 4096; flag values 0 or 1.  The forward
 * steps' z-chunk and tile-width choices give bit for bit the same fields,
 * the plain compensated FP32 step equals the staged one bit for bit
 * (explicit roundings), and the other plain kernels agree with the staged
 * ones to rounding.  The FP64 transposed step holds w in fixed point at a
 * scale shared by a CTA's tile and z-chunk, so its chunk can change the
 * low-order bits of Tbar (values more than four binades below the largest
 * of the chunk lose bits below 2^-56 of it), within the stated tolerance.
 * Setting a value that differs from the current one empties the
 * CUDA-graph cache (a captured graph keeps the shapes of its capture).
 * ------------------------------------------------------------------- */
typedef enum {
    PS_OVERRIDE_KCHUNK = 0,     /* z-planes per CTA of the one-step z-march kernels */
    PS_OVERRIDE_KCHUNK2 = 1,    /* z-planes per CTA of the fused-pair kernels */
    PS_OVERRIDE_ADJ_KCHUNK = 2, /* z-planes per CTA of the staged transposed-step kernels */
    PS_OVERRIDE_CHUNK2D = 3,    /* rows per warp of the 2-D kernel */
    PS_OVERRIDE_ADJ_PLAIN = 4,  /* 1: transposed steps take the plain one-thread-per-column kernel */
    PS_OVERRIDE_F64_PX2 = 5,    /* 1: the pre-scaled FP64 step keeps two nodes per thread */
    PS_OVERRIDE_STEP_PLAIN = 6, /* 1: single forward steps take the plain one-thread-per-column
                                   kernel (fused pairs are not affected) */
    PS_OVERRIDE_COUNT = 7
} ps_override;
/* Set override `which` to `value` (PS_ERR_ARG when out of range). */
int ps_set_launch_override(int which, int value);
/* Current value of override `which` to *value (host int). */
int ps_get_launch_override(int which, int *value);

/* ---------------------------------------------------------------------
 * Adjoint of one step (the transpose of step!'s Jacobian; derived from
 * Fig. 1's step, no paper line).  With ybar = dL/dT_{t+1} and T = T_t,
 * the state the forward step read:
 *   w[q]      = dt*lam*Ci[q]*ybar[q] at interior q, 0 elsewhere;
 *   Tbar[p]   = ybar[p] + sum_d (w[p-e_d] - 2 w[p] + w[p+e_d]) * _d^2
 *               at EVERY node p (w = 0 outside the grid);
 *   Cibar[q] += dt*lam*ybar[q]*Lap(T)[q] at interior q.
 * Tbar is written at all nodes and must not overlap any input; Cibar is
 * read-modify-written (accumulated) at interior nodes only.
 * dtype PS_F64: all fields double.  PS_F32: all fields float.
 * ------------------------------------------------------------------- */
int ps_diffusion3d_adjoint(void *Tbar, void *Cibar, const void *ybar, const void *T,
                           const void *Ci, double lam, double dt, double _dx, double _dy,
                           double _dz, int64_t nx, int64_t ny, int64_t nz, int dtype,
                           void *stream);

/* As ps_diffusion3d_adjoint with flags.  PS_RUN_CI_SCALED (PS_F64, equal
 * spacings, else PS_ERR_UNSUPPORTED): `Ci` holds the pre-scaled field
 * Cs = dt*lam*_dx^2*Ci of ps_diffusion3d_scale_ci, the transpose of the step
 * T2 = T + Cs*L(T) with L(A) = (sum of the six neighbours) - 6 A:
 *   w[q] = Cs[q]*ybar[q] at interior q (0 elsewhere), Tbar = ybar + L(w)
 *   at every node, Cibar[q] += ybar[q]*L(T)[q] at interior q,
 * so Cibar accumulates dL/dCs; dL/dCi = dt*lam*_dx^2 * dL/dCs (e.g. by
 * ps_diffusion3d_scale_ci on the accumulated field).  lam, dt and the
 * spacings are then only checked.  No other flag is accepted. */
int ps_diffusion3d_adjoint_ex(void *Tbar, void *Cibar, const void *ybar, const void *T,
                              const void *Ci, double lam, double dt, double _dx, double _dy,
                              double _dz, int64_t nx, int64_t ny, int64_t nz, int dtype,
                              unsigned flags, void *stream);

/* Two transposed steps in one pass (temporal blocking of depth 2 of the
 * reverse sweep): with ybar = dL/dT_{t+2}, T_first = T_{t+1} and T_second =
 * T_t (the inputs of steps t+1 and t), Tbar := dL/dT_t and Cibar accumulates
 * both steps' terms - bit for bit two ps_diffusion3d_adjoint calls (the first
 * with T_first, the second with T_second on its output), without the
 * intermediate field leaving the chip.  PS_F32 only (PS_ERR_UNSUPPORTED for
 * PS_F64, whose step is bound by instruction issue, or when nx*4 is not a
 * multiple of 16); flags must be 0.  Same aliasing rules as the one-step call. */
int ps_diffusion3d_adjoint2_ex(void *Tbar, void *Cibar, const void *ybar, const void *T_first,
                               const void *T_second, const void *Ci, double lam, double dt, double _dx,
                               double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz, int dtype,
                               unsigned flags, void *stream);

/* ---------------------------------------------------------------------
 * Reductions in FP64 (deterministic: a fixed partition and a fixed
 * summation order, independent of timing).  A, B are device arrays of n
 * elements of `dtype`; out_dev is a device double; workspace is a device
 * buffer of ps_workspace_bytes().
 * ------------------------------------------------------------------- */
/* maximum(A) (Fig. 1's maximum(Ci)); result to a device double. */
int ps_maximum_async(double *out_dev, const void *A, int64_t n, int dtype, void *workspace,
                     void *stream);
/* maximum(A) returned to the host (synchronizes `stream`).  The finishing
 * kernel stores the result into a pinned, mapped host slot taken from a
 * pool for the duration of the call (allocating one when every slot is in
 * use; a failed allocation returns PS_ERR_CUDA), so the read-back uses no
 * copy engine and does not wait behind copies that other streams have in
 * flight. */
int ps_maximum(double *out_host, const void *A, int64_t n, int dtype, void *workspace,
               void *stream);
/* Fig. 1: dt = min(dx^2,dy^2,dz^2)/lam/maximum(Ci)/6.1 with dd = ld/(nd-1);
 * the maximum is reduced on the device, dt is formed on the host in FP64 and
 * returned in *dt_host (synchronizes `stream`). */
int ps_diffusion3d_stable_dt(double *dt_host, const void *Ci, int64_t nx, int64_t ny, int64_t nz,
                             double lam, double lx, double ly, double lz, int dtype,
                             void *workspace, void *stream);
/* sum_p A[p]*B[p], accumulated in FP64, to a device double. */
int ps_dot(double *out_dev, const void *A, const void *B, int64_t n, int dtype, void *workspace,
           void *stream);
/* sum_p A[p]*B[p] in FP64, like ps_dot, for callers that cannot allocate
 * device memory (for example a plugin inside a host application that owns
 * every device allocation, or a loop that must not allocate while it runs):
 * it takes no workspace and allocates nothing.  The paper has no counterpart;
 * this is a library convenience.  A and B need only be aligned to their
 * element size (8 bytes PS_F64, 4 bytes PS_F32), unlike the other calls.
 *   - Scratch: the per-block partial sums live in a 256 KiB array inside
 *     the library image, resident on every GPU that uses the library until
 *     the process exits.  n may be at most 134217728 (4096 elements per
 *     partial x 32768 partials); larger n returns PS_ERR_UNSUPPORTED and
 *     launches nothing.
 *   - The first call on a device looks up the array's device address once
 *     (again after cudaDeviceReset, which gives the device a new context);
 *     make that first call before any stream capture on the device.
 *   - Every call shares the one array (it keeps the last call's partials,
 *     each call overwrites what it reads): calls that can overlap on the GPU,
 *     e.g. on two streams, race and must be serialized by the caller.
 *   - Rounding: a contiguous-chunk partition, so results may differ from
 *     ps_dot's in the last bits; each call is deterministic. */
int ps_dot_static(double *out_dev, const void *A, const void *B, int64_t n, int dtype,
                  void *stream);

/* Loss of the inverse problem: 1/2 * sum_p (A[p]-B[p])^2 in FP64 to
 * *out_dev, and, if R is not NULL, the residual R = A - B (the cotangent
 * dL/dA) in `dtype`. */
int ps_half_sq_dist(double *out_dev, void *R, const void *A, const void *B, int64_t n, int dtype,
                    void *workspace, void *stream);

/* FP32 deviation storage: D[p] = (float)(T[p] - t_ref), with the
 * subtraction in FP64 and one rounding to float. */
int ps_to_deviation(float *D, const double *T, double t_ref, int64_t n, void *stream);
/* T[p] = (double)D[p] + t_ref in FP64. */
int ps_from_deviation(double *T, const float *D, double t_ref, int64_t n, void *stream);
/* Two-float deviation for the compensated step: v = T[p] - t_ref in FP64,
 * D[p] = (float)v, E[p] = (float)(v - D[p]) (D + E carries about 48 bits of v).
 * D, E and T must not overlap. */
int ps_to_deviation_pair(float *D, float *E, const double *T, double t_ref, int64_t n, void *stream);
/* T[p] = ((double)D[p] + (double)E[p]) + t_ref in FP64 (the value of a two-float
 * state). */
int ps_from_deviation_pair(double *T, const float *D, const float *E, double t_ref, int64_t n,
                           void *stream);

/* ---------------------------------------------------------------------
 * 2-D form of the step: Fig. 1's step! with the z term dropped (the
 * dimension argument of the initialization call set to 2):
 *   T2[inner] = T + dt*(lam*Ci*(d2x(T)*_dx^2 + d2y(T)*_dy^2))
 * on (ny, nx) fields, x fastest, boundary held fixed.  Same conventions as
 * ps_diffusion3d_step: device pointers, 16-byte aligned, T2 not overlapping
 * T or Ci, nx, ny >= 3, T2's boundary already equal to T's (run sets it).
 * Flags: PS_RUN_CI_SCALED (PS_F64, _dx == _dy: Ci holds dt*lam*_dx^2*Ci of
 * ps_diffusion3d_scale_ci over nx*ny values).  Kernel: a warp-level y-march
 * (16-byte accesses when nx*elem is a multiple of 16), the 3-D step's
 * per-node arithmetic with the z difference zero.
 * ------------------------------------------------------------------- */
int ps_diffusion2d_step(void *T2, const void *T, const void *Ci, double lam, double dt, double _dx,
                        double _dy, int64_t nx, int64_t ny, int dtype, unsigned flags, void *stream);
/* dt for the 2-D form, Fig. 1's rule with the two-axis bound:
 * dt = min(dx^2, dy^2)/lam/maximum(Ci)/4.1 with dx = lx/(nx-1), dy = ly/(ny-1);
 * maximum(Ci) over nx*ny values reduced on the device (workspace as for the
 * reductions below), dt formed on the host in FP64 to *dt_host (synchronizes
 * `stream`). */
int ps_diffusion2d_stable_dt(double *dt_host, const void *Ci, int64_t nx, int64_t ny, double lam,
                             double lx, double ly, int dtype, void *workspace, void *stream);
/* nt 2-D steps with T and T2 swapped after each (T2's edges first set to T's);
 * *result_in_T2 = nt & 1 (may be NULL).  Flags: PS_RUN_GRAPH (capture once per
 * argument set, replay), PS_RUN_CI_SCALED. */
int ps_diffusion2d_run(void *T, void *T2, const void *Ci, double lam, double dt, double _dx, double _dy,
                       int64_t nx, int64_t ny, int nt, int dtype, unsigned flags, void *stream,
                       int *result_in_T2);

/* ---------------------------------------------------------------------
 * Batched step: many independent problems of different sizes, one launch
 * per step (configs: many problems stepped together; Fig. 1's step per
 * problem).  The host describes each problem with a ps_problem; the
 * library lays them out in a table (problem records followed by a static
 * work list of (problem, x-y tile, z-chunk) items) that the caller copies
 * to device memory once.  A step processes every work item of the table;
 * `parity` 0 reads T and writes T2, parity 1 reads T2 and writes T (so
 * parity = step index & 1 reproduces the swap of Fig. 1's loop).
 *
 * Two kernels serve a table:
 *  - the column march (PS_BATCH_COLUMN): one thread per interior (i, j)
 *    column of a tile_x x tile_y x tile_z item, neighbours through the
 *    caches; any sizes and pitches;
 *  - the TMA z-march (PS_BATCH_ZMARCH): one CTA per item, the x-y tile of
 *    the single-grid step kernel (64 x 8 nodes FP64, 128 x 8 FP32, boundary
 *    included) and tile_z planes, staged by TMA, with the single-grid step's
 *    arithmetic (a problem's result equals its single run's bit for bit).
 *    Needs rows that start on 16-byte boundaries (pitch * element size a
 *    multiple of 16; see `pitch`), the CUDA driver's tensor-map encoder, and
 *    for FP64 equal spacings with dt*lam*_dx^2 > 0 (or PS_BATCH_CI_SCALED).
 *    tile_x and tile_y do not apply.
 * Flags 0 pick the z-march when every problem qualifies, else the column
 * march.  The z-march table embeds tensor maps of the fields: rebuild the
 * table when a field moves.
 * ------------------------------------------------------------------- */
typedef struct {
    void *T;          /* device field, nx*ny*nz of dtype, rows `pitch` apart */
    void *T2;         /* device field, same size and pitch, boundary equal to T's */
    const void *Ci;   /* device field, same size and pitch */
    double lam, dt, _dx, _dy, _dz;
    int64_t nx, ny, nz;
    int32_t tile_x, tile_y, tile_z; /* this problem's work-item shape; 0 = the call's */
    int32_t pitch;    /* elements from one row (fixed y, z) to the next, >= nx; planes are
                         pitch*ny apart; 0 = nx (contiguous fields) */
} ps_problem;

#define PS_BATCH_COLUMN 1u     /* the column march */
#define PS_BATCH_ZMARCH 2u     /* the TMA z-march; PS_ERR_UNSUPPORTED if a problem cannot take it */
#define PS_BATCH_CI_SCALED 4u  /* PS_F64, z-march, equal spacings: each Ci holds the pre-scaled
                                  dt*lam*_dx^2*Ci (see ps_diffusion3d_scale_ci); one FP64
                                  multiply-add per node */
#define PS_BATCH_TEMPORAL2 8u  /* z-march, PS_F32 or PS_F64 with PS_BATCH_CI_SCALED: the table
                                  also lists two-steps-per-pass items (temporal blocking of
                                  depth 2, the single-grid fused-pair kernel's tiles: 64 x 8
                                  FP64, 128 x 8 FP32, the problem's tile_z planes) for
                                  ps_diffusion3d_batch_run_ex with PS_RUN_TEMPORAL2 */

/* Bytes of the table for these problems, tile shape and flags (tile_x,
 * tile_y: interior nodes per column-march item in x and y, tile_x*tile_y
 * <= 4096; tile_z: planes per item; 0 picks the library default for the
 * dtype and kernel (z-march: 64 planes); a problem's own nonzero tile
 * fields override these).  0 when an
 * argument is invalid (ps_batch_table_fill_ex reports why). */
size_t ps_batch_table_bytes_ex(const ps_problem *probs, int nprob, int dtype, int tile_x, int tile_y,
                               int tile_z, unsigned flags);
/* Fill host_buf (bytes >= ps_batch_table_bytes_ex, 64-byte aligned) with the
 * table.  Checks every problem like ps_diffusion3d_step, over its pitch.
 * *nitems_out = work items. */
int ps_batch_table_fill_ex(void *host_buf, size_t bytes, const ps_problem *probs, int nprob,
                           int dtype, int tile_x, int tile_y, int tile_z, unsigned flags,
                           int64_t *nitems_out);
/* Kernel of a filled table: 0 column march, 1 z-march. */
int ps_batch_table_kernel(const void *host_table);
/* One step of every problem in the device table (dev_table = device copy
 * of the filled host buffer host_table, which the call reads on the host). */
int ps_diffusion3d_batch_step_ex(const void *dev_table, const void *host_table, int parity,
                                 void *stream);
/* Two steps of every problem in one launch (a table built with
 * PS_BATCH_TEMPORAL2): parity 0 reads T and writes T2, 1 the reverse.  Bit
 * for bit two ps_diffusion3d_batch_step_ex calls, in one pass over HBM. */
int ps_diffusion3d_batch_step2_ex(const void *dev_table, const void *host_table, int parity,
                                  void *stream);
/* nt batched steps (the buffers of problem p hold its final state in T2 when
 * nt is odd, in T when even).  Flags: PS_RUN_GRAPH captures the launches once
 * per (table address, item count, kernel, nt, dtype, pairs) and replays them;
 * PS_RUN_TEMPORAL2 (a table built with PS_BATCH_TEMPORAL2) runs the steps as
 * fused pairs, each launch swapping the buffers - where the pair count would
 * leave the result in the other buffer, one pair runs as two single steps. */
int ps_diffusion3d_batch_run_ex(const void *dev_table, const void *host_table, int nt,
                                unsigned flags, void *stream);

/* Column-march forms: the _ex calls with flags PS_BATCH_COLUMN; step and run
 * take only a column-march table (a z-march table makes them set bit 1 of
 * ps_device_error and leave the fields unchanged). */
size_t ps_batch_table_bytes(const ps_problem *probs, int nprob, int dtype, int tile_x, int tile_y,
                            int tile_z);
int ps_batch_table_fill(void *host_buf, size_t bytes, const ps_problem *probs, int nprob,
                        int dtype, int tile_x, int tile_y, int tile_z, int64_t *nitems_out);
int ps_diffusion3d_batch_step(const void *dev_table, int parity, int dtype, void *stream);
int ps_diffusion3d_batch_run(const void *dev_table, int nt, int dtype, unsigned flags,
                             void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PS_DIFFUSION3D_H */

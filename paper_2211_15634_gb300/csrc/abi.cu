// C ABI of the library: host-side argument checks, dispatch to the kernels,
// the CUDA-graph cache of ps_diffusion3d_run_ex and the batch-table builder.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "emu64.cuh"
#include "internal.h"

namespace psd {

static thread_local std::string g_err;

static int fail(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return status;
}

static int cuda_fail(cudaError_t e, const char *where) {
    return fail(PS_ERR_CUDA, "%s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
}

int api_fail(int status, const char *msg) { return fail(status, "%s", msg); }
int api_cuda_fail(cudaError_t e, const char *where) { return cuda_fail(e, where); }

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

int sm_count() {
    static int cache[64] = {0};
    const int d = current_device();
    if (d < 0 || d >= 64) return 148;
    if (cache[d] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0)
            v = 148;
        cache[d] = v;
    }
    return cache[d];
}

static int elem_bytes(int dtype) { return dtype == PS_F64 ? 8 : 4; }

static int check_dtype(int dtype) {
    if (dtype != PS_F32 && dtype != PS_F64) return fail(PS_ERR_ARG, "dtype %d is not PS_F32/PS_F64", dtype);
    return PS_OK;
}

static int check_grid(int64_t nx, int64_t ny, int64_t nz) {
    if (nx < 3 || ny < 3 || nz < 3)
        return fail(PS_ERR_ARG, "grid %lld x %lld x %lld: every size must be >= 3", (long long)nx,
                    (long long)ny, (long long)nz);
    if (nx > (1LL << 31) || ny > (1LL << 31) || nz > (1LL << 31) ||
        (double)nx * (double)ny * (double)nz > 9.0e15)
        return fail(PS_ERR_ARG, "grid %lld x %lld x %lld is too large", (long long)nx, (long long)ny,
                    (long long)nz);
    return PS_OK;
}

static int check_ptr(const void *p, const char *name) {
    if (!p) return fail(PS_ERR_ARG, "%s is NULL", name);
    if (((uintptr_t)p) & 15u) return fail(PS_ERR_ALIGN, "%s = %p is not 16-byte aligned", name, p);
    return PS_OK;
}

static bool overlap2(const void *a, size_t abytes, const void *b, size_t bbytes) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bbytes && y < x + abytes;
}

static bool overlap(const void *a, const void *b, size_t bytes) { return overlap2(a, bytes, b, bytes); }

static int check_finite(double v, const char *name) {
    if (!std::isfinite(v)) return fail(PS_ERR_ARG, "%s is not finite", name);
    return PS_OK;
}

#define PS_TRY(x)                    \
    do {                             \
        int _st = (x);               \
        if (_st != PS_OK) return _st; \
    } while (0)

static int check_step_args(const void *T2, const void *T, const void *Ci, double lam, double dt,
                           double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz,
                           int dtype) {
    PS_TRY(check_dtype(dtype));
    PS_TRY(check_grid(nx, ny, nz));
    PS_TRY(check_ptr(T2, "T2"));
    PS_TRY(check_ptr(T, "T"));
    PS_TRY(check_ptr(Ci, "Ci"));
    PS_TRY(check_finite(lam, "lam"));
    PS_TRY(check_finite(dt, "dt"));
    PS_TRY(check_finite(_dx, "_dx"));
    PS_TRY(check_finite(_dy, "_dy"));
    PS_TRY(check_finite(_dz, "_dz"));
    const size_t bytes = (size_t)(nx * ny * nz) * elem_bytes(dtype);
    if (overlap(T2, T, bytes)) return fail(PS_ERR_ALIAS, "T2 overlaps T");
    if (overlap(T2, Ci, bytes)) return fail(PS_ERR_ALIAS, "T2 overlaps Ci");
    return PS_OK;
}

static cudaError_t enqueue_step(void *T2, const void *T, void *comp, const void *Ci, StepCoef c,
                                Grid3 g, int dtype, unsigned flags, cudaStream_t s) {
    if (dtype == PS_F64) {
        if (flags & PS_RUN_CI_SCALED)
            return launch_step_f64_scaled((double *)T2, (const double *)T, (const double *)Ci, g, s);
        if (flags & PS_RUN_NATIVE_F64)
            return launch_step_f64_native((double *)T2, (const double *)T, (const double *)Ci, c, g, s);
        return launch_step_f64_fast((double *)T2, (const double *)T, (const double *)Ci, c, g, s);
    }
    if (flags & PS_RUN_COMPENSATED)
        return launch_step_f32_comp((float *)T2, (const float *)T, (float *)comp, (const float *)Ci,
                                    c, g, s);
    return launch_step_f32((float *)T2, (const float *)T, (const float *)Ci, c, g, s);
}

// True when PS_RUN_TEMPORAL2 can fuse step pairs for these arguments (the mode
// is checked by the caller: FP32 plain, or FP64 on the pre-scaled coefficient).
static bool temporal2_ok(Grid3 g, int dtype, const void *T, const void *T2, const void *Ci) {
    return zmarch2_supported(g, elem_bytes(dtype), T, T2, Ci) &&
           zmarch2_supported(g, elem_bytes(dtype), T2, T, Ci);
}

static cudaError_t enqueue_step2(void *T2, const void *T, const void *Ci, StepCoef c, Grid3 g,
                                 int dtype, cudaStream_t s) {
    if (dtype == PS_F64) return launch_step2_f64_scaled((double *)T2, (const double *)T, (const double *)Ci, g, s);
    return launch_step2_f32((float *)T2, (const float *)T, (const float *)Ci, c, g, s);
}

// Boundary copy followed by nt steps with alternating buffers.  With
// PS_RUN_TEMPORAL2 the steps go in fused pairs; when the number of passes would
// leave the result in the other buffer than nt's parity says, one pair is run
// as two single steps.
static cudaError_t enqueue_run(void *T, void *T2, void *comp, const void *Ci, StepCoef c, Grid3 g,
                               int nt, int dtype, unsigned flags, cudaStream_t s) {
    cudaError_t e = launch_copy_boundary(T2, T, g, elem_bytes(dtype), s);
    int pairs = 0, singles = nt;
    if ((flags & PS_RUN_TEMPORAL2) && temporal2_ok(g, dtype, T, T2, Ci)) {
        pairs = nt / 2;
        singles = nt & 1;
        if (((pairs + singles) & 1) != (nt & 1)) {
            pairs -= 1;
            singles += 2;
        }
    }
    for (int it = 0; it < pairs + singles && e == cudaSuccess; ++it) {
        void *src = (it & 1) ? T2 : T;
        void *dst = (it & 1) ? T : T2;
        e = it < pairs ? enqueue_step2(dst, src, Ci, c, g, dtype, s)
                       : enqueue_step(dst, src, comp, Ci, c, g, dtype, flags, s);
    }
    return e;
}

// ---------------------------------------------------------------- graphs
using GraphKey = std::tuple<int, const void *, const void *, const void *, const void *, double,
                            double, double, double, double, int64_t, int64_t, int64_t, int, int,
                            unsigned>;
static std::mutex g_graph_mu;
static std::map<GraphKey, cudaGraphExec_t> g_graphs;
static cudaStream_t g_capture_stream[64] = {nullptr};

static cudaError_t capture_stream(cudaStream_t *out) {
    const int d = current_device();
    if (d < 0 || d >= 64) return cudaErrorInvalidDevice;
    if (!g_capture_stream[d]) {
        cudaError_t e = cudaStreamCreateWithFlags(&g_capture_stream[d], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    *out = g_capture_stream[d];
    return cudaSuccess;
}

static int run_graph(void *T, void *T2, void *comp, const void *Ci, double lam, double dt,
                     double _dx, double _dy, double _dz, Grid3 g, int nt, int dtype,
                     unsigned flags, cudaStream_t s) {
    const GraphKey key{current_device(), T, T2, comp, Ci, lam, dt, _dx, _dy, _dz, g.nx, g.ny, g.nz,
                       nt, dtype, flags & ~PS_RUN_GRAPH};
    std::lock_guard<std::mutex> lock(g_graph_mu);
    auto it = g_graphs.find(key);
    if (it == g_graphs.end()) {
        cudaStream_t cs;
        cudaError_t e = capture_stream(&cs);
        if (e != cudaSuccess) return cuda_fail(e, "capture stream");
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        cudaError_t le = enqueue_run(T, T2, comp, Ci, make_coef(lam, dt, _dx, _dy, _dz), g, nt, dtype,
                                     flags, cs);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(le, "capturing the time loop");
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        it = g_graphs.emplace(key, exec).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return PS_OK;
}

}  // namespace psd

using namespace psd;

extern "C" {

int ps_version(void) { return 100; }

const char *ps_last_error(void) { return g_err.c_str(); }

int ps_device_error(unsigned *out_host, int clear) {
    if (!out_host) return fail(PS_ERR_ARG, "out_host is NULL");
    *out_host = zmarch_device_error(clear != 0) | adjoint_device_error(clear != 0) |
                adjoint_scaled_device_error(clear != 0) | zmarch2_device_error(clear != 0) |
                adjoint_f32_device_error(clear != 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ps_device_error");
    return PS_OK;
}

int ps_selftest_bounded_wait(unsigned polls, unsigned suspend_ns, void *stream) {
    if (polls < 1 || polls > (1u << 24)) return fail(PS_ERR_ARG, "polls = %u not in [1, 2^24]", polls);
    if (suspend_ns < 1 || suspend_ns > 1000000u)
        return fail(PS_ERR_ARG, "suspend_ns = %u not in [1, 10^6]", suspend_ns);
    cudaError_t e = launch_selftest_wait(polls, suspend_ns, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_selftest_bounded_wait");
    return PS_OK;
}

const char *ps_diffusion3d_step_kernel(const void *T2, const void *T, const void *Ci, double lam,
                                       double dt, double _dx, double _dy, double _dz, int64_t nx,
                                       int64_t ny, int64_t nz, int dtype, unsigned flags) {
    const Grid3 g{nx, ny, nz};
    if ((flags & PS_RUN_TEMPORAL2) && temporal2_ok(g, dtype, T, T2, Ci)) {
        if (dtype == PS_F32 && !(flags & PS_RUN_COMPENSATED)) return "k_zmarch2<F32>";
        if (dtype == PS_F64 && (flags & PS_RUN_CI_SCALED)) return "k_zmarch2<F64_SCALED>";
    }
    if (dtype == PS_F64)
        return step_f64_kernel_name(g, T2, T, Ci, make_coef(lam, dt, _dx, _dy, _dz),
                                    (flags & PS_RUN_CI_SCALED) != 0);
    return step_f32_kernel_name(g, T2, T, Ci);
}

size_t ps_workspace_bytes(void) { return kWorkspaceBytes; }

static int check_scaled(unsigned flags, int dtype, double _dx, double _dy, double _dz) {
    if (!(flags & PS_RUN_CI_SCALED)) return PS_OK;
    if (dtype != PS_F64) return fail(PS_ERR_UNSUPPORTED, "a pre-scaled Ci needs PS_F64");
    if (!(_dx == _dy && _dy == _dz))
        return fail(PS_ERR_UNSUPPORTED, "a pre-scaled Ci needs equal spacings (_dx == _dy == _dz)");
    return PS_OK;
}

int ps_diffusion3d_step(void *T2, const void *T, const void *Ci, double lam, double dt, double _dx,
                        double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz, int dtype,
                        void *stream) {
    PS_TRY(check_step_args(T2, T, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz, dtype));
    cudaError_t e = enqueue_step(T2, T, nullptr, Ci, make_coef(lam, dt, _dx, _dy, _dz),
                                 Grid3{nx, ny, nz}, dtype, 0u, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_step");
    return PS_OK;
}

int ps_diffusion3d_step_ex(void *T2, const void *T, const void *Ci, double lam, double dt,
                           double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz,
                           int dtype, unsigned flags, void *stream) {
    PS_TRY(check_step_args(T2, T, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz, dtype));
    if (flags & ~(PS_RUN_CI_SCALED | PS_RUN_NATIVE_F64)) return fail(PS_ERR_ARG, "unknown flags 0x%x", flags);
    PS_TRY(check_scaled(flags, dtype, _dx, _dy, _dz));
    if ((flags & PS_RUN_NATIVE_F64) && dtype != PS_F64)
        return fail(PS_ERR_UNSUPPORTED, "PS_RUN_NATIVE_F64 needs PS_F64");
    cudaError_t e = enqueue_step(T2, T, nullptr, Ci, make_coef(lam, dt, _dx, _dy, _dz),
                                 Grid3{nx, ny, nz}, dtype, flags, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_step_ex");
    return PS_OK;
}

int ps_diffusion3d_scale_ci(double *Cs, const double *Ci, double lam, double dt, double _dx,
                            int64_t n, void *stream) {
    if (n < 1) return fail(PS_ERR_ARG, "n = %lld < 1", (long long)n);
    PS_TRY(check_ptr(Cs, "Cs"));
    PS_TRY(check_ptr(Ci, "Ci"));
    PS_TRY(check_finite(lam, "lam"));
    PS_TRY(check_finite(dt, "dt"));
    PS_TRY(check_finite(_dx, "_dx"));
    if (Cs != Ci && overlap(Cs, Ci, (size_t)n * 8)) return fail(PS_ERR_ALIAS, "Cs partly overlaps Ci");
    cudaError_t e = launch_scale_ci(Cs, Ci, dt * lam * (_dx * _dx), n, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_scale_ci");
    return PS_OK;
}

int ps_diffusion3d_step_comp_f32(float *T2, const float *T, float *comp, const float *Ci,
                                 double lam, double dt, double _dx, double _dy, double _dz,
                                 int64_t nx, int64_t ny, int64_t nz, void *stream) {
    PS_TRY(check_step_args(T2, T, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz, PS_F32));
    PS_TRY(check_ptr(comp, "comp"));
    const size_t bytes = (size_t)(nx * ny * nz) * 4;
    if (overlap(comp, T, bytes) || overlap(comp, T2, bytes) || overlap(comp, Ci, bytes))
        return fail(PS_ERR_ALIAS, "comp overlaps T, T2 or Ci");
    cudaError_t e = launch_step_f32_comp(T2, T, comp, Ci, make_coef(lam, dt, _dx, _dy, _dz),
                                         Grid3{nx, ny, nz}, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_step_comp_f32");
    return PS_OK;
}

int ps_diffusion3d_copy_boundary(void *T2, const void *T, int64_t nx, int64_t ny, int64_t nz,
                                 int dtype, void *stream) {
    PS_TRY(check_dtype(dtype));
    PS_TRY(check_grid(nx, ny, nz));
    PS_TRY(check_ptr(T2, "T2"));
    PS_TRY(check_ptr(T, "T"));
    if (overlap(T2, T, (size_t)(nx * ny * nz) * elem_bytes(dtype))) return fail(PS_ERR_ALIAS, "T2 overlaps T");
    cudaError_t e = launch_copy_boundary(T2, T, Grid3{nx, ny, nz}, elem_bytes(dtype), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_copy_boundary");
    return PS_OK;
}

int ps_diffusion3d_copy_boundary_many(void *dst, int64_t count, int64_t grid_stride,
                                      const void *T, int64_t nx, int64_t ny, int64_t nz, int dtype,
                                      void *stream) {
    PS_TRY(check_dtype(dtype));
    PS_TRY(check_grid(nx, ny, nz));
    PS_TRY(check_ptr(dst, "dst"));
    PS_TRY(check_ptr(T, "T"));
    if (count < 1) return fail(PS_ERR_ARG, "count = %lld < 1", (long long)count);
    const int64_t n = nx * ny * nz;
    if (grid_stride < n || (grid_stride * elem_bytes(dtype)) % 16 != 0)
        return fail(PS_ERR_ARG, "grid_stride = %lld: need >= nx*ny*nz and a multiple of 16 bytes",
                    (long long)grid_stride);
    const size_t gbytes = (size_t)grid_stride * elem_bytes(dtype);
    if ((const char *)T < (const char *)dst + gbytes * (size_t)count &&
        (const char *)dst < (const char *)T + (size_t)n * elem_bytes(dtype))
        return fail(PS_ERR_ALIAS, "T overlaps the destination grids");
    cudaError_t e = launch_copy_boundary_many(dst, count, grid_stride, T, Grid3{nx, ny, nz},
                                              elem_bytes(dtype), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_copy_boundary_many");
    return PS_OK;
}

int ps_diffusion3d_run_states(const void *T0, void *states, int64_t grid_stride, int every,
                              const void *Ci, double lam, double dt, double _dx, double _dy,
                              double _dz, int64_t nx, int64_t ny, int64_t nz, int nt, int dtype,
                              unsigned flags, void *stream, int *final_slot) {
    PS_TRY(check_step_args(states, T0, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz, dtype));
    if (nt < 0) return fail(PS_ERR_ARG, "nt = %d < 0", nt);
    if (every < 1) return fail(PS_ERR_ARG, "every = %d < 1", every);
    if (!final_slot) return fail(PS_ERR_ARG, "final_slot is NULL");
    if (flags & ~(PS_RUN_CI_SCALED | PS_RUN_NATIVE_F64)) return fail(PS_ERR_ARG, "unknown flags 0x%x", flags);
    PS_TRY(check_scaled(flags, dtype, _dx, _dy, _dz));
    if ((flags & PS_RUN_NATIVE_F64) && dtype != PS_F64)
        return fail(PS_ERR_UNSUPPORTED, "PS_RUN_NATIVE_F64 needs PS_F64");
    const int64_t n = nx * ny * nz;
    const size_t esz = elem_bytes(dtype);
    if (grid_stride < n || (grid_stride * (int64_t)esz) % 16 != 0)
        return fail(PS_ERR_ARG, "grid_stride = %lld: need >= nx*ny*nz and a multiple of 16 bytes",
                    (long long)grid_stride);
    const int nslots = nt / every, nwork = (every > 1 && nt > 0) ? 2 : 0;
    const size_t span = (size_t)grid_stride * esz * (size_t)(nslots + nwork);
    if (span && (overlap2(states, span, T0, (size_t)n * esz) || overlap2(states, span, Ci, (size_t)n * esz)))
        return fail(PS_ERR_ALIAS, "the state grids overlap T0 or Ci");
    char *base = (char *)states;
    auto grid = [&](int slot) { return (void *)(base + (size_t)slot * (size_t)grid_stride * esz); };
    const StepCoef c = make_coef(lam, dt, _dx, _dy, _dz);
    const Grid3 g{nx, ny, nz};
    const void *cur = T0;
    int cur_slot = -3, work_next = 0;  // -3: T0; -1, -2: work grids 0, 1
    for (int t = 1; t <= nt; ++t) {
        int slot;
        void *dst;
        if (t % every == 0) {
            slot = t / every - 1;
            dst = grid(slot);
        } else {  // a work grid, never the one this step reads
            if (cur_slot == -1 - work_next) work_next ^= 1;
            slot = -1 - work_next;
            dst = grid(nslots + work_next);
            work_next ^= 1;
        }
        cudaError_t e = enqueue_step(dst, cur, nullptr, Ci, c, g, dtype, flags, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_run_states");
        cur = dst;
        cur_slot = slot;
    }
    *final_slot = cur_slot;
    return PS_OK;
}

int ps_diffusion3d_run_ex(void *T, void *T2, void *comp, const void *Ci, double lam, double dt,
                          double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz,
                          int nt, int dtype, unsigned flags, void *stream, int *result_in_T2) {
    PS_TRY(check_step_args(T2, T, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz, dtype));
    if (nt < 0) return fail(PS_ERR_ARG, "nt = %d < 0", nt);
    if (flags & ~(PS_RUN_GRAPH | PS_RUN_COMPENSATED | PS_RUN_NATIVE_F64 | PS_RUN_CI_SCALED |
                  PS_RUN_TEMPORAL2))
        return fail(PS_ERR_ARG, "unknown flags 0x%x", flags);
    PS_TRY(check_scaled(flags, dtype, _dx, _dy, _dz));
    if ((flags & PS_RUN_TEMPORAL2) &&
        !(dtype == PS_F32 ? !(flags & PS_RUN_COMPENSATED) : (flags & PS_RUN_CI_SCALED) != 0))
        return fail(PS_ERR_UNSUPPORTED,
                    "PS_RUN_TEMPORAL2 needs PS_F32 (not compensated) or PS_F64 with PS_RUN_CI_SCALED");
    if (flags & PS_RUN_COMPENSATED) {
        if (dtype != PS_F32) return fail(PS_ERR_UNSUPPORTED, "PS_RUN_COMPENSATED needs PS_F32");
        PS_TRY(check_ptr(comp, "comp"));
        const size_t bytes = (size_t)(nx * ny * nz) * 4;
        if (overlap(comp, T, bytes) || overlap(comp, T2, bytes) || overlap(comp, Ci, bytes))
            return fail(PS_ERR_ALIAS, "comp overlaps T, T2 or Ci");
    } else {
        comp = nullptr;
    }
    if ((flags & PS_RUN_NATIVE_F64) && dtype != PS_F64)
        return fail(PS_ERR_UNSUPPORTED, "PS_RUN_NATIVE_F64 needs PS_F64");
    const Grid3 g{nx, ny, nz};
    if (result_in_T2) *result_in_T2 = nt & 1;
    if (flags & PS_RUN_GRAPH)
        return run_graph(T, T2, comp, Ci, lam, dt, _dx, _dy, _dz, g, nt, dtype, flags,
                         (cudaStream_t)stream);
    cudaError_t e = enqueue_run(T, T2, comp, Ci, make_coef(lam, dt, _dx, _dy, _dz), g, nt, dtype,
                                flags, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_run");
    return PS_OK;
}

int ps_diffusion3d_run(void *T, void *T2, const void *Ci, double lam, double dt, double _dx,
                       double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz, int nt, int dtype,
                       void *stream, int *result_in_T2) {
    return ps_diffusion3d_run_ex(T, T2, nullptr, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz, nt, dtype,
                                 0u, stream, result_in_T2);
}

int ps_clear_graph_cache(void) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (auto &kv : g_graphs) cudaGraphExecDestroy(kv.second);
    g_graphs.clear();
    return PS_OK;
}

int ps_diffusion3d_adjoint(void *Tbar, void *Cibar, const void *ybar, const void *T,
                           const void *Ci, double lam, double dt, double _dx, double _dy,
                           double _dz, int64_t nx, int64_t ny, int64_t nz, int dtype,
                           void *stream) {
    return ps_diffusion3d_adjoint_ex(Tbar, Cibar, ybar, T, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz,
                                     dtype, 0u, stream);
}

int ps_diffusion3d_adjoint_ex(void *Tbar, void *Cibar, const void *ybar, const void *T,
                              const void *Ci, double lam, double dt, double _dx, double _dy,
                              double _dz, int64_t nx, int64_t ny, int64_t nz, int dtype,
                              unsigned flags, void *stream) {
    if (flags & ~PS_RUN_CI_SCALED) return fail(PS_ERR_ARG, "unknown flags 0x%x", flags);
    PS_TRY(check_dtype(dtype));
    PS_TRY(check_grid(nx, ny, nz));
    PS_TRY(check_ptr(Tbar, "Tbar"));
    PS_TRY(check_ptr(Cibar, "Cibar"));
    PS_TRY(check_ptr(ybar, "ybar"));
    PS_TRY(check_ptr(T, "T"));
    PS_TRY(check_ptr(Ci, "Ci"));
    PS_TRY(check_finite(lam, "lam"));
    PS_TRY(check_finite(dt, "dt"));
    PS_TRY(check_finite(_dx, "_dx"));
    PS_TRY(check_finite(_dy, "_dy"));
    PS_TRY(check_finite(_dz, "_dz"));
    const size_t bytes = (size_t)(nx * ny * nz) * elem_bytes(dtype);
    if (overlap(Tbar, ybar, bytes) || overlap(Tbar, T, bytes) || overlap(Tbar, Ci, bytes) ||
        overlap(Tbar, Cibar, bytes))
        return fail(PS_ERR_ALIAS, "Tbar overlaps an input");
    if (overlap(Cibar, ybar, bytes) || overlap(Cibar, T, bytes) || overlap(Cibar, Ci, bytes))
        return fail(PS_ERR_ALIAS, "Cibar overlaps an input");
    PS_TRY(check_scaled(flags, dtype, _dx, _dy, _dz));
    const StepCoef c = make_coef(lam, dt, _dx, _dy, _dz);
    const Grid3 g{nx, ny, nz};
    cudaError_t e;
    if (flags & PS_RUN_CI_SCALED)
        e = launch_adjoint_f64_scaled((double *)Tbar, (double *)Cibar, (const double *)ybar,
                                      (const double *)T, (const double *)Ci, g, (cudaStream_t)stream);
    else if (dtype == PS_F64)
        e = launch_adjoint_f64((double *)Tbar, (double *)Cibar, (const double *)ybar,
                               (const double *)T, (const double *)Ci, c, g, (cudaStream_t)stream);
    else
        e = launch_adjoint_f32((float *)Tbar, (float *)Cibar, (const float *)ybar, (const float *)T,
                               (const float *)Ci, c, g, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_adjoint");
    return PS_OK;
}

static int check_reduce(const void *A, int64_t n, int dtype, const void *ws) {
    PS_TRY(check_dtype(dtype));
    if (n < 1) return fail(PS_ERR_ARG, "n = %lld < 1", (long long)n);
    PS_TRY(check_ptr(A, "A"));
    PS_TRY(check_ptr(ws, "workspace"));
    return PS_OK;
}

int ps_maximum_async(double *out_dev, const void *A, int64_t n, int dtype, void *workspace,
                     void *stream) {
    PS_TRY(check_reduce(A, n, dtype, workspace));
    if (!out_dev) return fail(PS_ERR_ARG, "out_dev is NULL");
    cudaError_t e = launch_maximum(out_dev, A, n, dtype, workspace, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_maximum");
    return PS_OK;
}

int ps_maximum(double *out_host, const void *A, int64_t n, int dtype, void *workspace,
               void *stream) {
    if (!out_host) return fail(PS_ERR_ARG, "out_host is NULL");
    PS_TRY(check_reduce(A, n, dtype, workspace));
    double *slot = (double *)((char *)workspace + 8);  // scratch slot inside the workspace
    cudaError_t e = launch_maximum(slot, A, n, dtype, workspace, (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, slot, sizeof(double), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_maximum");
    return PS_OK;
}

int ps_diffusion3d_stable_dt(double *dt_host, const void *Ci, int64_t nx, int64_t ny, int64_t nz,
                             double lam, double lx, double ly, double lz, int dtype,
                             void *workspace, void *stream) {
    if (!dt_host) return fail(PS_ERR_ARG, "dt_host is NULL");
    PS_TRY(check_grid(nx, ny, nz));
    PS_TRY(check_finite(lam, "lam"));
    double mx = 0.0;
    PS_TRY(ps_maximum(&mx, Ci, nx * ny * nz, dtype, workspace, stream));
    const double dx = lx / (double)(nx - 1), dy = ly / (double)(ny - 1), dz = lz / (double)(nz - 1);
    double m = dx * dx;
    if (dy * dy < m) m = dy * dy;
    if (dz * dz < m) m = dz * dz;
    *dt_host = m / lam / mx / 6.1;
    return PS_OK;
}

int ps_dot(double *out_dev, const void *A, const void *B, int64_t n, int dtype, void *workspace,
           void *stream) {
    PS_TRY(check_reduce(A, n, dtype, workspace));
    PS_TRY(check_ptr(B, "B"));
    if (!out_dev) return fail(PS_ERR_ARG, "out_dev is NULL");
    cudaError_t e = launch_dot(out_dev, A, B, n, dtype, workspace, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_dot");
    return PS_OK;
}

int ps_half_sq_dist(double *out_dev, void *R, const void *A, const void *B, int64_t n, int dtype,
                    void *workspace, void *stream) {
    PS_TRY(check_reduce(A, n, dtype, workspace));
    PS_TRY(check_ptr(B, "B"));
    if (!out_dev) return fail(PS_ERR_ARG, "out_dev is NULL");
    if (R) {
        PS_TRY(check_ptr(R, "R"));
        const size_t bytes = (size_t)n * elem_bytes(dtype);
        if (overlap(R, A, bytes) || overlap(R, B, bytes)) return fail(PS_ERR_ALIAS, "R overlaps A or B");
    }
    cudaError_t e = launch_half_sq_dist(out_dev, R, A, B, n, dtype, workspace, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_half_sq_dist");
    return PS_OK;
}

int ps_to_deviation(float *D, const double *T, double t_ref, int64_t n, void *stream) {
    if (n < 1) return fail(PS_ERR_ARG, "n = %lld < 1", (long long)n);
    PS_TRY(check_ptr(D, "D"));
    PS_TRY(check_ptr(T, "T"));
    PS_TRY(check_finite(t_ref, "t_ref"));
    if (overlap2(D, (size_t)n * 4, T, (size_t)n * 8)) return fail(PS_ERR_ALIAS, "D overlaps T");
    cudaError_t e = launch_to_deviation(D, T, t_ref, n, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_to_deviation");
    return PS_OK;
}

int ps_from_deviation(double *T, const float *D, double t_ref, int64_t n, void *stream) {
    if (n < 1) return fail(PS_ERR_ARG, "n = %lld < 1", (long long)n);
    PS_TRY(check_ptr(D, "D"));
    PS_TRY(check_ptr(T, "T"));
    PS_TRY(check_finite(t_ref, "t_ref"));
    if (overlap2(D, (size_t)n * 4, T, (size_t)n * 8)) return fail(PS_ERR_ALIAS, "T overlaps D");
    cudaError_t e = launch_from_deviation(T, D, t_ref, n, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_from_deviation");
    return PS_OK;
}

// ------------------------------------------------------------------ batch
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static int resolve_tiles(int dtype, int *tx, int *ty, int *tz) {
    int dx, dy, dz;
    batch_default_tile(dtype, &dx, &dy, &dz);
    if (*tx == 0) *tx = dx;
    if (*ty == 0) *ty = dy;
    if (*tz == 0) *tz = dz;
    if (*tx < 1 || *ty < 1 || *tz < 1 || (int64_t)*tx * *ty > 4096 || *tx > 4096 || *ty > 4096 ||
        *tz > 32767)
        return fail(PS_ERR_ARG, "tile %d x %d x %d is invalid (x*y <= 4096, z <= 32767)", *tx, *ty, *tz);
    return PS_OK;
}

// A problem's own tile fields override the call's.
static int problem_tiles(const ps_problem &p, int dtype, int tx, int ty, int tz, int *ox, int *oy,
                         int *oz) {
    *ox = p.tile_x ? p.tile_x : tx;
    *oy = p.tile_y ? p.tile_y : ty;
    *oz = p.tile_z ? p.tile_z : tz;
    return resolve_tiles(dtype, ox, oy, oz);
}

static int64_t items_of(const ps_problem &p, int tx, int ty, int tz) {
    return ((p.nx - 2 + tx - 1) / tx) * ((p.ny - 2 + ty - 1) / ty) * ((p.nz - 2 + tz - 1) / tz);
}

static size_t table_bytes(int nprob, int64_t nitems) {
    return align_up(sizeof(BatchHeader), 64) + align_up(sizeof(BatchProblem) * (size_t)nprob, 64) +
           sizeof(BatchItem) * (size_t)nitems;
}

size_t ps_batch_table_bytes(const ps_problem *probs, int nprob, int dtype, int tile_x, int tile_y,
                            int tile_z) {
    if (!probs || nprob < 1 || check_dtype(dtype) != PS_OK) return 0;
    if (resolve_tiles(dtype, &tile_x, &tile_y, &tile_z) != PS_OK) return 0;
    int64_t nitems = 0;
    for (int q = 0; q < nprob; ++q) {
        int tx, ty, tz;
        if (probs[q].nx < 3 || probs[q].ny < 3 || probs[q].nz < 3) return 0;
        if (problem_tiles(probs[q], dtype, tile_x, tile_y, tile_z, &tx, &ty, &tz) != PS_OK) return 0;
        nitems += items_of(probs[q], tx, ty, tz);
    }
    return table_bytes(nprob, nitems);
}

int ps_batch_table_fill(void *host_buf, size_t bytes, const ps_problem *probs, int nprob, int dtype,
                        int tile_x, int tile_y, int tile_z, int64_t *nitems_out) {
    if (!host_buf || !probs) return fail(PS_ERR_ARG, "host_buf or probs is NULL");
    if (nprob < 1) return fail(PS_ERR_ARG, "nprob = %d < 1", nprob);
    PS_TRY(check_dtype(dtype));
    PS_TRY(resolve_tiles(dtype, &tile_x, &tile_y, &tile_z));
    int64_t nitems = 0;
    for (int q = 0; q < nprob; ++q) {
        const ps_problem &p = probs[q];
        int st = check_step_args(p.T2, p.T, p.Ci, p.lam, p.dt, p._dx, p._dy, p._dz, p.nx, p.ny, p.nz, dtype);
        if (st != PS_OK) return fail(st, "problem %d: %s", q, g_err.c_str());
        int tx, ty, tz;
        st = problem_tiles(p, dtype, tile_x, tile_y, tile_z, &tx, &ty, &tz);
        if (st != PS_OK) return fail(st, "problem %d: %s", q, g_err.c_str());
        if (p.nx * p.ny * p.nz >= (1LL << 31) || p.nx + tx > (1LL << 31) || p.ny + ty > (1LL << 31) ||
            p.nz + tz > (1LL << 31))
            return fail(PS_ERR_ARG, "problem %d is too large for the batch table (2^31 nodes at most)", q);
        nitems += items_of(p, tx, ty, tz);
    }
    const size_t need = table_bytes(nprob, nitems);
    if (bytes < need) return fail(PS_ERR_ARG, "table buffer has %zu bytes, needs %zu", bytes, need);
    std::memset(host_buf, 0, need);
    char *base = (char *)host_buf;
    BatchHeader *h = (BatchHeader *)base;
    h->nprob = nprob;
    h->nitems = nitems;
    h->dtype = dtype;
    h->tile_x = tile_x;
    h->tile_y = tile_y;
    h->tile_z = tile_z;
    h->problems_offset = (int64_t)align_up(sizeof(BatchHeader), 64);
    h->items_offset = h->problems_offset + (int64_t)align_up(sizeof(BatchProblem) * (size_t)nprob, 64);
    BatchProblem *bp = (BatchProblem *)(base + h->problems_offset);
    std::vector<std::pair<int64_t, BatchItem>> work;
    work.reserve((size_t)nitems);
    for (int q = 0; q < nprob; ++q) {
        const ps_problem &p = probs[q];
        const StepCoef c = make_coef(p.lam, p.dt, p._dx, p._dy, p._dz);
        BatchProblem r{};
        r.T = p.T;
        r.T2 = p.T2;
        r.Ci = p.Ci;
        r.dtlam = c.dtlam;
        r.ax = c.ax;
        r.ay = c.ay;
        r.az = c.az;
        r.nx = p.nx;
        r.ny = p.ny;
        r.nz = p.nz;
        const double K[3] = {c.dtlam * c.ax, c.dtlam * c.ay, c.dtlam * c.az};
        bool emu = true;
        for (double v : K) emu = emu && v > 2.2250738585072014e-308 && v < 1e300;
        if (emu) {
            const EmuK kx = emu_const(K[0]), ky = emu_const(K[1]), kz = emu_const(K[2]);
            r.kxm = kx.m;
            r.kym = ky.m;
            r.kzm = kz.m;
            r.kxe = kx.e;
            r.kye = ky.e;
            r.kze = kz.e;
            r.iso = (c.ax == c.ay && c.ay == c.az) ? 1 : 0;
        } else {
            r.iso = -1;  // the kernel takes the plain FP64 expression
        }
        bp[q] = r;
        int tx, ty, tz;
        problem_tiles(p, dtype, tile_x, tile_y, tile_z, &tx, &ty, &tz);
        for (int64_t k0 = 1; k0 < p.nz - 1; k0 += tz)
            for (int64_t j0 = 1; j0 < p.ny - 1; j0 += ty)
                for (int64_t i0 = 1; i0 < p.nx - 1; i0 += tx) {
                    const int64_t ni = std::min<int64_t>(tx, p.nx - 1 - i0);
                    const int64_t nj = std::min<int64_t>(ty, p.ny - 1 - j0);
                    const int64_t nk = std::min<int64_t>(tz, p.nz - 1 - k0);
                    BatchItem it{q, (int32_t)i0, (int32_t)j0, (int32_t)k0, (int16_t)ni, (int16_t)nj,
                                 (int16_t)nk, 0};
                    work.push_back({ni * nj * nk, it});
                }
    }
    // largest items first: the round-robin hand-out then stays balanced
    std::stable_sort(work.begin(), work.end(),
                     [](const std::pair<int64_t, BatchItem> &a, const std::pair<int64_t, BatchItem> &b) {
                         return a.first > b.first;
                     });
    BatchItem *items = (BatchItem *)(base + h->items_offset);
    for (size_t t = 0; t < work.size(); ++t) items[t] = work[t].second;
    if (nitems_out) *nitems_out = nitems;
    return PS_OK;
}

int ps_diffusion3d_batch_step(const void *dev_table, int parity, int dtype, void *stream) {
    if (!dev_table) return fail(PS_ERR_ARG, "dev_table is NULL");
    PS_TRY(check_dtype(dtype));
    if (parity != 0 && parity != 1) return fail(PS_ERR_ARG, "parity %d is not 0 or 1", parity);
    cudaError_t e = launch_batch_step(dev_table, parity, dtype, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_batch_step");
    return PS_OK;
}

int ps_diffusion3d_batch_run(const void *dev_table, int nt, int dtype, unsigned flags,
                             void *stream) {
    if (!dev_table) return fail(PS_ERR_ARG, "dev_table is NULL");
    PS_TRY(check_dtype(dtype));
    if (nt < 0) return fail(PS_ERR_ARG, "nt = %d < 0", nt);
    if (flags & ~PS_RUN_GRAPH) return fail(PS_ERR_ARG, "unsupported flags 0x%x", flags);
    cudaStream_t s = (cudaStream_t)stream;
    batch_prepare(dtype);
    if (!(flags & PS_RUN_GRAPH)) {
        for (int it = 0; it < nt; ++it) {
            cudaError_t e = launch_batch_step(dev_table, it & 1, dtype, s);
            if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_batch_run");
        }
        return PS_OK;
    }
    const GraphKey key{current_device(), dev_table, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0, 0.0,
                       0.0, -1, -1, -1, nt, dtype, 0x80000000u};
    std::lock_guard<std::mutex> lock(g_graph_mu);
    auto it = g_graphs.find(key);
    if (it == g_graphs.end()) {
        cudaStream_t cs;
        cudaError_t e = capture_stream(&cs);
        if (e != cudaSuccess) return cuda_fail(e, "capture stream");
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        cudaError_t le = cudaSuccess;
        for (int t = 0; t < nt && le == cudaSuccess; ++t) le = launch_batch_step(dev_table, t & 1, dtype, cs);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(le, "capturing the batch loop");
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        it = g_graphs.emplace(key, exec).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return PS_OK;
}

}  // extern "C"

// C ABI of the library: host-side argument checks, dispatch to the kernels,
// the CUDA-graph cache of ps_diffusion3d_run_ex and the batch-table builder.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cudaTypedefs.h>

#include "emu64.cuh"
#include "internal.h"
#include "zmarch.h"

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

// Launch-shape overrides (ps_set_launch_override), read by the launchers.
static std::atomic<int> g_override[PS_OVERRIDE_COUNT];

int launch_override(int which) {
    return which >= 0 && which < PS_OVERRIDE_COUNT ? g_override[which].load(std::memory_order_relaxed) : 0;
}
int api_cuda_fail(cudaError_t e, const char *where) { return cuda_fail(e, where); }

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

// Generation of the current device's context: 1 for the first context seen on the
// device, +1 whenever the current context's unique id differs from the last one seen
// (cudaDeviceReset makes a new primary context).  State created inside a context -
// function attributes, the capture stream, cached graphs, a device symbol's address -
// is keyed on it.
unsigned context_generation() {
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_cur = (PFN_cuCtxGetCurrent_v4000)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = (PFN_cuCtxGetId_v12000)p;
    });
    static std::mutex mu;
    static unsigned long long last_id[64] = {0};
    static unsigned gen[64] = {0};
    const int d = current_device();
    if (d < 0 || d >= 64 || !get_cur || !get_id) return 1;
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) {
        cudaSetDevice(d);  // makes the device's primary context current on this thread
        if (get_cur(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    }
    unsigned long long id = 0;
    if (!ctx || get_id(ctx, &id) != CUDA_SUCCESS) return gen[d] ? gen[d] : 1;
    std::lock_guard<std::mutex> lock(mu);
    if (gen[d] == 0 || id != last_id[d]) {
        last_id[d] = id;
        ++gen[d];
    }
    return gen[d];
}

bool set_smem_attr_once(const void *func, int smem, unsigned *done_gen, cudaError_t *err) {
    const int dev = current_device();
    const unsigned g = context_generation();
    *err = cudaSuccess;
    if (dev < 0 || dev >= 64 || done_gen[dev] == g) return true;
    *err = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (*err != cudaSuccess) return false;
    done_gen[dev] = g;
    return true;
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

// One step; E2 / E: correction fields of the two-float state (PS_RUN_COMPENSATED).
// write_bnd: the step also stores T's x and y boundary nodes of planes 1 .. nz-2 into T2
// where the z-march serves it (step_writes_xy_boundary; not with PS_RUN_COMPENSATED).
static cudaError_t enqueue_step(void *T2, const void *T, void *E2, const void *E, const void *Ci,
                                StepCoef c, Grid3 g, int dtype, unsigned flags, cudaStream_t s,
                                bool write_bnd = false) {
    if (dtype == PS_F64) {
        if (flags & PS_RUN_CI_SCALED)
            return launch_step_f64_scaled((double *)T2, (const double *)T, (const double *)Ci, g, s,
                                          write_bnd);
        if (flags & PS_RUN_NATIVE_F64)
            return launch_step_f64_native((double *)T2, (const double *)T, (const double *)Ci, c, g, s);
        return launch_step_f64_fast((double *)T2, (const double *)T, (const double *)Ci, c, g, s, write_bnd);
    }
    if (flags & PS_RUN_COMPENSATED)
        return launch_step_f32_comp((float *)T2, (const float *)T, (float *)E2, (const float *)E,
                                    (const float *)Ci, c, g, s);
    return launch_step_f32((float *)T2, (const float *)T, (const float *)Ci, c, g, s, write_bnd);
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
// `comp` (PS_RUN_COMPENSATED): two correction fields, comp[0, n) paired with T and
// comp[n, 2n) with T2; their boundaries are copied like T's.
static cudaError_t enqueue_run(void *T, void *T2, void *comp, const void *Ci, StepCoef c, Grid3 g,
                               int nt, int dtype, unsigned flags, cudaStream_t s) {
    cudaError_t e = launch_copy_boundary(T2, T, g, elem_bytes(dtype), s);
    float *EA = (float *)comp, *EB = comp ? (float *)comp + g.n() : nullptr;
    if (comp && e == cudaSuccess) e = launch_copy_boundary(EB, EA, g, 4, s);
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
                       : enqueue_step(dst, src, (it & 1) ? EA : EB, (it & 1) ? EB : EA, Ci, c, g, dtype,
                                      flags, s);
    }
    return e;
}

// ---------------------------------------------------------------- graphs
// device, four pointers, lam, dt, _dx, _dy, _dz, nx, ny, nz, nt, dtype, flags (with a marker
// bit per kind of loop), and one more size (the grid stride of a state-keeping loop)
using GraphKey = std::tuple<int, const void *, const void *, const void *, const void *, double,
                            double, double, double, double, int64_t, int64_t, int64_t, int, int,
                            unsigned, int64_t>;
struct CachedGraph {
    cudaGraphExec_t exec;
    uint64_t last_use;  // value of g_graph_clock at the last replay
};
static std::mutex g_graph_mu;
static std::map<GraphKey, CachedGraph> g_graphs;
static uint64_t g_graph_clock = 0;
constexpr size_t kGraphCacheMax = 256;  // least recently used graphs beyond this are destroyed
static cudaStream_t g_capture_stream[64] = {nullptr};
static unsigned g_capture_gen[64] = {0};

// The device's capture stream, created in its current context.  After the context
// changed (cudaDeviceReset) the old stream and the graphs cached for the device are
// handles of a context that no longer exists: they are forgotten, not destroyed.
static cudaError_t capture_stream(cudaStream_t *out) {
    const int d = current_device();
    if (d < 0 || d >= 64) return cudaErrorInvalidDevice;
    const unsigned gen = context_generation();
    if (g_capture_gen[d] != gen) {
        for (auto it = g_graphs.begin(); it != g_graphs.end();)
            it = std::get<0>(it->first) == d ? g_graphs.erase(it) : std::next(it);
        g_capture_stream[d] = nullptr;
    }
    if (!g_capture_stream[d]) {
        cudaError_t e = cudaStreamCreateWithFlags(&g_capture_stream[d], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        g_capture_gen[d] = gen;
    }
    *out = g_capture_stream[d];
    return cudaSuccess;
}

// Replay the CUDA graph cached under `key`, capturing it first from enqueue(stream)
// on the device's capture stream when it is not cached yet.
template <typename F>
static int graph_replay(const GraphKey &key, F &&enqueue, const char *what, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    cudaStream_t cs;
    cudaError_t ce = capture_stream(&cs);  // also drops graphs of a context that is gone
    if (ce != cudaSuccess) return cuda_fail(ce, "capture stream");
    auto it = g_graphs.find(key);
    if (it == g_graphs.end()) {
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        const cudaError_t le = enqueue(cs);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(le, what);
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        if (g_graphs.size() >= kGraphCacheMax) {
            // a graph still running when destroyed is freed by the driver once it completes
            auto lru = g_graphs.begin();
            for (auto jt = g_graphs.begin(); jt != g_graphs.end(); ++jt)
                if (jt->second.last_use < lru->second.last_use) lru = jt;
            cudaGraphExecDestroy(lru->second.exec);
            g_graphs.erase(lru);
        }
        it = g_graphs.emplace(key, CachedGraph{exec, 0}).first;
    }
    it->second.last_use = ++g_graph_clock;
    cudaError_t e = cudaGraphLaunch(it->second.exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return PS_OK;
}

static int run_graph(void *T, void *T2, void *comp, const void *Ci, double lam, double dt,
                     double _dx, double _dy, double _dz, Grid3 g, int nt, int dtype,
                     unsigned flags, cudaStream_t s) {
    const GraphKey key{current_device(), T, T2, comp, Ci, lam, dt, _dx, _dy, _dz, g.nx, g.ny, g.nz,
                       nt, dtype, flags & ~PS_RUN_GRAPH, 0};
    return graph_replay(
        key,
        [&](cudaStream_t cs) {
            return enqueue_run(T, T2, comp, Ci, make_coef(lam, dt, _dx, _dy, _dz), g, nt, dtype, flags, cs);
        },
        "capturing the time loop", s);
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
                adjoint_f32_device_error(clear != 0) | batch_device_error(clear != 0) |
                batch_zmarch_device_error(clear != 0);
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
    cudaError_t e = enqueue_step(T2, T, nullptr, nullptr, Ci, make_coef(lam, dt, _dx, _dy, _dz),
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
    cudaError_t e = enqueue_step(T2, T, nullptr, nullptr, Ci, make_coef(lam, dt, _dx, _dy, _dz),
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

int ps_diffusion3d_step_comp_f32(float *T2, const float *T, float *E2, const float *E, const float *Ci,
                                 double lam, double dt, double _dx, double _dy, double _dz,
                                 int64_t nx, int64_t ny, int64_t nz, void *stream) {
    PS_TRY(check_step_args(T2, T, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz, PS_F32));
    PS_TRY(check_ptr(E2, "E2"));
    PS_TRY(check_ptr(E, "E"));
    const size_t bytes = (size_t)(nx * ny * nz) * 4;
    if (overlap(E2, T, bytes) || overlap(E2, T2, bytes) || overlap(E2, Ci, bytes) || overlap(E2, E, bytes))
        return fail(PS_ERR_ALIAS, "E2 overlaps T, T2, E or Ci");
    if (overlap(E, T2, bytes)) return fail(PS_ERR_ALIAS, "E overlaps T2");
    cudaError_t e = launch_step_f32_comp(T2, T, E2, E, Ci, make_coef(lam, dt, _dx, _dy, _dz),
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

// The grid slot holding the state after step t of a state-keeping loop (see
// ps_diffusion3d_run_states), and the enqueue of its boundary copy and steps.
namespace psd {
static int states_slot_after(int t, int every, int &cur_slot, int &work_next) {
    int slot;
    if (t % every == 0) {
        slot = t / every - 1;
    } else {  // a work grid, never the one this step reads
        if (cur_slot == -1 - work_next) work_next ^= 1;
        slot = -1 - work_next;
        work_next ^= 1;
    }
    cur_slot = slot;
    return slot;
}

// The launches of a state-keeping loop: each advances the state by `steps` (1, or 2
// for a fused pair) and writes it to slot `dst` (>= 0 a state slot, -1 / -2 work grid
// 0 / 1).  With every = 1 a pair also keeps its intermediate state (in slot dst - 1);
// with every > 1 a pair never steps over a state that is kept.  Returns the slot of
// T(nt) (-3: T0 itself, nt = 0).
struct StatesOp {
    int steps, dst;
};
static int plan_states(int nt, int every, bool pairs, std::vector<StatesOp> *ops) {
    int cur_slot = -3, work_next = 0, t = 0;
    while (t < nt) {
        const int next_kept = every == 1 ? t + 2 : (t / every + 1) * every;
        const int k = (pairs && t + 2 <= nt && t + 2 <= next_kept) ? 2 : 1;
        if (k == 2 && every == 1) states_slot_after(t + 1, every, cur_slot, work_next);
        const int dst = states_slot_after(t + k, every, cur_slot, work_next);
        if (ops) ops->push_back({k, dst});
        t += k;
    }
    return cur_slot;
}

// Whether PS_RUN_TEMPORAL2 runs fused pairs for this state-keeping loop (at least two
// grids): FP32 where the pair kernel serves every grid (all 16-byte aligned at one
// stride, so T0 and the first two grids decide).
static bool states_pairs(unsigned flags, int dtype, int nt, Grid3 g, const void *T0, const void *grid0,
                         const void *grid1, const void *Ci) {
    return (flags & PS_RUN_TEMPORAL2) && dtype == PS_F32 && nt >= 2 && temporal2_ok(g, dtype, T0, grid0, Ci) &&
           temporal2_ok(g, dtype, grid0, grid1, Ci);
}

static cudaError_t enqueue_run_states(const void *T0, char *base, int64_t grid_stride, size_t esz, int every,
                                      const void *Ci, StepCoef c, Grid3 g, int nt, int dtype, unsigned flags,
                                      cudaStream_t s) {
    const int nslots = nt / every, nwork = (every > 1 && nt > 0) ? 2 : 0;
    auto grid = [&](int slot) { return (void *)(base + (size_t)slot * (size_t)grid_stride * esz); };
    auto slot_grid = [&](int slot) { return slot >= 0 ? grid(slot) : grid(nslots + (-1 - slot)); };
    // The boundary of every grid this call writes is T0's.  Where the z-march serves the
    // steps they store the x and y faces themselves (in their coalesced row stores), so
    // only the two z faces of each grid are copied here; else the whole boundary is.
    const bool scaled = (flags & PS_RUN_CI_SCALED) != 0, native = (flags & PS_RUN_NATIVE_F64) != 0;
    const int ngrids = nslots + nwork;
    bool steps_bnd = true;
    for (int k = 0; k < ngrids && steps_bnd; ++k)
        steps_bnd = step_writes_xy_boundary(dtype, scaled, native, c, g, grid(k), T0, Ci) &&
                    step_writes_xy_boundary(dtype, scaled, native, c, g, grid(k), grid(k), Ci);
    // PS_RUN_TEMPORAL2 (FP32): fused pairs.  With every = 1 they keep both states and
    // store both states' x and y faces; with every > 1 they keep only their second state
    // and write interior nodes only, so the whole boundary is copied then.
    const bool pairs = ngrids >= 2 && states_pairs(flags, dtype, nt, g, T0, grid(0), grid(1), Ci);
    const bool faces_by_steps = steps_bnd && !(pairs && every > 1);
    if (nt > 0 && ngrids > 0) {
        cudaError_t e = launch_copy_boundary_many(base, ngrids, grid_stride, T0, g, (int)esz, s, faces_by_steps);
        if (e != cudaSuccess) return e;
    }
    std::vector<StatesOp> ops;
    plan_states(nt, every, pairs, &ops);
    const void *cur = T0;
    for (const StatesOp &op : ops) {
        void *dst = slot_grid(op.dst);
        cudaError_t e;
        if (op.steps == 2 && every == 1)
            e = launch_step2_states_f32((float *)grid(op.dst - 1), (float *)dst, (const float *)cur,
                                        (const float *)Ci, c, g, s);
        else if (op.steps == 2)
            e = enqueue_step2(dst, cur, Ci, c, g, dtype, s);
        else
            e = enqueue_step(dst, cur, nullptr, nullptr, Ci, c, g, dtype, flags, s, faces_by_steps);
        if (e != cudaSuccess) return e;
        cur = dst;
    }
    return cudaSuccess;
}
}  // namespace psd

int ps_diffusion3d_run_states(const void *T0, void *states, int64_t grid_stride, int every,
                              const void *Ci, double lam, double dt, double _dx, double _dy,
                              double _dz, int64_t nx, int64_t ny, int64_t nz, int nt, int dtype,
                              unsigned flags, void *stream, int *final_slot) {
    PS_TRY(check_step_args(states, T0, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz, dtype));
    if (nt < 0) return fail(PS_ERR_ARG, "nt = %d < 0", nt);
    if (every < 1) return fail(PS_ERR_ARG, "every = %d < 1", every);
    if (!final_slot) return fail(PS_ERR_ARG, "final_slot is NULL");
    if (flags & ~(PS_RUN_CI_SCALED | PS_RUN_NATIVE_F64 | PS_RUN_GRAPH | PS_RUN_TEMPORAL2))
        return fail(PS_ERR_ARG, "unknown flags 0x%x", flags);
    PS_TRY(check_scaled(flags, dtype, _dx, _dy, _dz));
    if ((flags & PS_RUN_NATIVE_F64) && dtype != PS_F64)
        return fail(PS_ERR_UNSUPPORTED, "PS_RUN_NATIVE_F64 needs PS_F64");
    if ((flags & PS_RUN_TEMPORAL2) && dtype != PS_F32)
        return fail(PS_ERR_UNSUPPORTED, "PS_RUN_TEMPORAL2 in the state-keeping loop needs PS_F32");
    const int64_t n = nx * ny * nz;
    const size_t esz = elem_bytes(dtype);
    if (grid_stride < n || (grid_stride * (int64_t)esz) % 16 != 0)
        return fail(PS_ERR_ARG, "grid_stride = %lld: need >= nx*ny*nz and a multiple of 16 bytes",
                    (long long)grid_stride);
    const int nslots = nt / every, nwork = (every > 1 && nt > 0) ? 2 : 0;
    const size_t span = (size_t)grid_stride * esz * (size_t)(nslots + nwork);
    if (span && (overlap2(states, span, T0, (size_t)n * esz) || overlap2(states, span, Ci, (size_t)n * esz)))
        return fail(PS_ERR_ALIAS, "the state grids overlap T0 or Ci");
    const StepCoef c = make_coef(lam, dt, _dx, _dy, _dz);
    const Grid3 g{nx, ny, nz};
    char *base = (char *)states;
    // the slot of T(nt), from the same plan the launches follow
    const int nall = nslots + nwork;
    auto grid_at = [&](int k) { return (const void *)(base + (size_t)k * (size_t)grid_stride * esz); };
    const bool pairs = nall >= 2 && states_pairs(flags, dtype, nt, g, T0, grid_at(0), grid_at(1), Ci);
    const int cur_slot = plan_states(nt, every, pairs, nullptr);
    const unsigned f = flags & ~PS_RUN_GRAPH;
    cudaStream_t s = (cudaStream_t)stream;
    if ((flags & PS_RUN_GRAPH) && nt > 0) {
        // state-keeping keys: marker bit 0x40000000, `every` in the third pointer slot
        const GraphKey key{current_device(), T0, states, (const void *)(intptr_t)every, Ci, lam, dt, _dx, _dy,
                           _dz, nx, ny, nz, nt, dtype, 0x40000000u | f, grid_stride};
        const int st = graph_replay(
            key,
            [&](cudaStream_t cs) {
                return enqueue_run_states(T0, base, grid_stride, esz, every, Ci, c, g, nt, dtype, f, cs);
            },
            "capturing the state-keeping time loop", s);
        if (st != PS_OK) return st;
    } else {
        cudaError_t e = enqueue_run_states(T0, base, grid_stride, esz, every, Ci, c, g, nt, dtype, f, s);
        if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_run_states");
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
        if (overlap2(comp, 2 * bytes, T, bytes) || overlap2(comp, 2 * bytes, T2, bytes) ||
            overlap2(comp, 2 * bytes, Ci, bytes))
            return fail(PS_ERR_ALIAS, "comp (two fields) overlaps T, T2 or Ci");
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

size_t ps_graph_cache_size(void) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    return g_graphs.size();
}

int ps_clear_graph_cache(void) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (auto &kv : g_graphs) cudaGraphExecDestroy(kv.second.exec);
    g_graphs.clear();
    return PS_OK;
}

int ps_set_launch_override(int which, int value) {
    if (which < 0 || which >= PS_OVERRIDE_COUNT)
        return fail(PS_ERR_ARG, "override %d is not a PS_OVERRIDE_* value", which);
    const bool flag = which == PS_OVERRIDE_ADJ_PLAIN || which == PS_OVERRIDE_F64_PX2 ||
                      which == PS_OVERRIDE_STEP_PLAIN;
    if (value < 0 || (flag && value > 1) || (!flag && value > 4096))
        return fail(PS_ERR_ARG, "override %d: value %d out of range (%s)", which, value,
                    flag ? "0 or 1" : "0 .. 4096");
    // cached graphs hold the launch shapes chosen at capture: drop them on a change
    if (g_override[which].exchange(value) != value) return ps_clear_graph_cache();
    return PS_OK;
}

int ps_get_launch_override(int which, int *value) {
    if (!value) return fail(PS_ERR_ARG, "value is NULL");
    if (which < 0 || which >= PS_OVERRIDE_COUNT)
        return fail(PS_ERR_ARG, "override %d is not a PS_OVERRIDE_* value", which);
    *value = g_override[which].load();
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

int ps_diffusion3d_adjoint2_ex(void *Tbar, void *Cibar, const void *ybar, const void *T_first,
                               const void *T_second, const void *Ci, double lam, double dt, double _dx,
                               double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz, int dtype,
                               unsigned flags, void *stream) {
    if (flags) return fail(PS_ERR_ARG, "unknown flags 0x%x", flags);
    PS_TRY(check_dtype(dtype));
    PS_TRY(check_grid(nx, ny, nz));
    PS_TRY(check_ptr(Tbar, "Tbar"));
    PS_TRY(check_ptr(Cibar, "Cibar"));
    PS_TRY(check_ptr(ybar, "ybar"));
    PS_TRY(check_ptr(T_first, "T_first"));
    PS_TRY(check_ptr(T_second, "T_second"));
    PS_TRY(check_ptr(Ci, "Ci"));
    PS_TRY(check_finite(lam, "lam"));
    PS_TRY(check_finite(dt, "dt"));
    PS_TRY(check_finite(_dx, "_dx"));
    PS_TRY(check_finite(_dy, "_dy"));
    PS_TRY(check_finite(_dz, "_dz"));
    const size_t bytes = (size_t)(nx * ny * nz) * elem_bytes(dtype);
    if (overlap(Tbar, ybar, bytes) || overlap(Tbar, T_first, bytes) || overlap(Tbar, T_second, bytes) ||
        overlap(Tbar, Ci, bytes) || overlap(Tbar, Cibar, bytes))
        return fail(PS_ERR_ALIAS, "Tbar overlaps an input");
    if (overlap(Cibar, ybar, bytes) || overlap(Cibar, T_first, bytes) || overlap(Cibar, T_second, bytes) ||
        overlap(Cibar, Ci, bytes))
        return fail(PS_ERR_ALIAS, "Cibar overlaps an input");
    if (dtype != PS_F32)
        return fail(PS_ERR_UNSUPPORTED, "fused transposed pairs are FP32 (the FP64 step is issue-bound)");
    const Grid3 g{nx, ny, nz};
    const void *ptrs[6] = {T_first, T_second, ybar, Ci, Cibar, Tbar};
    if (!adjoint_f32_supported(g, ptrs, 6))
        return fail(PS_ERR_UNSUPPORTED, "fused transposed pairs need nx*4 a multiple of 16 and a CUDA driver");
    const StepCoef c = make_coef(lam, dt, _dx, _dy, _dz);
    cudaError_t e = launch_adjoint2_f32((float *)Tbar, (float *)Cibar, (const float *)ybar,
                                        (const float *)T_first, (const float *)T_second, (const float *)Ci,
                                        c, g, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_adjoint2_ex");
    return PS_OK;
}

// ------------------------------------------------------------------ 2-D
static int check_2d(const void *T2, const void *T, const void *Ci, double lam, double dt, double _dx,
                    double _dy, int64_t nx, int64_t ny, int dtype, unsigned flags, unsigned allowed) {
    if (flags & ~allowed) return fail(PS_ERR_ARG, "unknown flags 0x%x", flags);
    PS_TRY(check_dtype(dtype));
    if (nx < 3 || ny < 3) return fail(PS_ERR_ARG, "grid %lld x %lld: every size must be >= 3", (long long)nx,
                                      (long long)ny);
    if (nx > (1LL << 40) || ny > (1LL << 40) || (double)nx * (double)ny > 9.0e15)
        return fail(PS_ERR_ARG, "grid %lld x %lld is too large", (long long)nx, (long long)ny);
    PS_TRY(check_ptr(T2, "T2"));
    PS_TRY(check_ptr(T, "T"));
    PS_TRY(check_ptr(Ci, "Ci"));
    PS_TRY(check_finite(lam, "lam"));
    PS_TRY(check_finite(dt, "dt"));
    PS_TRY(check_finite(_dx, "_dx"));
    PS_TRY(check_finite(_dy, "_dy"));
    const size_t bytes = (size_t)(nx * ny) * elem_bytes(dtype);
    if (overlap(T2, T, bytes)) return fail(PS_ERR_ALIAS, "T2 overlaps T");
    if (overlap(T2, Ci, bytes)) return fail(PS_ERR_ALIAS, "T2 overlaps Ci");
    if (flags & PS_RUN_CI_SCALED) {
        if (dtype != PS_F64) return fail(PS_ERR_UNSUPPORTED, "a pre-scaled Ci needs PS_F64");
        if (_dx != _dy) return fail(PS_ERR_UNSUPPORTED, "a pre-scaled Ci needs equal spacings (_dx == _dy)");
    }
    return PS_OK;
}

static int mode_2d(int dtype, unsigned flags, StepCoef c) {
    if (dtype == PS_F32) return Z_F32;
    if (flags & PS_RUN_CI_SCALED) return Z_F64_SCALED;
    const double K = c.dtlam * c.ax;
    if (c.ax == c.ay && K > 2.2250738585072014e-308 && K < 1e300) return Z_F64_EMU_ISO_DMUL;
    return Z_F64_NATIVE;
}

int ps_diffusion2d_step(void *T2, const void *T, const void *Ci, double lam, double dt, double _dx,
                        double _dy, int64_t nx, int64_t ny, int dtype, unsigned flags, void *stream) {
    PS_TRY(check_2d(T2, T, Ci, lam, dt, _dx, _dy, nx, ny, dtype, flags, PS_RUN_CI_SCALED));
    const StepCoef c = make_coef(lam, dt, _dx, _dy, 0.0);
    cudaError_t e = launch_step2d(mode_2d(dtype, flags, c), T2, T, Ci, c, nx, ny, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion2d_step");
    return PS_OK;
}

static cudaError_t enqueue_run2d(void *T, void *T2, const void *Ci, StepCoef c, int64_t nx, int64_t ny,
                                 int nt, int dtype, unsigned flags, cudaStream_t s) {
    if (nt == 0) return cudaSuccess;
    cudaError_t e = launch_copy_edges2d(T2, T, nx, ny, (int)elem_bytes(dtype), s);
    const int mode = mode_2d(dtype, flags, c);
    for (int it = 0; it < nt && e == cudaSuccess; ++it)
        e = it & 1 ? launch_step2d(mode, T, T2, Ci, c, nx, ny, s) : launch_step2d(mode, T2, T, Ci, c, nx, ny, s);
    return e;
}

int ps_diffusion2d_run(void *T, void *T2, const void *Ci, double lam, double dt, double _dx, double _dy,
                       int64_t nx, int64_t ny, int nt, int dtype, unsigned flags, void *stream,
                       int *result_in_T2) {
    PS_TRY(check_2d(T2, T, Ci, lam, dt, _dx, _dy, nx, ny, dtype, flags, PS_RUN_CI_SCALED | PS_RUN_GRAPH));
    if (nt < 0) return fail(PS_ERR_ARG, "nt = %d < 0", nt);
    if (result_in_T2) *result_in_T2 = nt & 1;
    const StepCoef c = make_coef(lam, dt, _dx, _dy, 0.0);
    cudaStream_t s = (cudaStream_t)stream;
    if (flags & PS_RUN_GRAPH) {
        // 2-D keys: nz = -2 marks them apart from the 3-D time loops
        const GraphKey key{current_device(), T, T2, nullptr, Ci, lam, dt, _dx, _dy, 0.0, nx, ny, -2, nt, dtype,
                           flags & ~PS_RUN_GRAPH, 0};
        return graph_replay(
            key, [&](cudaStream_t cs) { return enqueue_run2d(T, T2, Ci, c, nx, ny, nt, dtype, flags, cs); },
            "capturing the 2-D time loop", s);
    }
    cudaError_t e = enqueue_run2d(T, T2, Ci, c, nx, ny, nt, dtype, flags, s);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion2d_run");
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

// Result slots of the blocking reductions: pinned, mapped host memory that the
// finishing kernel stores to directly.  A device-to-host memcpy of the 8-byte result
// would wait behind large copies that other streams have in flight on the copy
// engine (a 1 GiB copy out of an earlier result holds it for milliseconds); a kernel
// store does not use the copy engine.  One slot per concurrent call, kept for the
// life of the context (device, context generation) that allocated it.
class HostSlots {
public:
    double *acquire(cudaError_t *err) {
        const uint64_t key = ((uint64_t)(unsigned)current_device() << 32) | context_generation();
        {
            std::lock_guard<std::mutex> lock(mu_);
            auto &v = free_[key];
            if (!v.empty()) {
                double *p = v.back();
                v.pop_back();
                *err = cudaSuccess;
                return p;
            }
        }
        void *p = nullptr;
        *err = cudaHostAlloc(&p, 64, cudaHostAllocMapped);
        return *err == cudaSuccess ? (double *)p : nullptr;
    }
    void release(double *p) {
        const uint64_t key = ((uint64_t)(unsigned)current_device() << 32) | context_generation();
        std::lock_guard<std::mutex> lock(mu_);
        free_[key].push_back(p);
    }

private:
    std::mutex mu_;
    std::map<uint64_t, std::vector<double *>> free_;
};
static HostSlots g_host_slots;

int ps_maximum(double *out_host, const void *A, int64_t n, int dtype, void *workspace,
               void *stream) {
    if (!out_host) return fail(PS_ERR_ARG, "out_host is NULL");
    PS_TRY(check_reduce(A, n, dtype, workspace));
    cudaError_t e = cudaSuccess;
    double *slot = g_host_slots.acquire(&e);
    if (!slot) return cuda_fail(e, "ps_maximum: allocating its host result slot");
    double *slot_dev = nullptr;
    e = cudaHostGetDevicePointer((void **)&slot_dev, slot, 0);
    if (e == cudaSuccess) e = launch_maximum(slot_dev, A, n, dtype, workspace, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) *out_host = *(volatile double *)slot;
    g_host_slots.release(slot);
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

int ps_diffusion2d_stable_dt(double *dt_host, const void *Ci, int64_t nx, int64_t ny, double lam,
                             double lx, double ly, int dtype, void *workspace, void *stream) {
    if (!dt_host) return fail(PS_ERR_ARG, "dt_host is NULL");
    if (nx < 3 || ny < 3) return fail(PS_ERR_ARG, "grid %lld x %lld: every size must be >= 3", (long long)nx,
                                      (long long)ny);
    PS_TRY(check_finite(lam, "lam"));
    double mx = 0.0;
    PS_TRY(ps_maximum(&mx, Ci, nx * ny, dtype, workspace, stream));
    const double dx = lx / (double)(nx - 1), dy = ly / (double)(ny - 1);
    const double m = dy * dy < dx * dx ? dy * dy : dx * dx;
    *dt_host = m / lam / mx / 4.1;
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

int ps_to_deviation_pair(float *D, float *E, const double *T, double t_ref, int64_t n, void *stream) {
    if (n < 1) return fail(PS_ERR_ARG, "n = %lld < 1", (long long)n);
    PS_TRY(check_ptr(D, "D"));
    PS_TRY(check_ptr(E, "E"));
    PS_TRY(check_ptr(T, "T"));
    PS_TRY(check_finite(t_ref, "t_ref"));
    if (overlap2(D, (size_t)n * 4, T, (size_t)n * 8) || overlap2(E, (size_t)n * 4, T, (size_t)n * 8) ||
        overlap(D, E, (size_t)n * 4))
        return fail(PS_ERR_ALIAS, "D, E and T must not overlap");
    cudaError_t e = launch_to_deviation_pair(D, E, T, t_ref, n, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_to_deviation_pair");
    return PS_OK;
}

int ps_from_deviation_pair(double *T, const float *D, const float *E, double t_ref, int64_t n,
                           void *stream) {
    if (n < 1) return fail(PS_ERR_ARG, "n = %lld < 1", (long long)n);
    PS_TRY(check_ptr(T, "T"));
    PS_TRY(check_ptr(D, "D"));
    PS_TRY(check_ptr(E, "E"));
    PS_TRY(check_finite(t_ref, "t_ref"));
    if (overlap2(D, (size_t)n * 4, T, (size_t)n * 8) || overlap2(E, (size_t)n * 4, T, (size_t)n * 8))
        return fail(PS_ERR_ALIAS, "T overlaps D or E");
    cudaError_t e = launch_from_deviation_pair(T, D, E, t_ref, n, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_from_deviation_pair");
    return PS_OK;
}

// ------------------------------------------------------------------ batch
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// kernel 1 (z-march): the x-y tile is the kernel's own; default chunks of 64 planes
// (measured on the 256-problem workload: 64 >= 32 > 16 > 8 planes, FP32 and FP64)
static int resolve_tiles(int dtype, int *tx, int *ty, int *tz, int kernel = 0) {
    int dx, dy, dz;
    batch_default_tile(dtype, &dx, &dy, &dz);
    if (kernel == 1) dz = 64;
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
                         int *oz, int kernel) {
    *ox = p.tile_x ? p.tile_x : tx;
    *oy = p.tile_y ? p.tile_y : ty;
    *oz = p.tile_z ? p.tile_z : tz;
    return resolve_tiles(dtype, ox, oy, oz, kernel);
}

static int64_t pitch_of(const ps_problem &p) { return p.pitch ? p.pitch : p.nx; }

// Everything ps_diffusion3d_step checks, over fields whose rows are pitch elements apart.
static int check_batch_problem(const ps_problem &p, int dtype) {
    PS_TRY(check_dtype(dtype));
    PS_TRY(check_grid(p.nx, p.ny, p.nz));
    PS_TRY(check_ptr(p.T2, "T2"));
    PS_TRY(check_ptr(p.T, "T"));
    PS_TRY(check_ptr(p.Ci, "Ci"));
    PS_TRY(check_finite(p.lam, "lam"));
    PS_TRY(check_finite(p.dt, "dt"));
    PS_TRY(check_finite(p._dx, "_dx"));
    PS_TRY(check_finite(p._dy, "_dy"));
    PS_TRY(check_finite(p._dz, "_dz"));
    const int64_t pitch = pitch_of(p);
    if (pitch < p.nx) return fail(PS_ERR_ARG, "pitch %d < nx = %lld", p.pitch, (long long)p.nx);
    // column-kernel offsets are 32-bit
    if ((double)pitch * (double)p.ny * (double)p.nz >= 2147483648.0 || p.nx + 4096 > (1LL << 31) ||
        p.ny + 4096 > (1LL << 31) || p.nz + 32767 > (1LL << 31))
        return fail(PS_ERR_ARG, "problem is too large for the batch table (2^31 nodes at most)");
    const size_t span = (size_t)((pitch * p.ny) * (p.nz - 1) + pitch * (p.ny - 1) + p.nx) * elem_bytes(dtype);
    if (overlap(p.T2, p.T, span)) return fail(PS_ERR_ALIAS, "T2 overlaps T");
    if (overlap(p.T2, p.Ci, span)) return fail(PS_ERR_ALIAS, "T2 overlaps Ci");
    return PS_OK;
}

// Why the z-march kernel cannot take this problem (nullptr: it can).
static const char *zmarch_refusal(const ps_problem &p, int dtype, bool scaled) {
    const int esz = (int)elem_bytes(dtype);
    if (!tma_encoder_available()) return "the tensor-map encoder of the CUDA driver is not available";
    if ((pitch_of(p) * esz) % 16 != 0) return "the row pitch is not a multiple of 16 bytes";
    if (p.nx > (1LL << 31) - 256 || p.ny > (1LL << 31) - 64 || p.nz > (1LL << 31) - 2)
        return "the grid is too large for 32-bit tensor coordinates";
    if (dtype == PS_F64) {
        if (p._dx != p._dy || p._dy != p._dz) return "FP64 needs equal spacings";
        if (!scaled) {
            const StepCoef c = make_coef(p.lam, p.dt, p._dx, p._dy, p._dz);
            const double K = c.dtlam * c.ax;
            if (!(K > 2.2250738585072014e-308 && K < 1e300))
                return "FP64 needs a positive step coefficient dt*lam*_dx^2 in the normal range";
        }
    }
    return nullptr;
}

// Kernel of a table for these problems and flags: 0 column, 1 z-march, or an error status.
static int choose_kernel(const ps_problem *probs, int nprob, int dtype, unsigned flags) {
    if (flags & ~(PS_BATCH_COLUMN | PS_BATCH_ZMARCH | PS_BATCH_CI_SCALED | PS_BATCH_TEMPORAL2))
        return fail(PS_ERR_ARG, "unsupported batch flags 0x%x", flags);
    if ((flags & PS_BATCH_TEMPORAL2) && (flags & PS_BATCH_COLUMN))
        return fail(PS_ERR_ARG, "PS_BATCH_TEMPORAL2 needs the z-march kernel");
    if ((flags & PS_BATCH_TEMPORAL2) && dtype == PS_F64 && !(flags & PS_BATCH_CI_SCALED))
        return fail(PS_ERR_ARG, "PS_BATCH_TEMPORAL2 on FP64 needs PS_BATCH_CI_SCALED");
    if ((flags & PS_BATCH_COLUMN) && (flags & PS_BATCH_ZMARCH))
        return fail(PS_ERR_ARG, "PS_BATCH_COLUMN and PS_BATCH_ZMARCH exclude each other");
    const bool scaled = (flags & PS_BATCH_CI_SCALED) != 0;
    if (scaled && dtype != PS_F64) return fail(PS_ERR_ARG, "PS_BATCH_CI_SCALED is for FP64 problems");
    if (scaled && (flags & PS_BATCH_COLUMN))
        return fail(PS_ERR_ARG, "PS_BATCH_CI_SCALED needs the z-march kernel");
    if (flags & PS_BATCH_COLUMN) return 0;
    for (int q = 0; q < nprob; ++q) {
        const char *why = zmarch_refusal(probs[q], dtype, scaled);
        if (why) {
            if ((flags & (PS_BATCH_ZMARCH | PS_BATCH_TEMPORAL2)) || scaled)
                return fail(PS_ERR_UNSUPPORTED, "problem %d: %s", q, why);
            return 0;
        }
    }
    return 1;
}

static int64_t items_of(const ps_problem &p, int kernel, int dtype, int tx, int ty, int tz) {
    if (kernel == 1) return batch_zmarch_xy_tiles(dtype, p.nx, p.ny, nullptr) * ((p.nz - 2 + tz - 1) / tz);
    return ((p.nx - 2 + tx - 1) / tx) * ((p.ny - 2 + ty - 1) / ty) * ((p.nz - 2 + tz - 1) / tz);
}

struct TableLayout {
    size_t problems, zparams, z2params, maps, items, items2, bytes;
};

static TableLayout table_layout(int nprob, int64_t nitems, int64_t nitems2, int kernel) {
    TableLayout L{};
    L.problems = align_up(sizeof(BatchHeader), 128);
    size_t end = L.problems + align_up(sizeof(BatchProblem) * (size_t)nprob, 128);
    if (kernel == 1) {
        L.zparams = end;
        end += align_up(sizeof(ZParams) * (size_t)nprob, 128);
        L.z2params = end;
        end += align_up(batch_z2params_bytes() * (size_t)nprob, 128);
        L.maps = end;  // tensor maps want 64-byte alignment
        end += sizeof(CUtensorMap) * kBatchZmarchMaps * (size_t)nprob;
    }
    L.items = end;
    end += sizeof(BatchItem) * (size_t)nitems;
    L.items2 = end;
    L.bytes = end + sizeof(BatchItem) * (size_t)nitems2;
    return L;
}

// Work items and layout of a table (status, or PS_OK with *nitems and *kernel set).
static int plan_table(const ps_problem *probs, int nprob, int dtype, int tile_x, int tile_y, int tile_z,
                      unsigned flags, int64_t *nitems, int64_t *nitems2, int *kernel) {
    if (!probs) return fail(PS_ERR_ARG, "probs is NULL");
    if (nprob < 1) return fail(PS_ERR_ARG, "nprob = %d < 1", nprob);
    PS_TRY(check_dtype(dtype));
    {
        int tx = tile_x, ty = tile_y, tz = tile_z;
        PS_TRY(resolve_tiles(dtype, &tx, &ty, &tz));
    }
    for (int q = 0; q < nprob; ++q) {
        const int st = check_batch_problem(probs[q], dtype);
        if (st != PS_OK) return fail(st, "problem %d: %s", q, g_err.c_str());
    }
    const int k = choose_kernel(probs, nprob, dtype, flags);
    if (k < 0) return k;
    PS_TRY(resolve_tiles(dtype, &tile_x, &tile_y, &tile_z, k));
    int64_t n = 0, n2 = 0;
    for (int q = 0; q < nprob; ++q) {
        int tx, ty, tz;
        const int st = problem_tiles(probs[q], dtype, tile_x, tile_y, tile_z, &tx, &ty, &tz, k);
        if (st != PS_OK) return fail(st, "problem %d: %s", q, g_err.c_str());
        n += items_of(probs[q], k, dtype, tx, ty, tz);
        if (flags & PS_BATCH_TEMPORAL2)
            n2 += batch_zmarch2_xy_tiles(dtype, probs[q].nx, probs[q].ny, nullptr) * ((probs[q].nz - 2 + tz - 1) / tz);
    }
    if (k == 1 && (n > 0x7fffffffLL || n2 > 0x7fffffffLL))
        return fail(PS_ERR_ARG, "%lld work items: at most 2^31-1", (long long)std::max(n, n2));
    *nitems = n;
    *nitems2 = n2;
    *kernel = k;
    return PS_OK;
}

size_t ps_batch_table_bytes_ex(const ps_problem *probs, int nprob, int dtype, int tile_x, int tile_y,
                               int tile_z, unsigned flags) {
    int64_t nitems = 0, nitems2 = 0;
    int kernel = 0;
    if (plan_table(probs, nprob, dtype, tile_x, tile_y, tile_z, flags, &nitems, &nitems2, &kernel) != PS_OK)
        return 0;
    return table_layout(nprob, nitems, nitems2, kernel).bytes;
}

size_t ps_batch_table_bytes(const ps_problem *probs, int nprob, int dtype, int tile_x, int tile_y,
                            int tile_z) {
    return ps_batch_table_bytes_ex(probs, nprob, dtype, tile_x, tile_y, tile_z, PS_BATCH_COLUMN);
}

int ps_batch_table_fill_ex(void *host_buf, size_t bytes, const ps_problem *probs, int nprob, int dtype,
                           int tile_x, int tile_y, int tile_z, unsigned flags, int64_t *nitems_out) {
    if (!host_buf) return fail(PS_ERR_ARG, "host_buf is NULL");
    int64_t nitems = 0, nitems2 = 0;
    int kernel = 0;
    PS_TRY(plan_table(probs, nprob, dtype, tile_x, tile_y, tile_z, flags, &nitems, &nitems2, &kernel));
    PS_TRY(resolve_tiles(dtype, &tile_x, &tile_y, &tile_z, kernel));
    const TableLayout L = table_layout(nprob, nitems, nitems2, kernel);
    if (bytes < L.bytes) return fail(PS_ERR_ARG, "table buffer has %zu bytes, needs %zu", bytes, L.bytes);
    if (kernel == 1 && ((uintptr_t)host_buf & 63u))
        return fail(PS_ERR_ALIGN, "host_buf must be 64-byte aligned for the tensor maps");
    const bool scaled = (flags & PS_BATCH_CI_SCALED) != 0;
    std::memset(host_buf, 0, L.bytes);
    char *base = (char *)host_buf;
    BatchHeader *h = (BatchHeader *)base;
    h->nprob = nprob;
    h->nitems = nitems;
    h->dtype = dtype;
    h->tile_x = tile_x;
    h->tile_y = tile_y;
    h->tile_z = tile_z;
    h->problems_offset = (int64_t)L.problems;
    h->items_offset = (int64_t)L.items;
    h->kernel = kernel;
    h->zmode = kernel == 1 ? (dtype == PS_F32 ? Z_F32 : (scaled ? Z_F64_SCALED : Z_F64_EMU_ISO_DMUL)) : -1;
    h->zparams_offset = (int64_t)L.zparams;
    h->maps_offset = (int64_t)L.maps;
    h->nitems2 = nitems2;
    h->items2_offset = (int64_t)L.items2;
    h->z2params_offset = (int64_t)L.z2params;
    BatchProblem *bp = (BatchProblem *)(base + L.problems);
    std::vector<std::pair<int64_t, BatchItem>> work, work2;
    work.reserve((size_t)nitems);
    work2.reserve((size_t)nitems2);
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
        r.pitch = pitch_of(p);
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
            r.iso = -1;  // the column kernel takes the plain FP64 expression
        }
        bp[q] = r;
        int tx, ty, tz;
        problem_tiles(p, dtype, tile_x, tile_y, tile_z, &tx, &ty, &tz, kernel);
        if (kernel == 1) {
            if (!batch_zmarch_fill(base + L.zparams + sizeof(ZParams) * q,
                                   base + L.z2params + batch_z2params_bytes() * q,
                                   base + L.maps + sizeof(CUtensorMap) * kBatchZmarchMaps * q, r, c,
                                   dtype))
                return fail(PS_ERR_UNSUPPORTED, "problem %d: tensor-map encoding failed", q);
            // x-y tiles of the whole plane from the origin (boundary included), like the
            // single-grid kernel, times z-chunks of the interior planes
            std::vector<BatchItem> xy((size_t)batch_zmarch_xy_tiles(dtype, p.nx, p.ny, nullptr));
            batch_zmarch_xy_tiles(dtype, p.nx, p.ny, xy.data());
            for (int64_t k0 = 1; k0 < p.nz - 1; k0 += tz)
                for (const BatchItem &t : xy) {
                    BatchItem it = t;
                    it.prob = q;
                    it.k0 = (int32_t)k0;
                    it.ni = it.nj = 0;
                    it.nk = (int16_t)std::min<int64_t>(tz, p.nz - 1 - k0);
                    work.push_back({0, it});
                }
            if (nitems2) {  // the fused-pair list: wide tiles only, the same z-chunks
                std::vector<BatchItem> xy2((size_t)batch_zmarch2_xy_tiles(dtype, p.nx, p.ny, nullptr));
                batch_zmarch2_xy_tiles(dtype, p.nx, p.ny, xy2.data());
                for (int64_t k0 = 1; k0 < p.nz - 1; k0 += tz)
                    for (const BatchItem &t : xy2) {
                        BatchItem it = t;
                        it.prob = q;
                        it.k0 = (int32_t)k0;
                        it.ni = it.nj = 0;
                        it.nk = (int16_t)std::min<int64_t>(tz, p.nz - 1 - k0);
                        work2.push_back({0, it});
                    }
            }
            continue;
        }
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
    if (kernel == 1) {
        // z-march: problems largest first (the block scheduler's order stays balanced:
        // the small problems' items fill the tail), each problem's items together in
        // chunk, row, column order, so tiles that run at the same time are neighbours
        // and the halo rows and planes they share come from L2 (sorting single items
        // by size measured 32% extra DRAM reads on the 256-problem workload)
        std::vector<int64_t> pbytes(nprob);
        for (int q = 0; q < nprob; ++q) pbytes[q] = probs[q].nx * probs[q].ny * probs[q].nz;
        auto by_problem = [&](const std::pair<int64_t, BatchItem> &a, const std::pair<int64_t, BatchItem> &b) {
            const int64_t sa = pbytes[a.second.prob], sb = pbytes[b.second.prob];
            if (sa != sb) return sa > sb;
            return a.second.prob < b.second.prob;
        };
        std::stable_sort(work.begin(), work.end(), by_problem);
        std::stable_sort(work2.begin(), work2.end(), by_problem);
    } else {
        // column march: largest items first, so the persistent CTAs' round-robin
        // hand-out stays balanced (measured 13% faster than the problem order above)
        std::stable_sort(work.begin(), work.end(),
                         [](const std::pair<int64_t, BatchItem> &a, const std::pair<int64_t, BatchItem> &b) {
                             return a.first > b.first;
                         });
    }
    BatchItem *items = (BatchItem *)(base + L.items);
    for (size_t t = 0; t < work.size(); ++t) items[t] = work[t].second;
    BatchItem *items2 = (BatchItem *)(base + L.items2);
    for (size_t t = 0; t < work2.size(); ++t) items2[t] = work2[t].second;
    if (nitems_out) *nitems_out = nitems;
    return PS_OK;
}

int ps_batch_table_fill(void *host_buf, size_t bytes, const ps_problem *probs, int nprob, int dtype,
                        int tile_x, int tile_y, int tile_z, int64_t *nitems_out) {
    return ps_batch_table_fill_ex(host_buf, bytes, probs, nprob, dtype, tile_x, tile_y, tile_z,
                                  PS_BATCH_COLUMN, nitems_out);
}

int ps_batch_table_kernel(const void *host_table) {
    if (!host_table) return fail(PS_ERR_ARG, "host_table is NULL");
    return ((const BatchHeader *)host_table)->kernel;
}

static cudaError_t enqueue_batch(const void *dev_table, const BatchHeader &h, int parity, cudaStream_t s) {
    if (h.kernel == 1) return launch_batch_zmarch(dev_table, h.nitems, h.zmode, parity, s);
    return launch_batch_step(dev_table, parity, h.dtype, s);
}

static int batch_header(const void *host_table, BatchHeader *h) {
    if (!host_table) return fail(PS_ERR_ARG, "host_table is NULL");
    *h = *(const BatchHeader *)host_table;
    PS_TRY(check_dtype(h->dtype));
    if (h->kernel != 0 && h->kernel != 1) return fail(PS_ERR_ARG, "host_table is not a batch table");
    if (h->nitems < 1) return fail(PS_ERR_ARG, "the table has no work items");
    return PS_OK;
}

int ps_diffusion3d_batch_step_ex(const void *dev_table, const void *host_table, int parity, void *stream) {
    if (!dev_table) return fail(PS_ERR_ARG, "dev_table is NULL");
    BatchHeader h;
    PS_TRY(batch_header(host_table, &h));
    if (parity != 0 && parity != 1) return fail(PS_ERR_ARG, "parity %d is not 0 or 1", parity);
    cudaError_t e = enqueue_batch(dev_table, h, parity, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_batch_step");
    return PS_OK;
}

int ps_diffusion3d_batch_step2_ex(const void *dev_table, const void *host_table, int parity, void *stream) {
    if (!dev_table) return fail(PS_ERR_ARG, "dev_table is NULL");
    BatchHeader h;
    PS_TRY(batch_header(host_table, &h));
    if (parity != 0 && parity != 1) return fail(PS_ERR_ARG, "parity %d is not 0 or 1", parity);
    if (h.nitems2 < 1) return fail(PS_ERR_ARG, "the table was not built with PS_BATCH_TEMPORAL2");
    cudaError_t e = launch_batch_zmarch2(dev_table, h.nitems2, h.dtype, parity, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_batch_step2_ex");
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

// nt steps as launches: fused pairs (PS_RUN_TEMPORAL2) then single steps, each
// launch swapping the buffers; an odd pair count would leave the result in the
// wrong buffer, so then one pair runs as two single steps
static cudaError_t enqueue_batch_run(const void *dev_table, const BatchHeader &h, int nt, bool pairs,
                                     cudaStream_t s) {
    int m = pairs ? nt / 2 : 0, r = nt - 2 * m;
    if (m & 1) {
        m -= 1;
        r += 2;
    }
    int launch = 0;
    for (int i = 0; i < m; ++i, ++launch) {
        cudaError_t e = launch_batch_zmarch2(dev_table, h.nitems2, h.dtype, launch & 1, s);
        if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < r; ++i, ++launch) {
        cudaError_t e = enqueue_batch(dev_table, h, launch & 1, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static int batch_run(const void *dev_table, const BatchHeader &h, int nt, unsigned flags, cudaStream_t s) {
    if (nt < 0) return fail(PS_ERR_ARG, "nt = %d < 0", nt);
    if (flags & ~(PS_RUN_GRAPH | PS_RUN_TEMPORAL2)) return fail(PS_ERR_ARG, "unsupported flags 0x%x", flags);
    const bool pairs = (flags & PS_RUN_TEMPORAL2) != 0;
    if (pairs && h.nitems2 < 1)
        return fail(PS_ERR_ARG, "PS_RUN_TEMPORAL2 needs a table built with PS_BATCH_TEMPORAL2");
    if (h.kernel == 0) batch_prepare(h.dtype);
    if (!(flags & PS_RUN_GRAPH)) {
        cudaError_t e = enqueue_batch_run(dev_table, h, nt, pairs, s);
        if (e != cudaSuccess) return cuda_fail(e, "ps_diffusion3d_batch_run");
        return PS_OK;
    }
    // the table's work-item count and kernel are part of the key: the z-march launch
    // size is baked into the graph (a new table may reuse a freed table's address)
    const GraphKey key{current_device(), dev_table, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0, 0.0,
                       0.0, h.nitems, h.zmode, h.kernel, nt, h.dtype, 0x80000000u | (pairs ? 1u : 0u), 0};
    return graph_replay(
        key, [&](cudaStream_t cs) { return enqueue_batch_run(dev_table, h, nt, pairs, cs); },
        "capturing the batch loop", s);
}

int ps_diffusion3d_batch_run_ex(const void *dev_table, const void *host_table, int nt, unsigned flags,
                                void *stream) {
    if (!dev_table) return fail(PS_ERR_ARG, "dev_table is NULL");
    BatchHeader h;
    PS_TRY(batch_header(host_table, &h));
    return batch_run(dev_table, h, nt, flags, (cudaStream_t)stream);
}

int ps_diffusion3d_batch_run(const void *dev_table, int nt, int dtype, unsigned flags,
                             void *stream) {
    if (!dev_table) return fail(PS_ERR_ARG, "dev_table is NULL");
    PS_TRY(check_dtype(dtype));
    BatchHeader h{};
    h.dtype = dtype;
    h.kernel = 0;
    return batch_run(dev_table, h, nt, flags, (cudaStream_t)stream);
}

}  // extern "C"

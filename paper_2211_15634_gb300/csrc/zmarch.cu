// Tiled z-march step kernels fed by TMA over a single grid: CTA (tile, chunk)
// runs the z-march tile body of zmarch_tile.cuh on its x-y tile and z-chunk.
//
// Preconditions (checked by the host launcher, else the plain kernel runs):
// nx*sizeof(elem) is a multiple of 16 (TMA row pitch) and all base pointers
// are 16-byte aligned.
#include <cudaTypedefs.h>


#include <map>
#include <mutex>
#include <tuple>

#include "emu64.cuh"
#include "internal.h"
#include "node.cuh"
#include "pdl.cuh"
#include "tma.cuh"
#include "zmarch.h"
#include "zmarch_tile.cuh"

namespace psd {

__device__ unsigned g_zmarch_error;  // set when an mbarrier wait times out

template <int MODE, int BY, int NST, bool kBnd>
__global__ void __launch_bounds__(32 * BY, 1)
k_zmarch(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmC,
         const __grid_constant__ CUtensorMap tmE, void *__restrict__ T2v, void *__restrict__ E2v,
         const ZParams p) {
    grid_dep_wait();  // the previous step's writes (and its reads of T2) are complete
    grid_dep_launch();
    const int X0 = (int)(blockIdx.x % p.ntx) * (32 * ZTraits<MODE>::PX);
    const int Y0 = (int)(blockIdx.x / p.ntx) * BY;
    const int k0 = 1 + (int)blockIdx.y * p.kchunk;
    const int k1 = (int)min((int64_t)k0 + p.kchunk, p.nz - 1);  // output planes [k0, k1)
    zmarch_tile<MODE, BY, NST, 32, kBnd>(&tmT, &tmC, T2v, E2v, p, X0, Y0, k0, k1, &g_zmarch_error, &tmE);
}

// Failure-path self-test: one CTA waits on an mbarrier that nothing ever arrives on.
// The bounded wait gives up after `polls` polls of at most `ns` nanoseconds each and
// reports through the same device flag as a pipelined kernel's time-out.
__global__ void k_selftest_wait(unsigned polls, unsigned ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool done = false;
    for (unsigned i = 0; i < polls && !done; ++i) done = mbar_try_wait_hint(&bar, 0u, ns);
    if (!done && threadIdx.x == 0) atomicOr(&g_zmarch_error, 1u);
}

cudaError_t launch_selftest_wait(unsigned polls, unsigned ns, cudaStream_t s) {
    k_selftest_wait<<<1, 32, 0, s>>>(polls, ns);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    });
    return fn;
}

bool make_tensor_map_3d(CUtensorMap *m, const void *ptr, int esz, Grid3 g, unsigned bx, unsigned by) {
    return make_tensor_map_3d_pitch(m, ptr, esz, g, g.nx, bx, by);
}

bool make_tensor_map_3d_pitch(CUtensorMap *m, const void *ptr, int esz, Grid3 g, int64_t pitch,
                              unsigned bx, unsigned by) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)(pitch * esz), (cuuint64_t)(pitch * g.ny * esz)};
    const cuuint32_t box[3] = {bx, by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, esz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          3, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool zmarch_supported(Grid3 g, int esz, const void *a, const void *b, const void *c) {
    if ((g.nx * esz) % 16 != 0) return false;
    if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15u) return false;
    if (g.nx > (1LL << 31) - 256 || g.ny > (1LL << 31) - 64 || g.nz > (1LL << 31) - 2) return false;
    return encode_fn() != nullptr;
}

bool step_tma_ok(Grid3 g, int esz, const void *a, const void *b, const void *c) {
    return launch_override(PS_OVERRIDE_STEP_PLAIN) != 1 && zmarch_supported(g, esz, a, b, c);
}

template <int MODE, int BY, int NST, bool kBnd = false>
static cudaError_t launch_zmarch_t(void *T2, const void *T, void *E2, const void *Ein, const void *Ci,
                                   Grid3 g, ZParams p, int kchunk, cudaStream_t s) {
    using E = typename ZTraits<MODE>::E;
    constexpr int PX = ZTraits<MODE>::PX, BX = 32 * PX, W = BX + 2 * PX, H = BY + 2;
    constexpr unsigned TBA = (W * H * sizeof(E) + 127) / 128 * 128;
    constexpr unsigned CBA = (BX * BY * sizeof(E) + 127) / 128 * 128;
    constexpr unsigned EBA = MODE == Z_F32_COMP ? TBA : 0u;
    constexpr size_t smem = NST * (TBA + CBA + EBA) + NST * 8;
    static unsigned attr_gen[64] = {0};
    cudaError_t ae;
    if (!set_smem_attr_once((const void *)k_zmarch<MODE, BY, NST, kBnd>, (int)smem, attr_gen, &ae)) return ae;
    CUtensorMap mT, mC, mE;
    if (!make_tensor_map_3d(&mT, T, sizeof(E), g, W, H) ||
        !make_tensor_map_3d(&mC, Ci, sizeof(E), g, BX, BY))
        return cudaErrorInvalidValue;
    if (MODE == Z_F32_COMP) {
        if (!make_tensor_map_3d(&mE, Ein, sizeof(E), g, W, H)) return cudaErrorInvalidValue;
    } else {
        mE = mT;  // not read
    }
    const int64_t ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY;
    const int64_t tiles = ntx * nty;
    if (kchunk <= 0) {
        // Short chunks keep many CTAs in flight (no wave tail) while consecutive
        // CTAs - neighbouring tiles of one chunk - share their halo planes in L2;
        // each chunk pays two extra planes.  Measured (sweeps at 256^3 and 512^3):
        // FP32 is fastest at 8 planes; FP64 at 8 planes on small grids and flat from
        // 24 to 40 planes at 512^3, so about 64 CTAs per SM between 8 and 32 planes.
        const int64_t target = 64LL * sm_count();
        const int64_t kmax = sizeof(E) == 8 ? 32 : 8;
        int64_t kc = (g.nz - 2) * tiles / target;
        kchunk = (int)(kc < 8 ? 8 : (kc > kmax ? kmax : kc));
    }
    const int64_t gz = (g.nz - 2 + kchunk - 1) / kchunk;
    if (tiles > 0x7fffffffLL || gz > 65535) return cudaErrorInvalidConfiguration;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.pitch = g.nx;
    p.ntx = (int)ntx;
    p.kchunk = kchunk;
    return launch_pdl(k_zmarch<MODE, BY, NST, kBnd>, dim3((unsigned)tiles, (unsigned)gz, 1), dim3(32 * BY), smem,
                      s, mT, mC, mE, T2, E2, p);
}

static ZParams make_params(StepCoef c) {
    ZParams p{};
    p.ek = EmuCoef{emu_const(c.dtlam * c.ax), emu_const(c.dtlam * c.ay), emu_const(c.dtlam * c.az),
                   c.dtlam, c.ax, c.ay, c.az, c.dtlam * c.ax};
    p.fdtlam = (float)c.dtlam;
    p.fax = (float)c.ax;
    p.fay = (float)c.ay;
    p.faz = (float)c.az;
    return p;
}

bool tma_encoder_available() { return encode_fn() != nullptr; }

bool f64_scaled_wide(Grid3 g, const void *T2, const void *T, const void *Ci) {
    if (launch_override(PS_OVERRIDE_F64_PX2) == 1) return false;
    return g.nx % 4 == 0 && ((((uintptr_t)T2 | (uintptr_t)T | (uintptr_t)Ci) & 31u) == 0);
}

ZParams zparams_for(StepCoef c, Grid3 g, int64_t pitch) {
    ZParams p = make_params(c);
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.pitch = pitch;
    return p;
}

// One mode's launch, with the boundary-writing instantiation where asked (the forms
// that state-keeping time loops use; never the two-float step).
template <int MODE, int BY, int NST>
static cudaError_t launch_zmarch_b(void *T2, const void *T, void *E2, const void *Ein, const void *Ci, Grid3 g,
                                   ZParams p, int kchunk, cudaStream_t s, bool write_bnd) {
    if (MODE != Z_F32_COMP && write_bnd)
        return launch_zmarch_t<MODE, BY, NST, MODE != Z_F32_COMP>(T2, T, E2, Ein, Ci, g, p, kchunk, s);
    return launch_zmarch_t<MODE, BY, NST, false>(T2, T, E2, Ein, Ci, g, p, kchunk, s);
}

cudaError_t launch_zmarch(int mode, void *T2, const void *T, void *E2, const void *Ein, const void *Ci,
                          StepCoef c, Grid3 g, cudaStream_t s, bool write_bnd) {
    const ZParams p = make_params(c);
    const int kchunk = launch_override(PS_OVERRIDE_KCHUNK);
    const bool positive = c.dtlam * c.ax > 0 && c.dtlam * c.ay > 0 && c.dtlam * c.az > 0;
    const bool wb = write_bnd;
    switch (mode) {
        case Z_F64_EMU_ISO:
        case Z_F64_EMU_ANISO:
            if (!positive) return launch_zmarch_b<Z_F64_NATIVE, 8, 4>(T2, T, E2, Ein, Ci, g, p, kchunk, s, wb);
            // isotropic grids: fma(Ci*K, S, T), two FP64 ops and the fewest integer ops
            // (measured faster than one DFMA after a 64 x 64-bit high multiply by K)
            if (mode == Z_F64_EMU_ISO)
                return launch_zmarch_b<Z_F64_EMU_ISO_DMUL, 8, 4>(T2, T, E2, Ein, Ci, g, p, kchunk, s, wb);
            return launch_zmarch_b<Z_F64_EMU_ANISO, 8, 4>(T2, T, E2, Ein, Ci, g, p, kchunk, s, wb);
        case Z_F64_NATIVE:
            return launch_zmarch_b<Z_F64_NATIVE, 8, 4>(T2, T, E2, Ein, Ci, g, p, kchunk, s, wb);
        case Z_F64_SCALED:
            // four nodes per thread (4-row tiles, 128 threads) where rows allow 32-byte
            // accesses: measured 2-3% faster at 512^3 and 768^3 than two per thread
            // (8-row tiles of four per thread, at two CTAs per SM, were 15% slower)
            if (f64_scaled_wide(g, T2, T, Ci))
                return launch_zmarch_b<Z_F64_SCALED4, 4, 4>(T2, T, E2, Ein, Ci, g, p, kchunk, s, wb);
            return launch_zmarch_b<Z_F64_SCALED, 8, 4>(T2, T, E2, Ein, Ci, g, p, kchunk, s, wb);
        case Z_F32:
            return launch_zmarch_b<Z_F32, 8, 4>(T2, T, E2, Ein, Ci, g, p, kchunk, s, wb);
        case Z_F32_COMP:
            return launch_zmarch_t<Z_F32_COMP, 8, 4>(T2, T, E2, Ein, Ci, g, p, kchunk, s);
    }
    return cudaErrorInvalidValue;
}

unsigned zmarch_device_error(bool clear) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_zmarch_error, sizeof(v));
    if (clear) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_zmarch_error, &z, sizeof(z));
    }
    return v;
}

}  // namespace psd

// Two time steps per pass (temporal blocking of depth 2) over a single grid: CTA
// (tile, chunk) runs the fused-pair tile body of zmarch2_tile.cuh.
#include <cudaTypedefs.h>


#include "internal.h"
#include "node.cuh"
#include "pdl.cuh"
#include "tma.cuh"
#include "zmarch.h"
#include "zmarch2_tile.cuh"

namespace psd {

__device__ unsigned g_zmarch2_error;  // set when an mbarrier wait times out

// kStates: T1 = step(T) also goes to T1o, and T1o and T2 are written with their x and
// y faces (zmarch2_tile).
template <typename E, int BY, int NT, int NC, bool kStates>
__global__ void __launch_bounds__(32 * BY, Z2Ring<E>::MINB)
k_zmarch2(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmC,
          E *__restrict__ T2, const Z2Params p, E *__restrict__ T1o) {
    grid_dep_wait();  // the previous launch's writes (and its reads of T2) are complete
    grid_dep_launch();
    const int X0 = (int)(blockIdx.x % p.ntx) * (32 * Z2Traits<E>::PX), Y0 = (int)(blockIdx.x / p.ntx) * BY;
    const int k0 = 1 + (int)blockIdx.y * p.kchunk;
    const int k1 = (int)min((int64_t)k0 + p.kchunk, p.nz - 1);  // output planes [k0, k1)
    zmarch2_tile<E, BY, NT, NC, kStates>(&tmT, &tmC, T2, p, X0, Y0, k0, k1, &g_zmarch2_error, T1o);
}

bool zmarch2_supported(Grid3 g, int esz, const void *a, const void *b, const void *c) {
    return zmarch_supported(g, esz, a, b, c);
}

template <typename E, bool kStates = false>
static cudaError_t launch_z2(E *T2, const E *T, const E *Ci, Z2Params p, Grid3 g, cudaStream_t s,
                             E *T1o = nullptr) {
    constexpr int BY = 8, NT = Z2Ring<E>::NT, NC = Z2Ring<E>::NC, PX = Z2Traits<E>::PX,
                  HX = 16 / (int)sizeof(E), BX = 32 * PX, W = BX + 2 * HX;
    constexpr unsigned TBA = (W * (BY + 4) * sizeof(E) + 127) / 128 * 128;
    constexpr unsigned CBA = (W * (BY + 2) * sizeof(E) + 127) / 128 * 128;
    constexpr size_t smem = NT * TBA + (NC + 2) * CBA + (NT + NC) * 8;
    static unsigned attr_gen[64] = {0};
    cudaError_t ae;
    if (!set_smem_attr_once((const void *)k_zmarch2<E, BY, NT, NC, kStates>, (int)smem, attr_gen, &ae)) return ae;
    CUtensorMap mT, mC;
    if (!make_tensor_map_3d(&mT, T, sizeof(E), g, W, BY + 4) ||
        !make_tensor_map_3d(&mC, Ci, sizeof(E), g, W, BY + 2))
        return cudaErrorInvalidValue;
    const int64_t ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY, tiles = ntx * nty;
    int kchunk = launch_override(PS_OVERRIDE_KCHUNK2);
    if (kchunk <= 0) {
        // FP32: one wave when it takes chunks of 24-96 planes - every tile's z-range split
        // into as many chunks as there are CTA slots per tile, all CTAs resident at once
        // (no tail; 256^3: 29 planes, 5.6 against 6.1 ms for 200 states).  Else (and FP64)
        // the prologue costs two extra T1 planes: long chunks, but about three waves.
        const int64_t slots = (int64_t)Z2Ring<E>::MINB * sm_count();
        const int64_t per_tile = tiles > 0 ? slots / tiles : 0;
        const int64_t one_wave = per_tile > 0 ? (g.nz - 2 + per_tile - 1) / per_tile : 0;
        if (sizeof(E) == 4 && one_wave >= 24 && one_wave <= 96) {
            kchunk = (int)one_wave;
        } else {
            const int64_t waves = 3LL * 3 * sm_count();
            const int64_t kc = (g.nz - 2) * tiles / waves;
            kchunk = (int)(kc < 8 ? 8 : (kc > 32 ? 32 : kc));
        }
    }
    const int64_t gz = (g.nz - 2 + kchunk - 1) / kchunk;
    if (tiles > 0x7fffffffLL || gz > 65535) return cudaErrorInvalidConfiguration;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.pitch = g.nx;
    p.ntx = (int)ntx;
    p.kchunk = kchunk;
    return launch_pdl(k_zmarch2<E, BY, NT, NC, kStates>, dim3((unsigned)tiles, (unsigned)gz, 1), dim3(32 * BY), smem,
                      s, mT, mC, T2, p, T1o);
}

cudaError_t launch_step2_f32(float *T2, const float *T, const float *Ci, StepCoef c, Grid3 g,
                             cudaStream_t s) {
    Z2Params p{};
    p.dtlam = (float)c.dtlam;
    p.ax = (float)c.ax;
    p.ay = (float)c.ay;
    p.az = (float)c.az;
    return launch_z2<float>(T2, T, Ci, p, g, s);
}

cudaError_t launch_step2_f64_scaled(double *T2, const double *T, const double *Cs, Grid3 g,
                                    cudaStream_t s) {
    return launch_z2<double>(T2, T, Cs, Z2Params{}, g, s);
}

cudaError_t launch_step2_states_f32(float *T1o, float *T2, const float *T, const float *Ci, StepCoef c,
                                    Grid3 g, cudaStream_t s) {
    Z2Params p{};
    p.dtlam = (float)c.dtlam;
    p.ax = (float)c.ax;
    p.ay = (float)c.ay;
    p.az = (float)c.az;
    return launch_z2<float, true>(T2, T, Ci, p, g, s, T1o);
}

unsigned zmarch2_device_error(bool clear) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_zmarch2_error, sizeof(v));
    if (clear) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_zmarch2_error, &z, sizeof(z));
    }
    return v;
}

}  // namespace psd

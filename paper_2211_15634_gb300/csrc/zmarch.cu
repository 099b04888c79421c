// Tiled z-march step kernels fed by TMA.
//
// A CTA owns one x-y tile of BX x BY nodes (BX = 32 threads * PX nodes per
// thread, one warp per tile row) and a chunk of z-planes.  For every plane a
// single thread issues one TMA box load of the tile plus a one-node halo in
// y and a 16-byte halo in x (so every box starts on a 16-byte boundary) into
// a ring of NST shared-memory stages, together with the box of Ci of the same
// plane (output planes only), both counted on the stage's one mbarrier.  Each
// thread keeps its PX centre values of planes k-1, k, k+1 in registers (the
// z-neighbours) and reads x/y neighbours of plane k from shared memory, so
// every T value is read from HBM once (plus halos that mostly hit in L2).
// T2 is written with 16-byte stores.  Boundary nodes are never written.
//
// Preconditions (checked by the host launcher, else the plain kernel runs):
// nx*sizeof(elem) is a multiple of 16 (TMA row pitch) and all base pointers
// are 16-byte aligned.
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>

#include <map>
#include <mutex>
#include <tuple>

#include "emu64.cuh"
#include "internal.h"
#include "node.cuh"
#include "tma.cuh"
#include "zmarch.h"

namespace psd {

__device__ unsigned g_zmarch_error;  // set when an mbarrier wait times out

template <int MODE>
struct ZTraits;
template <>
struct ZTraits<Z_F64_EMU_ISO> {
    using E = double;
    using V = double2;
    static constexpr int PX = 2;
};
template <>
struct ZTraits<Z_F64_EMU_ANISO> : ZTraits<Z_F64_EMU_ISO> {};
template <>
struct ZTraits<Z_F64_NATIVE> : ZTraits<Z_F64_EMU_ISO> {};
template <>
struct ZTraits<Z_F64_EMU_ISO_DMUL> : ZTraits<Z_F64_EMU_ISO> {};
template <>
struct ZTraits<Z_F64_SCALED> : ZTraits<Z_F64_EMU_ISO> {};
template <>
struct ZTraits<Z_F32> {
    using E = float;
    using V = float4;
    static constexpr int PX = 4;
};
template <>
struct ZTraits<Z_F32_COMP> : ZTraits<Z_F32> {};

template <typename V, typename E>
__device__ __forceinline__ E vget(const V &v, int i) {
    return reinterpret_cast<const E *>(&v)[i];
}

template <int MODE, int BY, int NST>
__global__ void __launch_bounds__(32 * BY, 1)
k_zmarch(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmC,
         void *__restrict__ T2v, void *__restrict__ compv, const ZParams p) {
    using Tr = ZTraits<MODE>;
    using E = typename Tr::E;
    using V = typename Tr::V;
    constexpr int PX = Tr::PX, HX = PX, BX = 32 * PX, W = BX + 2 * HX, H = BY + 2;
    constexpr unsigned TB = W * H * sizeof(E), CB = BX * BY * sizeof(E);
    constexpr unsigned TBA = (TB + 127) / 128 * 128, CBA = (CB + 127) / 128 * 128;
    extern __shared__ __align__(128) unsigned char smem[];
    E *sT = (E *)smem;
    E *sC = (E *)(smem + NST * TBA);
    uint64_t *bar = (uint64_t *)(smem + NST * (TBA + CBA));
    __shared__ int s_abort;

    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int X0 = (int)(blockIdx.x % p.ntx) * BX, Y0 = (int)(blockIdx.x / p.ntx) * BY;
    const int k0 = 1 + (int)blockIdx.y * p.kchunk;
    const int k1 = (int)min((int64_t)k0 + p.kchunk, p.nz - 1);  // output planes [k0, k1)

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Plane q (q = k0-1 .. k1) lives in stage (q - (k0-1)) % NST: its T box, and its Ci
    // box when it is an output plane, counted on the stage's one mbarrier.
    constexpr unsigned TSTRIDE = TBA / sizeof(E), CSTRIDE = CBA / sizeof(E);
    auto issue = [&](int s, int q) {
        const bool ci = q >= k0 && q < k1;
        mbar_expect_tx(&bar[s], TB + (ci ? CB : 0u));
        tma_load_3d(sT + s * TSTRIDE, &tmT, &bar[s], X0 - HX, Y0 - 1, q);
        if (ci) tma_load_3d(sC + s * CSTRIDE, &tmC, &bar[s], X0, Y0, q);
    };
    if (threadIdx.x == 0)
        for (int s = 0; s < NST; ++s)
            if (k0 - 1 + s <= k1) issue(s, k0 - 1 + s);
    // bit s of tpar is the parity of the next completion of stage s
    unsigned tpar = 0u;
    auto tnext = [](int s) { return s + 1 == NST ? 0 : s + 1; };
    auto acquire = [&](int s) -> bool {
        const unsigned ph = (tpar >> s) & 1u;
        tpar ^= 1u << s;
        return mbar_wait(&bar[s], ph);
    };
    // After a timed-out wait: bounded waits for the copies of the last NST planes issued
    // (up to plane q_iss), so that no TMA write lands after the CTA exits.
    auto drain = [&](int q_iss) {
        for (int q = max(k0 - 1, q_iss - NST + 1); q <= q_iss; ++q) {
            const int i = q - (k0 - 1);
            mbar_wait(&bar[i % NST], (unsigned)(i / NST) & 1u);
        }
    };

    const int row = ty + 1, col = HX + lane * PX;
    bool ok = acquire(0);
    V qm = *(const V *)(sT + row * W + col);
    ok = acquire(1 % NST) && ok;
    V qc = *(const V *)(sT + (1 % NST) * TSTRIDE + row * W + col);
    if (!ok) {
        s_abort = 1;
        atomicOr(&g_zmarch_error, 1u);
    }
    __syncthreads();
    if (s_abort) {
        drain(min(k0 - 2 + NST, k1));
        return;
    }
    if (threadIdx.x == 0 && k0 - 1 + NST <= k1) issue(0, k0 - 1 + NST);  // stage 0 held plane k0-1

    const int gy = Y0 + ty;
    const int gx0 = X0 + lane * PX;
    const bool row_ok = gy >= 1 && gy <= p.ny - 2;
    bool all_x = gx0 >= 1 && gx0 + PX - 1 <= p.nx - 2;
    E *__restrict__ T2 = (E *)T2v;
    E *__restrict__ comp = (E *)compv;
    int sk = 1 % NST;  // stage of plane k
    const int64_t plane = p.nx * p.ny;
    int64_t base = (int64_t)gx0 + p.nx * ((int64_t)gy + p.ny * (int64_t)k0);  // own nodes, plane k

    for (int k = k0; k < k1; ++k, base += plane) {
        const int sk1 = tnext(sk);
        ok = acquire(sk1);  // plane k+1 (plane k, with its Ci, was acquired before)
        const E *Tk = sT + sk * TSTRIDE;
        const V qn = *(const V *)(sT + sk1 * TSTRIDE + row * W + col);
        const E left = Tk[row * W + col - 1], right = Tk[row * W + col + PX];
        const V up = *(const V *)(Tk + (row - 1) * W + col);
        const V dn = *(const V *)(Tk + (row + 1) * W + col);
        const V civ = *(const V *)(sC + sk * CSTRIDE + ty * BX + lane * PX);

        if (row_ok) {
            V cv{};
            if constexpr (MODE == Z_F32_COMP) {
                if (all_x) cv = *(const V *)(comp + base);
                else
#pragma unroll
                    for (int i = 0; i < PX; ++i) {
                        const int gx = gx0 + i;
                        reinterpret_cast<E *>(&cv)[i] = (gx >= 1 && gx <= p.nx - 2) ? comp[base + i] : E(0);
                    }
            }
            V out;
            if constexpr (MODE == Z_F64_EMU_ISO || MODE == Z_F64_EMU_ANISO ||
                          MODE == Z_F64_EMU_ISO_DMUL || MODE == Z_F64_SCALED) {
                constexpr bool kIso = MODE != Z_F64_EMU_ANISO;
                constexpr bool kDmul = MODE == Z_F64_EMU_ISO_DMUL;
                constexpr bool kScaled = MODE == Z_F64_SCALED;
                unsigned long long c[PX], xm[PX], xp[PX], ym[PX], yp[PX], zm[PX], zp[PX];
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    c[i] = dbits((double)vget<V, E>(qc, i));
                    xm[i] = dbits((double)(i == 0 ? left : vget<V, E>(qc, i - 1)));
                    xp[i] = dbits((double)(i == PX - 1 ? right : vget<V, E>(qc, i + 1)));
                    ym[i] = dbits((double)vget<V, E>(up, i));
                    yp[i] = dbits((double)vget<V, E>(dn, i));
                    zm[i] = dbits((double)vget<V, E>(qm, i));
                    zp[i] = dbits((double)vget<V, E>(qn, i));
                }
                // one check over the 5*PX + 2 distinct values of this thread's PX stencils
                unsigned hw[5 * PX + 1];
                hw[0] = (unsigned)(xm[0] >> 32);
                hw[1] = (unsigned)(xp[PX - 1] >> 32);
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    hw[2 + 4 * i] = (unsigned)(ym[i] >> 32);
                    hw[3 + 4 * i] = (unsigned)(yp[i] >> 32);
                    hw[4 + 4 * i] = (unsigned)(zm[i] >> 32);
                    hw[5 + 4 * i] = (unsigned)(zp[i] >> 32);
                }
#pragma unroll
                for (int i = 1; i < PX; ++i) hw[1 + 4 * PX + i] = (unsigned)(c[i] >> 32);
                const unsigned hc = (unsigned)(c[0] >> 32);
                if (!all_x) {
                    // Lanes at the grid's x edges: a node that is not stored (x = 0,
                    // x = nx-1, or past the grid where TMA filled zeros) must not
                    // send the warp to the general path, so its private values are
                    // replaced by the reference word.
                    bool use[PX];
#pragma unroll
                    for (int i = 0; i < PX; ++i) use[i] = gx0 + i >= 1 && gx0 + i <= p.nx - 2;
                    if (!use[0]) hw[0] = hc;       // left: x-neighbour of node 0 only
                    if (!use[PX - 1]) hw[1] = hc;  // right: x-neighbour of the last node only
#pragma unroll
                    for (int i = 0; i < PX; ++i) {
                        if (!use[i]) {  // y and z neighbours belong to node i alone
                            hw[2 + 4 * i] = hc;
                            hw[3 + 4 * i] = hc;
                            hw[4 + 4 * i] = hc;
                            hw[5 + 4 * i] = hc;
                        }
                    }
#pragma unroll
                    for (int i = 1; i < PX; ++i) {  // centre i is also node i-1's and i+1's x-neighbour
                        const bool need = use[i] || use[i - 1] || (i + 1 < PX && use[i + 1]);
                        if (!need) hw[1 + 4 * PX + i] = hc;
                    }
                }
                const bool fast = emu_same_binade_hi(hw, hc);
                // warp-uniform branch: smooth fields take the short fast path
                if (__all_sync(0xffffffffu, fast)) {
#pragma unroll
                    for (int i = 0; i < PX; ++i) {
                        const double ci = (double)vget<V, E>(civ, i);
                        if constexpr (kScaled)
                            reinterpret_cast<E *>(&out)[i] =
                                emu_fast_node_scaled(c[i], xm[i], xp[i], ym[i], yp[i], zm[i], zp[i], ci);
                        else
                            reinterpret_cast<E *>(&out)[i] = emu_fast_node<kIso, kDmul>(
                                c[i], xm[i], xp[i], ym[i], yp[i], zm[i], zp[i], ci, p.ek);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < PX; ++i) {
                        const double ci = (double)vget<V, E>(civ, i);
                        if constexpr (kScaled)
                            reinterpret_cast<E *>(&out)[i] =
                                emu_step_node_scaled(c[i], xm[i], xp[i], ym[i], yp[i], zm[i], zp[i], ci);
                        else
                            reinterpret_cast<E *>(&out)[i] = emu_step_node<kIso, kDmul>(
                                c[i], xm[i], xp[i], ym[i], yp[i], zm[i], zp[i], ci, p.ek);
                    }
                }
            } else
#pragma unroll
            for (int i = 0; i < PX; ++i) {
                const E c = vget<V, E>(qc, i);
                const E xm = i == 0 ? left : vget<V, E>(qc, i - 1);
                const E xp = i == PX - 1 ? right : vget<V, E>(qc, i + 1);
                const E ym = vget<V, E>(up, i), yp = vget<V, E>(dn, i);
                const E zm = vget<V, E>(qm, i), zp = vget<V, E>(qn, i);
                const E ci = vget<V, E>(civ, i);
                E r;
                if constexpr (MODE == Z_F64_NATIVE) {
                    const double d2x = (xp - c) - (c - xm), d2y = (yp - c) - (c - ym);
                    const double d2z = (zp - c) - (c - zm);
                    r = c + p.ek.dtlam * (ci * ((d2x * p.ek.ax + d2y * p.ek.ay) + d2z * p.ek.az));
                } else if constexpr (MODE == Z_F32) {
                    r = f32_node(c, xm, xp, ym, yp, zm, zp, ci, p.fdtlam, p.fax, p.fay, p.faz);
                } else {
                    const float d2x = (xp - c) - (c - xm), d2y = (yp - c) - (c - ym);
                    const float d2z = (zp - c) - (c - zm);
                    const float lap = (d2x * p.fax + d2y * p.fay) + d2z * p.faz;
                    {
                        const float delta = p.fdtlam * (ci * lap);
                        const float yv = delta - vget<V, E>(cv, i);
                        const float t = c + yv;
                        reinterpret_cast<E *>(&cv)[i] = (t - c) - yv;
                        r = t;
                    }
                }
                reinterpret_cast<E *>(&out)[i] = r;
            }
            if (all_x) {
                *(V *)(T2 + base) = out;
                if constexpr (MODE == Z_F32_COMP) *(V *)(comp + base) = cv;
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i) {
                    const int gx = gx0 + i;
                    if (gx >= 1 && gx <= p.nx - 2) {
                        T2[base + i] = vget<V, E>(out, i);
                        if constexpr (MODE == Z_F32_COMP) comp[base + i] = vget<V, E>(cv, i);
                    }
                }
            }
        }
        if (!ok) {
            s_abort = 1;
            atomicOr(&g_zmarch_error, 1u);
        }
        __syncthreads();  // every thread is done with plane k's stage (T and Ci)
        if (s_abort) {
            drain(min(k - 1 + NST, k1));
            return;
        }
        if (threadIdx.x == 0 && k + NST <= k1) issue(sk, k + NST);  // plane k's stage
        sk = sk1;
        qm = qc;
        qc = qn;
    }
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
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)(g.nx * esz), (cuuint64_t)(g.nx * g.ny * esz)};
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

template <int MODE, int BY, int NST>
static cudaError_t launch_zmarch_t(void *T2, const void *T, void *comp, const void *Ci, Grid3 g,
                                   ZParams p, int kchunk, cudaStream_t s) {
    using E = typename ZTraits<MODE>::E;
    constexpr int PX = ZTraits<MODE>::PX, BX = 32 * PX, W = BX + 2 * PX, H = BY + 2;
    constexpr unsigned TBA = (W * H * sizeof(E) + 127) / 128 * 128;
    constexpr unsigned CBA = (BX * BY * sizeof(E) + 127) / 128 * 128;
    constexpr size_t smem = NST * (TBA + CBA) + NST * 8;
    static bool attr_done[64] = {false};
    const int dev = current_device();
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_zmarch<MODE, BY, NST>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    CUtensorMap mT, mC;
    if (!make_tensor_map_3d(&mT, T, sizeof(E), g, W, H) ||
        !make_tensor_map_3d(&mC, Ci, sizeof(E), g, BX, BY))
        return cudaErrorInvalidValue;
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
    p.ntx = (int)ntx;
    p.kchunk = kchunk;
    k_zmarch<MODE, BY, NST><<<dim3((unsigned)tiles, (unsigned)gz, 1), 32 * BY, smem, s>>>(
        mT, mC, T2, comp, p);
    return cudaGetLastError();
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

static int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return v ? atoi(v) : dflt;
}

cudaError_t launch_zmarch(int mode, void *T2, const void *T, void *comp, const void *Ci, StepCoef c,
                          Grid3 g, cudaStream_t s) {
    const ZParams p = make_params(c);
    const int kchunk = env_int("PS_KCHUNK", 0);
    const bool positive = c.dtlam * c.ax > 0 && c.dtlam * c.ay > 0 && c.dtlam * c.az > 0;
    // Isotropic FP64 grids default to fma(Ci*K, S, T) (two FP64 ops, fewest
    // integer ops: measured fastest).  PS_F64_VARIANT selects an alternative
    // for measurements: "umul" = one DFMA plus a 64-bit high multiply,
    // "by16" = 64 x 16 tiles.
    const char *var = getenv("PS_F64_VARIANT");
    const bool dmul = !(var && (strcmp(var, "umul") == 0 || strcmp(var, "by16") == 0));
    const bool by16 = var && strcmp(var, "by16") == 0;
    switch (mode) {
        case Z_F64_EMU_ISO:
        case Z_F64_EMU_ANISO:
            if (!positive) return launch_zmarch_t<Z_F64_NATIVE, 8, 4>(T2, T, comp, Ci, g, p, kchunk, s);
            if (mode == Z_F64_EMU_ISO) {
                if (dmul)
                    return launch_zmarch_t<Z_F64_EMU_ISO_DMUL, 8, 4>(T2, T, comp, Ci, g, p, kchunk, s);
                if (by16)
                    return launch_zmarch_t<Z_F64_EMU_ISO, 16, 4>(T2, T, comp, Ci, g, p, kchunk, s);
                return launch_zmarch_t<Z_F64_EMU_ISO, 8, 4>(T2, T, comp, Ci, g, p, kchunk, s);
            }
            return launch_zmarch_t<Z_F64_EMU_ANISO, 8, 4>(T2, T, comp, Ci, g, p, kchunk, s);
        case Z_F64_NATIVE:
            return launch_zmarch_t<Z_F64_NATIVE, 8, 4>(T2, T, comp, Ci, g, p, kchunk, s);
        case Z_F64_SCALED:
            return launch_zmarch_t<Z_F64_SCALED, 8, 4>(T2, T, comp, Ci, g, p, kchunk, s);
        case Z_F32:
            return launch_zmarch_t<Z_F32, 8, 4>(T2, T, comp, Ci, g, p, kchunk, s);
        case Z_F32_COMP:
            return launch_zmarch_t<Z_F32_COMP, 8, 4>(T2, T, comp, Ci, g, p, kchunk, s);
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

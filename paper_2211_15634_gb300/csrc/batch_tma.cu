// Batched step as a TMA-fed z-march: one launch per step, one CTA per work item.
//
// The table holds, besides the header, problem records and work list of the
// column kernel (batch.cu), the step parameters of every problem and six
// tensor maps per problem (T and T2 with the halo box, Ci with the tile box,
// for each of the two tile shapes), encoded on the host over the problem's own
// row pitch.  Work item (problem, X0, Y0, k0, nk, kind) is an x-y tile at
// (X0, Y0) (boundary included, like the single-grid tiles) and output planes
// [k0, k0+nk): kind 0 the single-grid tile (32 lanes x PX nodes wide, 8 rows),
// kind 1 a narrow one (16 lanes x PX wide, 16 rows, two rows per warp) that
// closes a row of tiles when at most half a wide tile of columns is left -
// batch grids are small, and a wide last tile would leave up to half its lanes
// idle.  CTA b runs item b with the z-march tile body of the single-grid kernel
// (zmarch_tile.cuh), so every problem is stepped by the very arithmetic of its
// own single run.  The work list is static; a captured graph replays the same
// launches every time.
//
// Requirements (checked when the table is built): every row pitch times the
// element size is a multiple of 16 bytes and every base pointer is 16-byte
// aligned (padded rows, see ps_problem.pitch); FP64 problems on Ci as given
// have equal spacings and a positive step coefficient; FP64 problems on the
// pre-scaled coefficient (PS_BATCH_CI_SCALED) have equal spacings.
#include <cudaTypedefs.h>

#include "internal.h"
#include "zmarch.h"
#include "zmarch2_tile.cuh"
#include "zmarch_tile.cuh"

namespace psd {

__device__ unsigned g_batchz_error;  // set when an mbarrier wait times out

// tile shapes: wide = 32 lanes per row x 8 rows, narrow = 16 lanes per row x 16 rows
constexpr int kBZ_NST = 4, kBZ_WIDE_BY = 8, kBZ_NARROW_BY = 16;

// resident CTAs per SM the registers are sized for: Ci as given (two FP64 products
// per node and the emulation constants) spills at 64 registers, so 3 CTAs there
template <int MODE>
struct BZOcc {
    static constexpr int min_blocks = MODE == Z_F64_EMU_ISO_DMUL ? 3 : 4;
};

template <int MODE>
__global__ void __launch_bounds__(256, BZOcc<MODE>::min_blocks)
k_batch_zmarch(const char *__restrict__ table, int parity) {
    const BatchHeader *h = (const BatchHeader *)table;
    const BatchItem item = ((const BatchItem *)(table + h->items_offset))[blockIdx.x];
    __shared__ ZParams s_p;
    if (threadIdx.x == 0) s_p = ((const ZParams *)(table + h->zparams_offset))[item.prob];
    __syncthreads();
    const BatchProblem *P = (const BatchProblem *)(table + h->problems_offset) + item.prob;
    const CUtensorMap *maps =
        (const CUtensorMap *)(table + h->maps_offset) + kBatchZmarchMaps * item.prob;
    void *out = parity ? P->T : P->T2;
    if (item.kind == 0)  // CTA-uniform
        zmarch_tile<MODE, kBZ_WIDE_BY, kBZ_NST, 32>(maps + (parity ? 1 : 0), maps + 2, out, nullptr, s_p,
                                                    item.i0, item.j0, item.k0, item.k0 + item.nk,
                                                    &g_batchz_error);
    else
        zmarch_tile<MODE, kBZ_NARROW_BY, kBZ_NST, 16>(maps + 3 + (parity ? 1 : 0), maps + 5, out, nullptr,
                                                      s_p, item.i0, item.j0, item.k0, item.k0 + item.nk,
                                                      &g_batchz_error);
}

int64_t batch_zmarch_xy_tiles(int dtype, int64_t nx, int64_t ny, BatchItem *out) {
    const int64_t wide = dtype == PS_F64 ? 64 : 128, narrow = wide / 2;
    int64_t n = 0;
    // interior columns 1 .. nx-2 from tile origins 0, wide, 2*wide, ...: the last
    // origin takes a narrow tile when at most `narrow` columns are left
    for (int64_t x0 = 0; x0 < nx - 1;) {
        const bool nar = nx - 1 - x0 <= narrow;
        const int64_t by = nar ? kBZ_NARROW_BY : kBZ_WIDE_BY;
        for (int64_t y0 = 0; y0 < ny - 1; y0 += by, ++n)
            if (out) {
                out[n].i0 = (int32_t)x0;
                out[n].j0 = (int32_t)y0;
                out[n].kind = nar ? 1 : 0;
            }
        x0 += nar ? narrow : wide;
    }
    return n;
}

// Fused step pairs (temporal blocking of depth 2): one CTA per item of the second work
// list, the fused-pair tile body of the single-grid kernel (zmarch2_tile.cuh).
template <typename E>
__global__ void __launch_bounds__(256, Z2Ring<E>::MINB)
k_batch_zmarch2(const char *__restrict__ table, int parity) {
    const BatchHeader *h = (const BatchHeader *)table;
    const BatchItem item = ((const BatchItem *)(table + h->items2_offset))[blockIdx.x];
    __shared__ Z2Params s_p;
    if (threadIdx.x == 0) s_p = ((const Z2Params *)(table + h->z2params_offset))[item.prob];
    __syncthreads();
    const BatchProblem *P = (const BatchProblem *)(table + h->problems_offset) + item.prob;
    const CUtensorMap *maps =
        (const CUtensorMap *)(table + h->maps_offset) + kBatchZmarchMaps * item.prob + 6;
    E *out = (E *)(parity ? P->T : P->T2);
    zmarch2_tile<E, 8, Z2Ring<E>::NT, Z2Ring<E>::NC>(maps + (parity ? 1 : 0), maps + 2, out, s_p, item.i0,
                                                     item.j0, item.k0, item.k0 + item.nk,
                                                     &g_batchz_error);
}

int64_t batch_zmarch2_xy_tiles(int dtype, int64_t nx, int64_t ny, BatchItem *out) {
    const int64_t bx = dtype == PS_F64 ? 64 : 128, by = 8;
    int64_t n = 0;
    for (int64_t y0 = 0; y0 < ny - 1; y0 += by)
        for (int64_t x0 = 0; x0 < nx - 1; x0 += bx, ++n)
            if (out) {
                out[n].i0 = (int32_t)x0;
                out[n].j0 = (int32_t)y0;
                out[n].kind = 2;
            }
    return n;
}

size_t batch_z2params_bytes() { return sizeof(Z2Params); }

bool batch_zmarch_fill(void *zparams_dst, void *z2params_dst, void *maps_dst, const BatchProblem &r,
                       StepCoef c, int dtype) {
    const int esz = dtype == PS_F64 ? 8 : 4;
    const int px = dtype == PS_F64 ? 2 : 4;
    const Grid3 g{r.nx, r.ny, r.nz};
    ZParams zp = zparams_for(c, g, r.pitch);
    zp.kchunk = 0;
    zp.ntx = 0;
    *(ZParams *)zparams_dst = zp;
    CUtensorMap *m = (CUtensorMap *)maps_dst;
    bool ok = true;
    for (int v = 0; v < 2; ++v) {
        const int lpr = v == 0 ? 32 : 16, by = v == 0 ? kBZ_WIDE_BY : kBZ_NARROW_BY, bx = lpr * px;
        const unsigned W = (unsigned)(bx + 2 * px), H = (unsigned)(by + 2);
        ok = ok && make_tensor_map_3d_pitch(&m[3 * v + 0], r.T, esz, g, r.pitch, W, H) &&
             make_tensor_map_3d_pitch(&m[3 * v + 1], r.T2, esz, g, r.pitch, W, H) &&
             make_tensor_map_3d_pitch(&m[3 * v + 2], r.Ci, esz, g, r.pitch, (unsigned)bx, (unsigned)by);
    }
    // fused pairs: T box with a 2-row y halo, Ci box with a 1-row one, both 16-byte x halos
    Z2Params z2{};
    z2.nx = r.nx;
    z2.ny = r.ny;
    z2.nz = r.nz;
    z2.pitch = r.pitch;
    z2.dtlam = (float)c.dtlam;
    z2.ax = (float)c.ax;
    z2.ay = (float)c.ay;
    z2.az = (float)c.az;
    *(Z2Params *)z2params_dst = z2;
    const unsigned W2 = (unsigned)(32 * px + 2 * (16 / esz));
    ok = ok && make_tensor_map_3d_pitch(&m[6], r.T, esz, g, r.pitch, W2, 12) &&
         make_tensor_map_3d_pitch(&m[7], r.T2, esz, g, r.pitch, W2, 12) &&
         make_tensor_map_3d_pitch(&m[8], r.Ci, esz, g, r.pitch, W2, 10);
    return ok;
}

template <typename E, int PX, int LPR, int BY>
constexpr size_t bz_smem() {
    constexpr int BX = LPR * PX, W = BX + 2 * PX, H = BY + 2;
    constexpr unsigned TBA = (W * H * sizeof(E) + 127) / 128 * 128;
    constexpr unsigned CBA = (BX * BY * sizeof(E) + 127) / 128 * 128;
    return kBZ_NST * (TBA + CBA) + kBZ_NST * 8;
}

template <int MODE>
static cudaError_t launch_bz_t(const void *dev_table, int64_t nitems, int parity, cudaStream_t s) {
    using E = typename ZTraits<MODE>::E;
    constexpr int PX = ZTraits<MODE>::PX;
    constexpr size_t sw = bz_smem<E, PX, 32, kBZ_WIDE_BY>(), sn = bz_smem<E, PX, 16, kBZ_NARROW_BY>();
    constexpr size_t smem = sw > sn ? sw : sn;
    static unsigned attr_gen[64] = {0};
    cudaError_t ae;
    if (!set_smem_attr_once((const void *)k_batch_zmarch<MODE>, (int)smem, attr_gen, &ae)) return ae;
    if (nitems < 1 || nitems > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_batch_zmarch<MODE><<<(unsigned)nitems, 256, smem, s>>>((const char *)dev_table, parity);
    return cudaGetLastError();
}

cudaError_t launch_batch_zmarch(const void *dev_table, int64_t nitems, int zmode, int parity,
                                cudaStream_t s) {
    switch (zmode) {
        case Z_F32: return launch_bz_t<Z_F32>(dev_table, nitems, parity, s);
        case Z_F64_EMU_ISO_DMUL: return launch_bz_t<Z_F64_EMU_ISO_DMUL>(dev_table, nitems, parity, s);
        case Z_F64_SCALED: return launch_bz_t<Z_F64_SCALED>(dev_table, nitems, parity, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename E>
static cudaError_t launch_bz2_t(const void *dev_table, int64_t nitems2, int parity, cudaStream_t s) {
    constexpr int BY = 8, NT = Z2Ring<E>::NT, NC = Z2Ring<E>::NC, PX = Z2Traits<E>::PX,
                  HX = 16 / (int)sizeof(E), BX = 32 * PX, W = BX + 2 * HX;
    constexpr unsigned TBA = (W * (BY + 4) * sizeof(E) + 127) / 128 * 128;
    constexpr unsigned CBA = (W * (BY + 2) * sizeof(E) + 127) / 128 * 128;
    constexpr size_t smem = NT * TBA + (NC + 2) * CBA + (NT + NC) * 8;
    static unsigned attr_gen[64] = {0};
    cudaError_t ae;
    if (!set_smem_attr_once((const void *)k_batch_zmarch2<E>, (int)smem, attr_gen, &ae)) return ae;
    if (nitems2 < 1 || nitems2 > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_batch_zmarch2<E><<<(unsigned)nitems2, 32 * BY, smem, s>>>((const char *)dev_table, parity);
    return cudaGetLastError();
}

cudaError_t launch_batch_zmarch2(const void *dev_table, int64_t nitems2, int dtype, int parity,
                                 cudaStream_t s) {
    if (dtype == PS_F64) return launch_bz2_t<double>(dev_table, nitems2, parity, s);
    return launch_bz2_t<float>(dev_table, nitems2, parity, s);
}

unsigned batch_zmarch_device_error(bool clear) {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_batchz_error, sizeof(v));
    if (clear) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_batchz_error, &z, sizeof(z));
    }
    return v;
}

}  // namespace psd

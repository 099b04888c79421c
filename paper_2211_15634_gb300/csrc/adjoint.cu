// Adjoint (transposed) step kernels.
//
// The forward step is T_{t+1} = T_t + diag(dt*lam*Ci on interior) * Lap(T_t)
// with identity rows on the boundary, so for ybar = dL/dT_{t+1}:
//   w[q]      = dt*lam*Ci[q]*ybar[q] at interior q, 0 elsewhere (and outside),
//   Tbar[p]   = ybar[p] + sum_d (w[p-e_d] - 2 w[p] + w[p+e_d]) * _d^2  (all p),
//   Cibar[q] += dt*lam*ybar[q]*Lap(T_t)[q]                             (interior q).

#include "internal.h"
#include "stencil_basic.cuh"
#include "zmarch.h"

namespace psd {

template <typename F>
__device__ __forceinline__ F w_at(const F *__restrict__ ybar, const F *__restrict__ Ci, F dtlam,
                                  int64_t i, int64_t j, int64_t k, int64_t nx, int64_t ny,
                                  int64_t nz) {
    if (i < 1 || i > nx - 2 || j < 1 || j > ny - 2 || k < 1 || k > nz - 2) return F(0);
    const int64_t q = i + nx * (j + ny * k);
    return dtlam * (Ci[q] * ybar[q]);
}

// One thread per (i, j) column of the whole grid (boundary included),
// marching along z through [k0, k1).
template <typename F>
__global__ void __launch_bounds__(256)
k_adjoint_basic(F *__restrict__ Tbar, F *__restrict__ Cibar, const F *__restrict__ ybar,
                const F *__restrict__ T, const F *__restrict__ Ci, CoefT<F> c, int64_t nx,
                int64_t ny, int64_t nz, int kchunk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i > nx - 1 || j > ny - 1) return;
    const int64_t k0 = (int64_t)blockIdx.z * kchunk;
    const int64_t k1 = k0 + kchunk < nz ? k0 + kchunk : nz;
    if (k0 >= k1) return;
    const int64_t sy = nx, sz = nx * ny;
    const bool in_xy = i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2;
    F wm = w_at(ybar, Ci, c.dtlam, i, j, k0 - 1, nx, ny, nz);
    F wc = w_at(ybar, Ci, c.dtlam, i, j, k0, nx, ny, nz);
    for (int64_t k = k0; k < k1; ++k) {
        const int64_t p = i + sy * (j + ny * k);
        const F wp = w_at(ybar, Ci, c.dtlam, i, j, k + 1, nx, ny, nz);
        const F d2x = (w_at(ybar, Ci, c.dtlam, i + 1, j, k, nx, ny, nz) - wc) -
                      (wc - w_at(ybar, Ci, c.dtlam, i - 1, j, k, nx, ny, nz));
        const F d2y = (w_at(ybar, Ci, c.dtlam, i, j + 1, k, nx, ny, nz) - wc) -
                      (wc - w_at(ybar, Ci, c.dtlam, i, j - 1, k, nx, ny, nz));
        const F d2z = (wp - wc) - (wc - wm);
        const F yb = ybar[p];
        Tbar[p] = yb + ((d2x * c.ax + d2y * c.ay) + d2z * c.az);
        if (in_xy && k >= 1 && k <= nz - 2) {
            const F tc = T[p];
            const F t2x = (T[p + 1] - tc) - (tc - T[p - 1]);
            const F t2y = (T[p + sy] - tc) - (tc - T[p - sy]);
            const F t2z = (T[p + sz] - tc) - (tc - T[p - sz]);
            const F lap = (t2x * c.ax + t2y * c.ay) + t2z * c.az;
            Cibar[p] += c.dtlam * (yb * lap);
        }
        wm = wc;
        wc = wp;
    }
}

template <typename F>
static cudaError_t launch_adjoint_basic(F *Tbar, F *Cibar, const F *ybar, const F *T, const F *Ci,
                                        CoefT<F> c, Grid3 g, cudaStream_t s) {
    const dim3 block(32, 8, 1);
    const int64_t gx = (g.nx + block.x - 1) / block.x, gy = (g.ny + block.y - 1) / block.y;
    int64_t want = (8LL * sm_count() + gx * gy - 1) / (gx * gy);
    int64_t kchunk = (g.nz + want - 1) / want;
    if (kchunk < 16) kchunk = 16;
    const int64_t gz = (g.nz + kchunk - 1) / kchunk;
    if (gx > 0x7fffffff || gy > 65535 || gz > 65535) return cudaErrorInvalidConfiguration;
    k_adjoint_basic<F><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), block, 0, s>>>(
        Tbar, Cibar, ybar, T, Ci, c, g.nx, g.ny, g.nz, (int)kchunk);
    return cudaGetLastError();
}

// Pre-scaled coefficient (FP64, equal spacings): Ci holds Cs = dt*lam*_d^2*Ci,
//   w = Cs*ybar (interior), Tbar = ybar + L(w), Csbar += ybar*L(T)  (interior),
// with L(A) = sum of the six neighbours minus six times the centre.
__global__ void __launch_bounds__(256)
k_adjoint_basic_scaled(double *__restrict__ Tbar, double *__restrict__ Csbar,
                       const double *__restrict__ ybar, const double *__restrict__ T,
                       const double *__restrict__ Cs, int64_t nx, int64_t ny, int64_t nz, int kchunk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i > nx - 1 || j > ny - 1) return;
    const int64_t k0 = (int64_t)blockIdx.z * kchunk;
    const int64_t k1 = k0 + kchunk < nz ? k0 + kchunk : nz;
    if (k0 >= k1) return;
    const int64_t sy = nx, sz = nx * ny;
    const bool in_xy = i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2;
    auto w = [&](int64_t a, int64_t b, int64_t c) -> double {
        return w_at<double>(ybar, Cs, 1.0, a, b, c, nx, ny, nz);
    };
    double wm = w(i, j, k0 - 1), wc = w(i, j, k0);
    for (int64_t k = k0; k < k1; ++k) {
        const int64_t p = i + sy * (j + ny * k);
        const double wp = w(i, j, k + 1);
        const double Lw = ((w(i - 1, j, k) + w(i + 1, j, k)) + (w(i, j - 1, k) + w(i, j + 1, k))) +
                          (wm + wp) - 6.0 * wc;
        const double yb = ybar[p];
        Tbar[p] = yb + Lw;
        if (in_xy && k >= 1 && k <= nz - 2) {
            const double tc = T[p];
            const double LT = ((T[p - 1] + T[p + 1]) + (T[p - sy] + T[p + sy])) +
                              (T[p - sz] + T[p + sz]) - 6.0 * tc;
            Csbar[p] = fma(yb, LT, Csbar[p]);
        }
        wm = wc;
        wc = wp;
    }
}

static bool use_tma(Grid3 g, int esz, const void *a, const void *b, const void *c, const void *d,
                    const void *e) {
    const void *ptrs[5] = {c, d, e, a, b};  // the three TMA-read fields first
    if (launch_override(PS_OVERRIDE_ADJ_PLAIN) == 1) return false;
    return adjoint_zmarch_supported(g, esz, ptrs, 5);
}

cudaError_t launch_adjoint_f64(double *Tbar, double *Cibar, const double *ybar, const double *T,
                               const double *Ci, StepCoef c, Grid3 g, cudaStream_t s) {
    if (use_tma(g, 8, Tbar, Cibar, ybar, T, Ci))
        return launch_adjoint_zmarch<double>(Tbar, Cibar, ybar, T, Ci, c, g, s);
    return launch_adjoint_basic<double>(Tbar, Cibar, ybar, T, Ci,
                                        CoefT<double>{c.dtlam, c.ax, c.ay, c.az}, g, s);
}

cudaError_t launch_adjoint_f64_scaled(double *Tbar, double *Csbar, const double *ybar,
                                      const double *T, const double *Cs, Grid3 g, cudaStream_t s) {
    if (use_tma(g, 8, Tbar, Csbar, ybar, T, Cs))
        return launch_adjoint_scaled(Tbar, Csbar, ybar, T, Cs, g, s);
    const dim3 block(32, 8, 1);
    const int64_t gx = (g.nx + block.x - 1) / block.x, gy = (g.ny + block.y - 1) / block.y;
    int64_t want = (8LL * sm_count() + gx * gy - 1) / (gx * gy);
    int64_t kchunk = (g.nz + want - 1) / want;
    if (kchunk < 16) kchunk = 16;
    const int64_t gz = (g.nz + kchunk - 1) / kchunk;
    if (gx > 0x7fffffff || gy > 65535 || gz > 65535) return cudaErrorInvalidConfiguration;
    k_adjoint_basic_scaled<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), block, 0, s>>>(
        Tbar, Csbar, ybar, T, Cs, g.nx, g.ny, g.nz, (int)kchunk);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_f32(float *Tbar, float *Cibar, const float *ybar, const float *T,
                               const float *Ci, StepCoef c, Grid3 g, cudaStream_t s) {
    const void *ptrs[5] = {T, ybar, Ci, Cibar, Tbar};
    if (launch_override(PS_OVERRIDE_ADJ_PLAIN) != 1 && adjoint_f32_supported(g, ptrs, 5))
        return launch_adjoint_f32_tma(Tbar, Cibar, ybar, T, Ci, c, g, s);
    return launch_adjoint_basic<float>(
        Tbar, Cibar, ybar, T, Ci,
        CoefT<float>{(float)c.dtlam, (float)c.ax, (float)c.ay, (float)c.az}, g, s);
}

}  // namespace psd

/*
 * FP64 CPU oracle for the 3-D variable-coefficient heat diffusion solver of
 * Omlin & Raess, "High-performance xPU Stencil Computations in Julia"
 * (arXiv 2211.15634), Fig. 1.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  It shares no code, header,
 * table or helper with the CUDA library, and only the tests, the package's
 * smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp (no fast-math, no FMA
 * contraction) so every operation rounds exactly once, in the order written.
 *
 * Layout: arrays of nx*ny*nz doubles, node (i,j,k) at offset i + nx*(j + ny*k)
 * (x fastest, matching Julia's column-major T[i,j,k]).
 *
 * Readings of the paper used here (the paper does not spell these out):
 *  - @inn(A) is A at the interior nodes 1..n-2 of every axis; @d2_xi(A) is the
 *    three-point second difference along x, taken at interior nodes, written
 *    as a difference of forward differences: (A[i+1]-A[i]) - (A[i]-A[i-1]).
 *  - _dx^2 is _dx*_dx (Julia's literal integer power of a Float64).
 *  - The step writes interior nodes only; T2 starts as a full copy of T, so
 *    the boundary stays at its initial values in both buffers (Dirichlet).
 *  - Julia evaluates a+b+c as (a+b)+c and lam*Ci*X as (lam*Ci)*X.
 *
 * Parity pins (tests/test_oracle_pins.py): constant field, discrete sine
 * eigenmode decay, dense matrix form on tiny grids, adjoint dot-product test,
 * complex-step and finite-difference gradients; the explicit-notation step
 * (or_step_explicit) has its own pins in tests/test_oracle_explicit_pins.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

/* Number of host threads used by the step loops (1 = serial). */
void or_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int or_get_threads(void) { return g_threads; }
int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* maximum(Ci) of Fig. 1's dt line: the largest element. */
double or_maximum(const double *A, int64_t n) {
    double m = A[0];
    for (int64_t p = 1; p < n; ++p)
        if (A[p] > m) m = A[p];
    return m;
}

/* Fig. 1, stable time step: dt = min(dx^2,dy^2,dz^2)/lam/maximum(Ci)/6.1. */
double or_stable_dt(double dx, double dy, double dz, double lam, double maxCi) {
    double m = dx * dx;
    if (dy * dy < m) m = dy * dy;
    if (dz * dz < m) m = dz * dz;
    return m / lam / maxCi / 6.1;
}

/* Three-point second differences at interior node p, combined with the
 * squared inverse spacings as in Fig. 1's step!:
 * (d2x*_dx^2 + d2y*_dy^2) + d2z*_dz^2. */
static double laplacian_at(const double *T, int64_t p, int64_t sx, int64_t sy, int64_t sz,
                           double _dx2, double _dy2, double _dz2) {
    double c = T[p];
    double d2x = (T[p + sx] - c) - (c - T[p - sx]);
    double d2y = (T[p + sy] - c) - (c - T[p - sy]);
    double d2z = (T[p + sz] - c) - (c - T[p - sz]);
    return (d2x * _dx2 + d2y * _dy2) + d2z * _dz2;
}

/* Fig. 1, step!(T2, T, Ci, lam, dt, _dx, _dy, _dz):
 *   @inn(T2) = @inn(T) + dt*(lam*@inn(Ci)*(@d2_xi(T)*_dx^2 + @d2_yi(T)*_dy^2 + @d2_zi(T)*_dz^2))
 * Only interior nodes of T2 are written. */
void or_step(double *T2, const double *T, const double *Ci, double lam, double dt,
             double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz) {
    const double _dx2 = _dx * _dx, _dy2 = _dy * _dy, _dz2 = _dz * _dz;
    const int64_t sx = 1, sy = nx, sz = nx * ny;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t k = 1; k < nz - 1; ++k)
        for (int64_t j = 1; j < ny - 1; ++j)
            for (int64_t i = 1; i < nx - 1; ++i) {
                int64_t p = i + nx * (j + ny * k);
                double lap = laplacian_at(T, p, sx, sy, sz, _dx2, _dy2, _dz2);
                T2[p] = T[p] + dt * ((lam * Ci[p]) * lap);
            }
}

/* The explicit-notation solver the paper's Results set beside Fig. 1's (the same
 * step with the stencil written out on indices instead of @d2_xi): each second
 * difference as A[i+1] - 2*A[i] + A[i-1], evaluated left to right.  The same
 * operator as laplacian_at in exact arithmetic; the roundings differ. */
static double laplacian_explicit_at(const double *T, int64_t p, int64_t sx, int64_t sy, int64_t sz,
                                    double _dx2, double _dy2, double _dz2) {
    double c = T[p];
    double d2x = (T[p + sx] - 2.0 * c) + T[p - sx];
    double d2y = (T[p + sy] - 2.0 * c) + T[p - sy];
    double d2z = (T[p + sz] - 2.0 * c) + T[p - sz];
    return (d2x * _dx2 + d2y * _dy2) + d2z * _dz2;
}

/* step! in the explicit notation (interior nodes of T2 only, as or_step). */
void or_step_explicit(double *T2, const double *T, const double *Ci, double lam, double dt,
                      double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz) {
    const double _dx2 = _dx * _dx, _dy2 = _dy * _dy, _dz2 = _dz * _dz;
    const int64_t sx = 1, sy = nx, sz = nx * ny;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t k = 1; k < nz - 1; ++k)
        for (int64_t j = 1; j < ny - 1; ++j)
            for (int64_t i = 1; i < nx - 1; ++i) {
                int64_t p = i + nx * (j + ny * k);
                double lap = laplacian_explicit_at(T, p, sx, sy, sz, _dx2, _dy2, _dz2);
                T2[p] = T[p] + dt * ((lam * Ci[p]) * lap);
            }
}

/* Fig. 1 time loop with the explicit-notation step (see or_run). */
int or_run_explicit(double *T, double *T2, const double *Ci, double lam, double dt,
                    double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz, int nt) {
    memcpy(T2, T, sizeof(double) * (size_t)(nx * ny * nz));
    double *cur = T, *nxt = T2;
    for (int it = 0; it < nt; ++it) {
        or_step_explicit(nxt, cur, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz);
        double *t = cur; cur = nxt; nxt = t;
    }
    return cur == T2;
}

/* Fig. 1 time loop: T2 = copy(T), then nt times { step!(T2, T, ...); swap }.
 * Returns 1 if the final state is in the buffer passed as T2 (nt odd), 0 if it
 * is in the buffer passed as T. */
int or_run(double *T, double *T2, const double *Ci, double lam, double dt,
           double _dx, double _dy, double _dz, int64_t nx, int64_t ny, int64_t nz, int nt) {
    memcpy(T2, T, sizeof(double) * (size_t)(nx * ny * nz));
    double *cur = T, *nxt = T2;
    for (int it = 0; it < nt; ++it) {
        or_step(nxt, cur, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz);
        double *t = cur; cur = nxt; nxt = t;
    }
    return cur == T2;
}

/* 2-D form of Fig. 1's dt line (a reading: the paper's solver is 3-D): the
 * explicit scheme on two axes is stable while dt*lam*Ci*(2/dx^2 + 2/dy^2) <= 1,
 * and 4.1 stands to that bound (4 for equal spacings) as Fig. 1's 6.1 stands to
 * the three-axis bound 6: dt = min(dx^2,dy^2)/lam/maximum(Ci)/4.1. */
double or_stable_dt2d(double dx, double dy, double lam, double maxCi) {
    double m = dx * dx;
    if (dy * dy < m) m = dy * dy;
    return m / lam / maxCi / 4.1;
}

/* 2-D form of Fig. 1's step!: the same update with the z term dropped, i.e. the
 * kernel with FiniteDifferences2D and the dimension argument of the initialization
 * call set to 2 (Fig. 1 shows 3):
 *   @inn(T2) = @inn(T) + dt*(lam*@inn(Ci)*(@d2_xi(T)*_dx^2 + @d2_yi(T)*_dy^2))
 * Arrays of nx*ny doubles, node (i,j) at offset i + nx*j; interior nodes only. */
void or_step2d(double *T2, const double *T, const double *Ci, double lam, double dt,
               double _dx, double _dy, int64_t nx, int64_t ny) {
    const double _dx2 = _dx * _dx, _dy2 = _dy * _dy;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t j = 1; j < ny - 1; ++j)
        for (int64_t i = 1; i < nx - 1; ++i) {
            int64_t p = i + nx * j;
            double c = T[p];
            double d2x = (T[p + 1] - c) - (c - T[p - 1]);
            double d2y = (T[p + nx] - c) - (c - T[p - nx]);
            T2[p] = c + dt * ((lam * Ci[p]) * (d2x * _dx2 + d2y * _dy2));
        }
}

/* 2-D time loop: T2 = copy(T), then nt times { step; swap }.  Returns 1 if the final
 * state is in the buffer passed as T2 (nt odd). */
int or_run2d(double *T, double *T2, const double *Ci, double lam, double dt, double _dx,
             double _dy, int64_t nx, int64_t ny, int nt) {
    memcpy(T2, T, sizeof(double) * (size_t)(nx * ny));
    double *cur = T, *nxt = T2;
    for (int it = 0; it < nt; ++it) {
        or_step2d(nxt, cur, Ci, lam, dt, _dx, _dy, nx, ny);
        double *t = cur; cur = nxt; nxt = t;
    }
    return cur == T2;
}

/* Transpose of one step (the step's Jacobian, applied from the left).
 * The step is T_{t+1} = T_t + diag(dt*lam*Ci*[interior]) * Lap(T_t) with
 * boundary rows equal to identity, so for a cotangent ybar = dL/dT_{t+1}:
 *   w[q]      = dt*lam*Ci[q]*ybar[q] at interior q, 0 on the boundary;
 *   Tbar[p]   = ybar[p] + sum_d (w[p-e_d] - 2 w[p] + w[p+e_d]) * _dd^2, with w = 0
 *               outside the grid (every node p, boundary included);
 *   Cibar[q] += dt*lam*ybar[q]*Lap(T_t)[q] at interior q (accumulated).
 * T is the state the forward step read (T_t). */
void or_adjoint_step(double *Tbar, double *Cibar, const double *ybar, const double *T,
                     const double *Ci, double lam, double dt, double _dx, double _dy, double _dz,
                     int64_t nx, int64_t ny, int64_t nz) {
    const double _dx2 = _dx * _dx, _dy2 = _dy * _dy, _dz2 = _dz * _dz;
    const int64_t n = nx * ny * nz, sx = 1, sy = nx, sz = nx * ny;
    double *w = (double *)calloc((size_t)n, sizeof(double));
    for (int64_t k = 1; k < nz - 1; ++k)
        for (int64_t j = 1; j < ny - 1; ++j)
            for (int64_t i = 1; i < nx - 1; ++i) {
                int64_t q = i + nx * (j + ny * k);
                w[q] = dt * ((lam * Ci[q]) * ybar[q]);
            }
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = i + nx * (j + ny * k);
                double c = w[p];
                double wxm = i > 0 ? w[p - sx] : 0.0, wxp = i < nx - 1 ? w[p + sx] : 0.0;
                double wym = j > 0 ? w[p - sy] : 0.0, wyp = j < ny - 1 ? w[p + sy] : 0.0;
                double wzm = k > 0 ? w[p - sz] : 0.0, wzp = k < nz - 1 ? w[p + sz] : 0.0;
                double d2x = (wxp - c) - (c - wxm);
                double d2y = (wyp - c) - (c - wym);
                double d2z = (wzp - c) - (c - wzm);
                Tbar[p] = ybar[p] + ((d2x * _dx2 + d2y * _dy2) + d2z * _dz2);
            }
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t k = 1; k < nz - 1; ++k)
        for (int64_t j = 1; j < ny - 1; ++j)
            for (int64_t i = 1; i < nx - 1; ++i) {
                int64_t q = i + nx * (j + ny * k);
                double lap = laplacian_at(T, q, sx, sy, sz, _dx2, _dy2, _dz2);
                Cibar[q] += (dt * lam) * (ybar[q] * lap);
            }
    free(w);
}

/* Loss and gradient of L = 1/2 ||T(nt) - Tobs||^2 with respect to T0 and Ci,
 * dt held constant.  Stores every state (memory (nt+1)*n doubles), runs the
 * transposed steps in reverse order.  Returns L, or -1 if memory ran out. */
double or_gradient(double *dT0, double *dCi, const double *T0, const double *Ci,
                   const double *Tobs, double lam, double dt, double _dx, double _dy, double _dz,
                   int64_t nx, int64_t ny, int64_t nz, int nt) {
    const int64_t n = nx * ny * nz;
    const size_t bytes = sizeof(double) * (size_t)n;
    double *states = (double *)malloc(bytes * (size_t)(nt + 1));
    double *ybar = (double *)malloc(bytes);
    double *tmp = (double *)malloc(bytes);
    if (!states || !ybar || !tmp) { free(states); free(ybar); free(tmp); return -1.0; }
    memcpy(states, T0, bytes);
    for (int t = 0; t < nt; ++t) {
        double *cur = states + (size_t)t * n, *nxt = cur + n;
        memcpy(nxt, cur, bytes);
        or_step(nxt, cur, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz);
    }
    const double *Tn = states + (size_t)nt * n;
    double L = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        double r = Tn[p] - Tobs[p];
        L += r * r;
        ybar[p] = r;
    }
    L *= 0.5;
    memset(dCi, 0, bytes);
    for (int t = nt - 1; t >= 0; --t) {
        or_adjoint_step(tmp, dCi, ybar, states + (size_t)t * n, Ci, lam, dt, _dx, _dy, _dz, nx, ny, nz);
        double *s = ybar; ybar = tmp; tmp = s;
    }
    memcpy(dT0, ybar, bytes);
    free(states); free(ybar); free(tmp);
    return L;
}

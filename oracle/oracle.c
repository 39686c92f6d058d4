/*
 * oracle.c -- plain CPU oracle for iterated explicit 2D stencil sweeps.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (paper, Sec. II-C, the Jacobi update):
 *     u^{t+1}[i][j] = sum_{dy,dx in [-r,r]} W[dy+r][dx+r] * u~^{t}[i+dy][j+dx]
 * for t = 0 .. T-1, where u~ is u extended outside [0,ny) x [0,nx):
 *   - boundary 0 (zero): by zeros.  The paper pads the global grid with zeros
 *     and keeps that padding fixed, which is the zero boundary condition
 *     (Sec. IV-A, steps 1 and 3).
 *   - boundary 1 (periodic): by wrapping indices modulo ny and nx.
 * i is the row (y, slowest-varying index), j the column (x, contiguous).
 * W is the (2r+1)x(2r+1) weight array, row-major, entries off the stencil's
 * footprint are zero (Star and Box shapes, Sec. II-B).  The weighted sum is a
 * cross-correlation (no kernel flip) and is summed dy-major, then dx, one
 * product at a time, exactly as the naive scalar loop of the paper's
 * Sec. IV-E listing (centre-first ordering differs only in the order of exact
 * zero additions, which does not change results).
 *
 * The adjoint (used for gradients of L(u_T)) follows from the same
 * definition: with lambda_T = dL/du_T,
 *     lambda_t[p][q] = sum_{dy,dx} W[dy+r][dx+r] * lambda~_{t+1}[p-dy][q-dx]
 *     dL/dW[dy+r][dx+r] = sum_{t=0}^{T-1} sum_{i,j} lambda_{t+1}[i][j] * u~_t[i+dy][j+dx]
 *     dL/du_0 = lambda_0.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no FMA contraction,
 * so x86_64 and aarch64 hosts give bit-identical FP32 results).
 * Row loops carry an OpenMP parallel-for; every output element is computed by
 * the same sequence of operations whatever the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORACLE_OK = 0, ORACLE_ERR_ARG = 1, ORACLE_ERR_NOMEM = 2 };

static int64_t wrap_index(int64_t i, int64_t n) {
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

/* u~[i][j] in FP64: the grid extended by its boundary rule. */
static double ext_f64(const double* u, int64_t ny, int64_t nx, int64_t i, int64_t j,
                      int periodic) {
    if (periodic) {
        return u[wrap_index(i, ny) * nx + wrap_index(j, nx)];
    }
    if (i < 0 || i >= ny || j < 0 || j >= nx) return 0.0;
    return u[i * nx + j];
}

static float ext_f32(const float* u, int64_t ny, int64_t nx, int64_t i, int64_t j,
                     int periodic) {
    if (periodic) {
        return u[wrap_index(i, ny) * nx + wrap_index(j, nx)];
    }
    if (i < 0 || i >= ny || j < 0 || j >= nx) return 0.0f;
    return u[i * nx + j];
}

static int check_args(int64_t ny, int64_t nx, int r, int boundary, int64_t T) {
    if (ny < 1 || nx < 1 || r < 0 || r > 8 || T < 0) return ORACLE_ERR_ARG;
    if (boundary != 0 && boundary != 1) return ORACLE_ERR_ARG;
    return ORACLE_OK;
}

/* One Jacobi step in FP64 (Sec. II-C). */
static void step_f64(int64_t ny, int64_t nx, int r, const double* W, int periodic,
                     const double* u, double* v) {
    const int d = 2 * r + 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ny; ++i) {
        for (int64_t j = 0; j < nx; ++j) {
            double acc = 0.0;
            for (int dy = -r; dy <= r; ++dy) {
                for (int dx = -r; dx <= r; ++dx) {
                    acc += W[(dy + r) * d + (dx + r)] *
                           ext_f64(u, ny, nx, i + dy, j + dx, periodic);
                }
            }
            v[i * nx + j] = acc;
        }
    }
}

/* One Jacobi step in FP32 arithmetic, same operation order as step_f64. */
static void step_f32(int64_t ny, int64_t nx, int r, const float* W, int periodic,
                     const float* u, float* v) {
    const int d = 2 * r + 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ny; ++i) {
        for (int64_t j = 0; j < nx; ++j) {
            float acc = 0.0f;
            for (int dy = -r; dy <= r; ++dy) {
                for (int dx = -r; dx <= r; ++dx) {
                    float prod = W[(dy + r) * d + (dx + r)] *
                                 ext_f32(u, ny, nx, i + dy, j + dx, periodic);
                    acc = acc + prod;
                }
            }
            v[i * nx + j] = acc;
        }
    }
}

/* T Jacobi steps in FP64 with ping-pong buffers.  u0 and out may alias. */
int oracle_sweep_f64(int64_t ny, int64_t nx, int r, const double* W, int boundary,
                     int64_t T, const double* u0, double* out) {
    int rc = check_args(ny, nx, r, boundary, T);
    if (rc) return rc;
    const size_t n = (size_t)ny * (size_t)nx;
    double* a = (double*)malloc(n * sizeof(double));
    double* b = (double*)malloc(n * sizeof(double));
    if (!a || !b) { free(a); free(b); return ORACLE_ERR_NOMEM; }
    memcpy(a, u0, n * sizeof(double));
    for (int64_t t = 0; t < T; ++t) {
        step_f64(ny, nx, r, W, boundary == 1, a, b);
        double* s = a; a = b; b = s;
    }
    memcpy(out, a, n * sizeof(double));
    free(a); free(b);
    return ORACLE_OK;
}

/* T Jacobi steps in FP32 arithmetic (the FP32 reference and CPU baseline). */
int oracle_sweep_f32(int64_t ny, int64_t nx, int r, const float* W, int boundary,
                     int64_t T, const float* u0, float* out) {
    int rc = check_args(ny, nx, r, boundary, T);
    if (rc) return rc;
    const size_t n = (size_t)ny * (size_t)nx;
    float* a = (float*)malloc(n * sizeof(float));
    float* b = (float*)malloc(n * sizeof(float));
    if (!a || !b) { free(a); free(b); return ORACLE_ERR_NOMEM; }
    memcpy(a, u0, n * sizeof(float));
    for (int64_t t = 0; t < T; ++t) {
        step_f32(ny, nx, r, W, boundary == 1, a, b);
        float* s = a; a = b; b = s;
    }
    memcpy(out, a, n * sizeof(float));
    free(a); free(b);
    return ORACLE_OK;
}

/*
 * The Heat-2D update written literally, u' = u + c*(N + S + E + W - 4u), in FP64
 * with zero boundary.  A cross-check of the weight form (centre 1-4c, arms c);
 * the two agree only up to rounding.
 */
int oracle_heat_literal_f64(int64_t ny, int64_t nx, double c, int64_t T,
                            const double* u0, double* out) {
    int rc = check_args(ny, nx, 1, 0, T);
    if (rc) return rc;
    const size_t n = (size_t)ny * (size_t)nx;
    double* a = (double*)malloc(n * sizeof(double));
    double* b = (double*)malloc(n * sizeof(double));
    if (!a || !b) { free(a); free(b); return ORACLE_ERR_NOMEM; }
    memcpy(a, u0, n * sizeof(double));
    for (int64_t t = 0; t < T; ++t) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < ny; ++i) {
            for (int64_t j = 0; j < nx; ++j) {
                double uc = a[i * nx + j];
                double un = ext_f64(a, ny, nx, i - 1, j, 0);
                double us = ext_f64(a, ny, nx, i + 1, j, 0);
                double ue = ext_f64(a, ny, nx, i, j + 1, 0);
                double uw = ext_f64(a, ny, nx, i, j - 1, 0);
                b[i * nx + j] = uc + c * (un + us + ue + uw - 4.0 * uc);
            }
        }
        double* s = a; a = b; b = s;
    }
    memcpy(out, a, n * sizeof(double));
    free(a); free(b);
    return ORACLE_OK;
}

/*
 * Adjoint of T steps in FP64.  gT = dL/du_T (ny*nx).  Writes grad_u0 = dL/du_0
 * and grad_W = dL/dW ((2r+1)^2, row-major like W).  Stores every u_t, so it is
 * meant for small grids.
 */
int oracle_adjoint_f64(int64_t ny, int64_t nx, int r, const double* W, int boundary,
                       int64_t T, const double* u0, const double* gT,
                       double* grad_u0, double* grad_W) {
    int rc = check_args(ny, nx, r, boundary, T);
    if (rc) return rc;
    const int d = 2 * r + 1;
    const int periodic = boundary == 1;
    const size_t n = (size_t)ny * (size_t)nx;
    double* us = (double*)malloc((size_t)(T + 1) * n * sizeof(double));
    double* lam = (double*)malloc(n * sizeof(double));
    double* lam_prev = (double*)malloc(n * sizeof(double));
    if (!us || !lam || !lam_prev) {
        free(us); free(lam); free(lam_prev);
        return ORACLE_ERR_NOMEM;
    }
    /* forward pass, every state kept */
    memcpy(us, u0, n * sizeof(double));
    for (int64_t t = 0; t < T; ++t) {
        step_f64(ny, nx, r, W, periodic, us + (size_t)t * n, us + (size_t)(t + 1) * n);
    }
    for (int k = 0; k < d * d; ++k) grad_W[k] = 0.0;
    memcpy(lam, gT, n * sizeof(double));  /* lambda_T */
    for (int64_t t = T - 1; t >= 0; --t) {
        const double* ut = us + (size_t)t * n;
        /* dL/dW += sum_{i,j} lambda_{t+1}[i][j] * u~_t[i+dy][j+dx] */
        for (int dy = -r; dy <= r; ++dy) {
            for (int dx = -r; dx <= r; ++dx) {
                double s = 0.0;
                for (int64_t i = 0; i < ny; ++i) {
                    for (int64_t j = 0; j < nx; ++j) {
                        s += lam[i * nx + j] * ext_f64(ut, ny, nx, i + dy, j + dx, periodic);
                    }
                }
                grad_W[(dy + r) * d + (dx + r)] += s;
            }
        }
        /* lambda_t = A^T lambda_{t+1} */
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < ny; ++p) {
            for (int64_t q = 0; q < nx; ++q) {
                double acc = 0.0;
                for (int dy = -r; dy <= r; ++dy) {
                    for (int dx = -r; dx <= r; ++dx) {
                        acc += W[(dy + r) * d + (dx + r)] *
                               ext_f64(lam, ny, nx, p - dy, q - dx, periodic);
                    }
                }
                lam_prev[p * nx + q] = acc;
            }
        }
        double* s = lam; lam = lam_prev; lam_prev = s;
    }
    memcpy(grad_u0, lam, n * sizeof(double));
    free(us); free(lam); free(lam_prev);
    return ORACLE_OK;
}

/* Threads an OpenMP parallel region uses (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * FP64 CPU oracle: shifted finite-difference Hamiltonian and COCG.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is used
 * by the test-suite, by the smoke check and by the timed CPU baseline.  The CUDA
 * library never links it, and it shares no code with the CUDA library.
 *
 * Written for readability, not speed: straight loops, C99 complex doubles, a
 * bounds test for every stencil tap.
 *
 *   apply:  out = (H + sigma) in,  H = -1/2 L_h + diag(V_loc)
 *           L_h is the centred finite-difference Laplacian whose weights w[0..R]
 *           (already divided by h^2) are passed in; grid values outside the box are
 *           zero (Dirichlet) or, with `periodic`, those of the periodic continuation
 *           of the grid function (the bulk cells of the paper's Section "Results"),
 *           as in the real-space method of the paper (Section "Implementation":
 *           matrix-free high-order centred finite differences).
 *   cocg:   COCG (van der Vorst & Melissen 1990), the conjugate-orthogonal CG the
 *           paper uses for the complex-symmetric Sternheimer systems
 *           (H - eps_n + i omega) x = b  (Section "Implementation", Sternheimer
 *           equation of the Formulation).  Unconjugated bilinear form x^T y; stop
 *           when ||r||_2 / ||b||_2 <= tol (Hermitian 2-norm; Section "Results":
 *           tolerance on the relative residual).  Zero initial guess.
 *
 * Grid layout: point (i,j,k) at i + nx*(j + ny*k).  Complex vectors are
 * interleaved (re, im) doubles.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_NOT_CONVERGED 4
#define ORACLE_BREAKDOWN 5

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Grid index a along an axis of n points: itself inside [0, n), its periodic image when
 * `periodic`, else -1 (outside the box: a zero value). */
static int tap(int a, int n, int periodic) {
    if (a >= 0 && a < n) return a;
    if (!periodic) return -1;
    a %= n;
    return a < 0 ? a + n : a;
}

/* out = (-1/2 L_h + V + sigma) in, for one complex grid function. */
static void apply_shifted_h(int nx, int ny, int nz, int radius, const double *w, int periodic,
                            const double *vloc, double complex sigma,
                            const double complex *in, double complex *out) {
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long idx = i + (long)nx * (j + (long)ny * k);
                double complex lap = 3.0 * w[0] * in[idx];
                for (int s = 1; s <= radius; ++s) {
                    for (int sg = -1; sg <= 1; sg += 2) {
                        int a;
                        if ((a = tap(i + sg * s, nx, periodic)) >= 0)
                            lap += w[s] * in[a + (long)nx * (j + (long)ny * k)];
                        if ((a = tap(j + sg * s, ny, periodic)) >= 0)
                            lap += w[s] * in[i + (long)nx * (a + (long)ny * k)];
                        if ((a = tap(k + sg * s, nz, periodic)) >= 0)
                            lap += w[s] * in[i + (long)nx * (j + (long)ny * a)];
                    }
                }
                out[idx] = -0.5 * lap + (vloc[idx] + sigma) * in[idx];
            }
}

void oracle_apply_h(int nx, int ny, int nz, int radius, const double *w, int periodic, const double *vloc,
                    double sigma_re, double sigma_im, const double *in, double *out) {
    apply_shifted_h(nx, ny, nz, radius, w, periodic, vloc, sigma_re + I * sigma_im,
                    (const double complex *)in, (double complex *)out);
}

/* Unconjugated bilinear form x^T y. */
static double complex dotu(long n, const double complex *x, const double complex *y) {
    double complex s = 0.0;
    for (long i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

static double norm2(long n, const double complex *x) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
    return sqrt(s);
}

/* One COCG solve.  Returns the status; *iters gets the iteration count. */
static int cocg_one(int nx, int ny, int nz, int radius, const double *w, int periodic, const double *vloc,
                    double complex sigma, const double complex *b, double complex *x,
                    double tol, int maxit, int *iters) {
    long n = (long)nx * ny * nz;
    double complex *r = malloc(sizeof(double complex) * n);
    double complex *p = malloc(sizeof(double complex) * n);
    double complex *q = malloc(sizeof(double complex) * n);
    int status = ORACLE_NOT_CONVERGED;
    int it = 0;
    memset(x, 0, sizeof(double complex) * n);
    memcpy(r, b, sizeof(double complex) * n);
    memcpy(p, b, sizeof(double complex) * n);
    double bnorm = norm2(n, b);
    if (bnorm == 0.0) {
        status = ORACLE_OK;
        goto done;
    }
    double complex rho = dotu(n, r, r);
    for (it = 0; it < maxit;) {
        apply_shifted_h(nx, ny, nz, radius, w, periodic, vloc, sigma, p, q);
        double complex mu = dotu(n, p, q);
        if (cabs(mu) == 0.0 || cabs(rho) == 0.0) {
            status = ORACLE_BREAKDOWN;
            break;
        }
        double complex alpha = rho / mu;
        for (long i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        ++it;
        if (norm2(n, r) <= tol * bnorm) {
            status = ORACLE_OK;
            break;
        }
        double complex rho_new = dotu(n, r, r);
        double complex beta = rho_new / rho;
        rho = rho_new;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
done:
    free(r);
    free(p);
    free(q);
    *iters = it;
    return status;
}

/* Solve nsys independent systems (H + sigma_s) x_s = b_s; systems run in parallel
 * over the host's threads. */
void oracle_cocg_batch(int nx, int ny, int nz, int radius, const double *w, int periodic, const double *vloc,
                       int nsys, const double *sigma_re, const double *sigma_im, const double *b,
                       double *x, double tol, int maxit, int *iters, int *status) {
    long n = (long)nx * ny * nz;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int s = 0; s < nsys; ++s) {
        status[s] = cocg_one(nx, ny, nz, radius, w, periodic, vloc, sigma_re[s] + I * sigma_im[s],
                             (const double complex *)(b + 2 * n * s), (double complex *)(x + 2 * n * s),
                             tol, maxit, &iters[s]);
    }
}

/* Multi-threaded timing variant of the oracle's Jacobi-PCG (test
 * infrastructure: only the CPU baseline of the benchmark and the tests use
 * it; the CUDA library never links it).
 *
 * The same textbook preconditioned conjugate-gradient iteration as or_pcg in
 * cps_oracle.c (Sec. 3.2.2: the corrector systems are solved by PCG), with
 * the Jacobi preconditioner, on the same CSR matrix.  The only difference is
 * that every loop over the rows runs as an OpenMP parallel loop on all the
 * host cores, and the inner products are OpenMP reductions (their summation
 * order therefore differs from the single-threaded oracle's, so the iterates
 * agree with it up to rounding).  It exists to give an honest CPU baseline:
 * the single-threaded oracle is the parity checker, this is what a plain
 * shared-memory CPU code does with all the cores of the GPU's host.
 *
 * Built with -fopenmp into its own library (libcps_oracle_omp.so) so that
 * the parity oracle stays single-threaded and free of OpenMP.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORO_OK 0
#define ORO_ERR_ARG -1
#define ORO_ERR_NOT_SPD -5
#define ORO_ERR_NOT_CONVERGED -6
#define ORO_ERR_NOMEM -8

/* Threads the parallel loops use (1 without OpenMP). */
int oro_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void matvec(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                   const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Jacobi-PCG from the initial guess in x; stats[0] = iterations, stats[1] =
 * true relative residual ||b - A x|| / ||b|| at exit, stats[2] = recursive
 * relative residual at exit.  maxit bounds the iterations (rtol 0 runs
 * exactly maxit of them, the benchmark's bounded sample). */
int oro_pcg_jacobi(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                   const double* b, double* x, double rtol, int64_t maxit, double* stats) {
    if (n < 0 || !stats) return ORO_ERR_ARG;
    stats[0] = 0;
    stats[1] = 0;
    stats[2] = 0;
    if (n == 0) return ORO_OK;
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    double* dinv = (double*)malloc(sizeof(double) * n);
    int rc = ORO_OK;
    if (!r || !z || !p || !q || !dinv) {
        rc = ORO_ERR_NOMEM;
        goto done;
    }
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) d += v[k];
        if (!(d > 0.0)) bad = 1;
        dinv[i] = d > 0.0 ? 1.0 / d : 0.0;
    }
    if (bad) {
        rc = ORO_ERR_NOT_SPD;
        goto done;
    }
    const double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        goto done;
    }
    matvec(n, rp, ci, v, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        r[i] = b[i] - q[i];
        z[i] = dinv[i] * r[i];
        p[i] = z[i];
    }
    double rho = dot(n, r, z);
    double relres = sqrt(dot(n, r, r)) / bnorm;
    int64_t it = 0;
    while (relres > rtol && it < maxit) {
        matvec(n, rp, ci, v, p, q);
        const double gamma = dot(n, p, q);
        if (!(gamma > 0.0)) {
            rc = ORO_ERR_NOT_SPD;
            break;
        }
        const double alpha = rho / gamma;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        ++it;
        relres = sqrt(dot(n, r, r)) / bnorm;
        if (relres <= rtol) break;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        const double rho_new = dot(n, r, z);
        const double beta = rho_new / rho;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rho = rho_new;
    }
    stats[0] = (double)it;
    stats[2] = relres;
    matvec(n, rp, ci, v, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    stats[1] = sqrt(dot(n, r, r)) / bnorm;
    if (rc == ORO_OK && relres > rtol) rc = ORO_ERR_NOT_CONVERGED;
done:
    free(r);
    free(z);
    free(p);
    free(q);
    free(dinv);
    return rc;
}

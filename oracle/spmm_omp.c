/* CPU SpMM of the CPU baseline - test infrastructure, never on the product
 * path (only the tests and bench.py's cpu_baseline leg load it).
 *
 * Y = A X for a CSR matrix A (n rows, int32 row pointers and columns, FP64
 * values) and N right-hand sides stored interleaved (X[c][j] at X[c * N + j],
 * Y[i][j] at Y[i * N + j]): the plain definition of the product that the
 * block PCG of the N shifted problems of Algorithm 3 (step 1) applies every
 * iteration, rows split over OpenMP threads.  SciPy's CSR product runs on one
 * thread, so the baseline's SpMM bandwidth on all host cores comes from here.
 */
#include <stdint.h>

#include <omp.h>

void oracle_spmm(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, int N,
                 const double* X, double* Y, int threads) {
    if (threads < 1) threads = 1;
#pragma omp parallel for schedule(static) num_threads(threads)
    for (int64_t i = 0; i < n; ++i) {
        double* y = Y + i * N;
        for (int j = 0; j < N; ++j) y[j] = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const double a = val[p];
            const double* x = X + (int64_t)col[p] * N;
            for (int j = 0; j < N; ++j) y[j] += a * x[j];
        }
    }
}

/* Mean wall time in seconds of `reps` products after one untimed product. */
double oracle_spmm_seconds(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, int N,
                           const double* X, double* Y, int threads, int reps) {
    if (reps < 1) reps = 1;
    oracle_spmm(n, rowptr, col, val, N, X, Y, threads);
    const double t0 = omp_get_wtime();
    for (int r = 0; r < reps; ++r) oracle_spmm(n, rowptr, col, val, N, X, Y, threads);
    return (omp_get_wtime() - t0) / reps;
}

// Host solver for the small generalized eigenproblem F_A U = lambda F_B U of
// Algorithm 3 (eq. st1), F_A symmetric, F_B symmetric positive definite.
#pragma once

#include <cstdint>

namespace nas {

// Dense: A, B row-major [m][m] (only the lower triangle is read); computes
// the k smallest eigenvalues lam[k] (ascending) and B-orthonormal vectors
// U row-major [m][k].  Returns 0, or -1 if B is not positive definite.
int dense_gen_eig(int m, const double* A, const double* B, int k, double* lam, double* U);

// Symmetric eigenvalues/vectors of a small dense matrix by cyclic Jacobi
// (used for condition numbers and tiny problems): A [m][m] row-major is
// overwritten; w[m] ascending, V[m][m] row-major columns = eigenvectors.
void jacobi_eig(int m, double* A, double* w, double* V);

// Dense Cholesky A = L L^T in place (row-major [m][m]; the lower triangle
// receives L, the strict upper triangle is zeroed).  Returns 0 or -1 if A is
// not positive definite.
int chol_factor(int m, double* A);
// Solve (L L^T) X = B for B row-major [m][k] (overwritten by X).
void chol_solve(int m, const double* L, int k, double* B);

// Solve A x = b (n <= 8) by Gaussian elimination with partial pivoting.
// Returns 0 or -1 if singular.
int small_solve(int n, const double* A, const double* b, double* x);

}  // namespace nas

namespace nas {

// Arrow-structured symmetric matrix of the small problem (eq. st2):
//   F = [[S, Bd], [Bd^T, Cd]],  S sparse nH x nH (CSR, full symmetric storage),
//   Bd dense nH x Na (row-major), Cd dense Na x Na.
struct ArrowMat {
    int64_t nH = 0;
    int Na = 0;
    const int32_t* ptr = nullptr;
    const int32_t* col = nullptr;
    const double* sval = nullptr;
    const double* Bd = nullptr;
    const double* Cd = nullptr;
};

// Lowest `nev` eigenpairs of A u = lambda B u by LOBPCG (Knyazev 2001) with
// nguard extra block vectors, a diagonal preconditioner diag(A - sigma B)^-1,
// and an orthonormalised Rayleigh-Ritz basis [X, W, P] (eigen-decomposition
// of the basis Gram matrix, dropping near-dependent directions).
// U [m][nev] (row-major) holds a warm start when warm = true, and receives
// B-orthonormal eigenvectors.  Stops when every wanted residual satisfies
// ||A u - lambda B u|| <= tol (||A u|| + |lambda| ||B u||).  Returns iterations
// used, or -1 on failure.
int lobpcg_arrow(const ArrowMat& A, const ArrowMat& B, int nev, int nguard, double* lam, double* U, bool warm,
                 double tol, int maxit);

}  // namespace nas

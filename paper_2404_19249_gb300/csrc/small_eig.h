// Host solver for the small generalized eigenproblem F_A U = lambda F_B U of
// Algorithm 3 (Sec. 3.3), F_A symmetric, F_B symmetric positive definite.
#pragma once

#include <cstdint>
#include <vector>

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
// Inv = (L L^T)^-1, row-major [m][m] (symmetric), from the factor of chol_factor;
// columns in parallel, each row-oriented (contiguous reads of L and L^T).
void chol_inverse(int m, const double* L, double* Inv);

// Solve A x = b (n <= 16) by Gaussian elimination with partial pivoting.
// Returns 0, or -1 if singular or n is out of range.
int small_solve(int n, const double* A, const double* b, double* x);

}  // namespace nas

namespace nas {

// Arrow-structured symmetric matrix of the small problem (the 2 x 2 block form of F_A, F_B in Sec. 3.3):
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

// Rayleigh-Ritz step of LOBPCG from the Gram matrices of a basis S [m][ns]:
// G = S^T B S and H = S^T A S (row-major [ns][ns]; symmetrised in place).
// When G's Cholesky factor has every squared pivot above 1e-8 of the largest
// diagonal entry, the pencil (H, G) is solved through that factor; otherwise
// (*fallback = true when given) the basis is B-orthonormalised by two passes
// of G's eigen-decomposition, dropping directions whose Gram eigenvalue is
// below 1e-9 of the largest.  Then the lowest k Ritz pairs: theta[k] and
// coefficients Y [ns][k] (S Y is B-orthonormal).  Returns 0, or -1 if fewer
// than k directions remain.
int rayleigh_ritz_grams(int ns, std::vector<double>& G, std::vector<double>& H, int k, std::vector<double>& Y,
                        std::vector<double>& theta, bool* fallback = nullptr);

}  // namespace nas

// extern "C" entry points over the host small-problem eigensolver
// (paper_2404_19249_gb300/csrc/small_eig.cpp) for the CPU tests: the tests
// compile this file together with small_eig.cpp into a throw-away shared
// library and call it through ctypes.  Test infrastructure only.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "small_eig.h"

extern "C" {

int shim_dense_gen_eig(int m, const double* A, const double* B, int k, double* lam, double* U) {
    return nas::dense_gen_eig(m, A, B, k, lam, U);
}

int shim_rayleigh_ritz(int ns, const double* G, const double* H, int k, double* Y, double* theta) {
    std::vector<double> g(G, G + (size_t)ns * ns), h(H, H + (size_t)ns * ns), y, th;
    const int r = nas::rayleigh_ritz_grams(ns, g, h, k, y, th);
    if (r == 0) {
        std::copy(y.begin(), y.begin() + (size_t)ns * k, Y);
        std::copy(th.begin(), th.begin() + k, theta);
    }
    return r;
}

int shim_lobpcg_arrow(int64_t nH, int Na, const int32_t* ptr, const int32_t* col, const double* as, const double* ab,
                      const double* ac, const double* bs, const double* bb, const double* bc, int nev, int nguard,
                      double* lam, double* U, int warm, double tol, int maxit) {
    nas::ArrowMat A{nH, Na, ptr, col, as, ab, ac};
    nas::ArrowMat B{nH, Na, ptr, col, bs, bb, bc};
    return nas::lobpcg_arrow(A, B, nev, nguard, lam, U, warm != 0, tol, maxit);
}

int shim_chol_inverse(int m, double* A, double* Inv) {
    if (nas::chol_factor(m, A) != 0) return -1;
    nas::chol_inverse(m, A, Inv);
    return 0;
}

int shim_small_solve(int n, const double* A, const double* b, double* x) { return nas::small_solve(n, A, b, x); }

}  // extern "C"

// LOBPCG for the small pencil F_A U = lambda F_B U of Algorithm 3 (Sec. 3.3)
// with the block vectors on the device.  The arrow-structured products, the
// residuals, the orthogonalisation and the Gram matrices of the basis
// [X, W, P] run in device kernels; the host receives the residual norms
// (convergence test, active columns) and the Gram matrices (at most (3k)^2
// numbers, k = nev + nguard) and returns the Rayleigh-Ritz coefficients.
#pragma once

#include "common.h"
#include "kernels.h"

namespace nas {

struct DevLobpcg {
    // block vectors [m][k] (raw pointers are swapped between iterations)
    DBuf<double> bufs[11];
    DBuf<double> T, theta, nrm, gpart, gtmp, GAB, Y, C;  // GAB = S^T [AS | BS]
    DBuf<float> ppart;    // split partial products of the dense preconditioner
    DBuf<double> Yp;      // coefficients of the new search directions [2k][k]
    DBuf<int> actd;       // active (unlocked) block columns
    DBuf<double> X0;      // pseudo-random start block [m][k]
    int64_t x0_m = 0;
    int x0_k = 0;
    int64_t m_cap = 0;
    int k_cap = 0;
    bool tc = false;      // the dense preconditioner product on the tensor cores
    double rr_ms = 0.0;   // host time in Rayleigh-Ritz (accumulated)
    int rr_calls = 0;     // Rayleigh-Ritz steps, and those that took the two-pass path
    int rr_fallbacks = 0;
    double wait_ms = 0.0; // host time waiting for the device in synchronisations
    // pinned staging area for the per-iteration transfers (Grams, norms,
    // Ritz coefficients, active columns), so that they are truly asynchronous
    double* pin = nullptr;
    size_t pin_doubles = 0;
    DevLobpcg() = default;
    DevLobpcg(const DevLobpcg&) = delete;
    DevLobpcg& operator=(const DevLobpcg&) = delete;
    ~DevLobpcg() {
        if (pin) cudaFreeHost(pin);
    }

    // Lowest nev pairs.  U0: device [m][nev] warm start or null; Uout: device
    // [m][nev] (B-orthonormal eigenvectors); lam: host [nev].  diag_slot[i] is
    // the CSR slot of the coarse block's diagonal entry (i, i).  Stops when every
    // wanted residual satisfies ||A u - lambda B u|| <= tol (||A u|| + |lambda|
    // ||B u||).  Returns the iterations used, or -1 on failure.
    // TH (optional): FP32 [nH][nH] preconditioner block for the coarse rows
    // (the border rows keep the diagonal one).
    // reuse_block: start from the full block of the previous solve (same m and
    // k, same F_B) instead of U0 and random guard columns.
    int solve(const ArrowDev& A, const ArrowDev& B, const int32_t* diag_slot, int nev, int nguard, double* lam,
              const double* U0, double* Uout, double tol, int maxit, cudaStream_t s, const float* TH = nullptr,
              bool reuse_block = false);
    DBuf<double> Xkeep;   // last solve's block [m][k]
    int64_t keep_m = 0;
    int keep_k = 0;
};

}  // namespace nas

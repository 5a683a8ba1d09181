// Device kernels of the LOBPCG solver for the small pencil F_A U = lambda F_B U
// of Algorithm 3 (eq. st1/st2).  Both matrices have the arrow structure of the
// augmented basis {I phi_a} + {u^_j}: a sparse coarse block (CSR over the
// coarse unknowns), a dense border [nH][Na] and a dense corner [Na][Na].  The
// block vectors are row-major [m][w] with m = nH + Na.  Every sum runs in a
// fixed order (per-chunk partial sums, then an ordered final pass), so results
// are bit-reproducible.
#include <mutex>

#include "kernels.h"

namespace nas {

static int grid_of(int64_t n, int b) { return (int)std::max<int64_t>(1, (n + b - 1) / b); }

// ---- Y[i][j] = sum_p sval[p] X[col[p]][j] + sum_a Bd[i][a] X[nH+a][j]   (i < nH)
__global__ void k_arrow_rows(ArrowDev F, int w, const double* X, double* Y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= F.nH * w) return;
    const int64_t i = t / w;
    const int j = (int)(t - i * w);
    double acc = 0.0;
    for (int p = F.ptr[i]; p < F.ptr[i + 1]; ++p) acc += F.sval[p] * X[(int64_t)F.col[p] * w + j];
    const double* xa = X + F.nH * w + j;
    for (int a = 0; a < F.Na; ++a) acc += F.Bd[i * F.Na + a] * xa[(int64_t)a * w];
    Y[t] = acc;
}

// ---- border rows: Y[nH+a][j] = G[a][j] + sum_b Cd[a][b] X[nH+b][j], G = Bd^T X_H
__global__ void k_arrow_border(ArrowDev F, int w, const double* X, const double* G, double* Y) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= F.Na * w) return;
    const int a = t / w, j = t - (t / w) * w;
    double acc = G[t];
    const double* xa = X + F.nH * w + j;
    for (int b = 0; b < F.Na; ++b) acc += F.Cd[a * F.Na + b] * xa[(int64_t)b * w];
    Y[(F.nH + a) * w + j] = acc;
}

// ---- tiled Gram G[a][b] = sum_i L(i,a) R(i,b) over row chunks
// Block (chunk, ta, tb) handles output tile [32 ta, +32) x [32 tb, +32) for one
// 64-row chunk, staged in shared memory.  A loading thread always serves the
// same tile column, so its source pointer and stride are resolved once and its
// eight loads per operand are independent.  Thread t then owns row ta*32 + t/8
// and columns tb*32 + 4(t%8) .. +3 of the tile.
static const int kGramRows = 64;

struct ColPtr {
    const double* p;
    int64_t ld;
};

__device__ __forceinline__ ColPtr col_ptr(const ColBlocks& C, int a) {
    if (a >= C.ncols()) return ColPtr{nullptr, 0};
    int u = 0;
    while (u + 1 < C.nblk && a >= C.w[u]) {
        a -= C.w[u];
        ++u;
    }
    return ColPtr{C.p[u] + a, C.ld[u]};
}

__global__ void __launch_bounds__(256) k_gram_tiles(int64_t m, ColBlocks L, ColBlocks R, double* partial) {
    __shared__ double Ls[kGramRows][33];
    __shared__ double Rs[kGramRows][33];
    const int La = L.ncols(), Rb = R.ncols();
    const int a0 = blockIdx.y * 32, b0 = blockIdx.z * 32;
    const int64_t r0 = (int64_t)blockIdx.x * kGramRows;
    const int cc = threadIdx.x % 32, rr0 = threadIdx.x / 32;  // loader: column cc, rows rr0 + 8 q
    const ColPtr lp = col_ptr(L, a0 + cc), rp = col_ptr(R, b0 + cc);
    double lv[kGramRows / 8], rv[kGramRows / 8];
#pragma unroll
    for (int q = 0; q < kGramRows / 8; ++q) {
        const int64_t i = r0 + rr0 + 8 * q;
        lv[q] = (lp.p && i < m) ? lp.p[i * lp.ld] : 0.0;
        rv[q] = (rp.p && i < m) ? rp.p[i * rp.ld] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kGramRows / 8; ++q) {
        Ls[rr0 + 8 * q][cc] = lv[q];
        Rs[rr0 + 8 * q][cc] = rv[q];
    }
    __syncthreads();
    const int ta = threadIdx.x / 8, tb = (threadIdx.x % 8) * 4;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 8
    for (int rr = 0; rr < kGramRows; ++rr) {
        const double l = Ls[rr][ta];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += l * Rs[rr][tb + q];
    }
    const int a = a0 + ta;
    if (a < La)
        for (int q = 0; q < 4; ++q) {
            const int b = b0 + tb + q;
            if (b < Rb) partial[((int64_t)blockIdx.x * La + a) * Rb + b] = acc[q];
        }
}

__global__ void k_chunk_sum(int nchunks, int64_t width, const double* partial, double* out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= width) return;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += partial[(int64_t)c * width + j];
    out[j] = s;
}

int64_t gram_tiles_partial_size(int64_t m, int La, int Rb) {
    return std::max<int64_t>(1, (m + kGramRows - 1) / kGramRows) * La * Rb;
}

void launch_gram_tiles(int64_t m, const ColBlocks& L, const ColBlocks& R, double* partial, double* G,
                       cudaStream_t s) {
    const int La = L.ncols(), Rb = R.ncols();
    if (La <= 0 || Rb <= 0) return;
    const int nch = (int)std::max<int64_t>(1, (m + kGramRows - 1) / kGramRows);
    dim3 grid(nch, (La + 31) / 32, (Rb + 31) / 32);
    if (m > 0) {
        k_gram_tiles<<<grid, 256, 0, s>>>(m, L, R, partial);
        NAS_CHECK_LAUNCH();
    } else {
        NAS_CUDA(cudaMemsetAsync(partial, 0, sizeof(double) * La * Rb, s));
    }
    k_chunk_sum<<<grid_of((int64_t)La * Rb, 128), 128, 0, s>>>(m > 0 ? nch : 1, (int64_t)La * Rb, partial, G);
    NAS_CHECK_LAUNCH();
}

void launch_arrow_apply(const ArrowDev& F, int w, const double* X, double* Y, double* partial, double* G,
                        cudaStream_t s) {
    if (F.nH > 0) {
        k_arrow_rows<<<grid_of(F.nH * w, 256), 256, 0, s>>>(F, w, X, Y);
        NAS_CHECK_LAUNCH();
    }
    if (F.Na > 0) {
        ColBlocks L = ColBlocks::one(F.Bd, F.Na, F.Na);
        ColBlocks R = ColBlocks::one(X, w, w);
        launch_gram_tiles(F.nH, L, R, partial, G, s);
        k_arrow_border<<<grid_of((int64_t)F.Na * w, 128), 128, 0, s>>>(F, w, X, G, Y);
        NAS_CHECK_LAUNCH();
    }
}

// ---- Y[i][j] = alpha sum_a S(i,a) C[a][j] + beta Y[i][j]   (Y row-major [m][kout])
__global__ void k_cols_mult(int64_t m, ColBlocks S, const double* C, int kout, double alpha, double beta, double* Y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * kout) return;
    const int64_t i = t / kout;
    const int j = (int)(t - i * kout);
    double acc = 0.0;
    int a = 0;
    for (int u = 0; u < S.nblk; ++u) {
        const double* row = S.p[u] + i * S.ld[u];
        for (int c = 0; c < S.w[u]; ++c, ++a) acc += row[c] * C[(int64_t)a * kout + j];
    }
    Y[t] = beta == 0.0 ? alpha * acc : alpha * acc + beta * Y[t];
}

void launch_cols_mult(int64_t m, const ColBlocks& S, const double* C, int kout, double alpha, double beta,
                      double* Y, cudaStream_t s) {
    if (m <= 0 || kout <= 0) return;
    k_cols_mult<<<grid_of(m * kout, 256), 256, 0, s>>>(m, S, C, kout, alpha, beta, Y);
    NAS_CHECK_LAUNCH();
}

// ---- R = AX - BX diag(theta)
__global__ void k_eig_resid(int64_t m, int k, const double* AX, const double* BX, const double* theta, double* R) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * k) return;
    const int j = (int)(t % k);
    R[t] = AX[t] - theta[j] * BX[t];
}

void launch_eig_resid(int64_t m, int k, const double* AX, const double* BX, const double* theta, double* R,
                      cudaStream_t s) {
    if (m * k <= 0) return;
    k_eig_resid<<<grid_of(m * k, 256), 256, 0, s>>>(m, k, AX, BX, theta, R);
    NAS_CHECK_LAUNCH();
}

// ---- columns j of up to three [m][k] arrays scaled by 1/sqrt(nrm[j]) (0 if nrm <= 0)
__global__ void k_inv_sqrt_scale(int64_t m, int k, const double* nrm, double* A1, double* A2, double* A3) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * k) return;
    const double v = nrm[t % k];
    const double f = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
    if (A1) A1[t] *= f;
    if (A2) A2[t] *= f;
    if (A3) A3[t] *= f;
}

void launch_inv_sqrt_scale(int64_t m, int k, const double* nrm, double* A1, double* A2, double* A3,
                           cudaStream_t s) {
    if (m * k <= 0) return;
    k_inv_sqrt_scale<<<grid_of(m * k, 256), 256, 0, s>>>(m, k, nrm, A1, A2, A3);
    NAS_CHECK_LAUNCH();
}

// ---- T[i] = 1 / (A_ii - sigma B_ii) (1 where that is not positive)
__device__ __forceinline__ double arrow_diag(const ArrowDev& F, const int32_t* diag_slot, int64_t i) {
    if (i < F.nH) return diag_slot[i] >= 0 ? F.sval[diag_slot[i]] : 0.0;
    const int64_t a = i - F.nH;
    return F.Cd[a * F.Na + a];
}

__global__ void k_eig_precond(ArrowDev A, ArrowDev B, const int32_t* diag_slot, double sigma, double* T) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.nH + A.Na) return;
    const double d = arrow_diag(A, diag_slot, i) - sigma * arrow_diag(B, diag_slot, i);
    T[i] = d > 0.0 ? 1.0 / d : 1.0;
}

void launch_eig_precond(const ArrowDev& A, const ArrowDev& B, const int32_t* diag_slot, double sigma, double* T,
                        cudaStream_t s) {
    const int64_t m = A.nH + A.Na;
    if (m <= 0) return;
    k_eig_precond<<<grid_of(m, 256), 256, 0, s>>>(A, B, diag_slot, sigma, T);
    NAS_CHECK_LAUNCH();
}


// ---------------------------------------------------------------- Rayleigh-Ritz on the device
// One block solves the small pencil (H, G) of the basis Gram matrices
// (ns <= kRRMax): G = L L^T by Cholesky (status 1 if a squared pivot falls
// below pivot_tol x max diag G: the caller then uses the host fallback),
// Hr = L^-1 H L^-T, all eigenpairs of Hr by the cyclic Jacobi method with the
// round-robin ordering (ns/2 disjoint rotations per round, applied to rows,
// then columns, then the eigenvector matrix), the lowest k (ascending), and
// Y = L^-T Z.  Status 2: Jacobi did not reach the off-diagonal tolerance.
namespace {
constexpr int kRRMax = 80;
constexpr int kRRLd = kRRMax + 1;
constexpr int kRRThreads = 512;
}

int rr_device_max_ns() { return kRRMax; }

static size_t rr_device_smem_bytes() {
    return sizeof(double) * (3 * (size_t)kRRMax * kRRLd + 4 * kRRMax + kRRThreads) + sizeof(int) * (2 * kRRMax + 8);
}

__device__ double rr_block_sum(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kRRThreads) k_rr_small(int ns, int k, const double* GA, const double* GB,
                                                         double pivot_tol, double* Y, double* theta, int* status) {
    extern __shared__ double sm[];
    double* L = sm;                              // G, then its Cholesky factor (lower)
    double* A = L + kRRMax * kRRLd;              // H, then L^-1 H, then reused for V
    double* C = A + kRRMax * kRRLd;              // Hr = L^-1 H L^-T (Jacobi works here)
    double* cs = C + kRRMax * kRRLd;             // rotation cosines [kRRMax/2]
    double* sn = cs + kRRMax;                    // rotation sines
    double* ev = sn + kRRMax;                    // eigenvalues
    double* red = ev + 2 * kRRMax;               // reduction scratch [blockDim]
    int* pr = reinterpret_cast<int*>(red + kRRThreads);  // pair p per slot
    int* qr = pr + kRRMax;                               // pair q per slot
    int* flag = qr + kRRMax;
    const int tid = threadIdx.x, nt = blockDim.x;
    // ---- load and symmetrise
    for (int e = tid; e < ns * ns; e += nt) {
        const int i = e / ns, j = e % ns;
        L[i * kRRLd + j] = 0.5 * (GB[i * ns + j] + GB[j * ns + i]);
        A[i * kRRLd + j] = 0.5 * (GA[i * ns + j] + GA[j * ns + i]);
    }
    if (tid == 0) flag[0] = 0;
    __syncthreads();
    double gmax = 0.0;
    for (int i = 0; i < ns; ++i) gmax = fmax(gmax, L[i * kRRLd + i]);
    // ---- Cholesky (right-looking)
    for (int j = 0; j < ns; ++j) {
        if (tid == 0) {
            const double piv = L[j * kRRLd + j];
            if (!(piv >= pivot_tol * gmax) || !(piv > 0.0)) flag[0] = 1;
            L[j * kRRLd + j] = sqrt(fmax(piv, 0.0));
        }
        __syncthreads();
        if (flag[0]) {
            if (tid == 0) *status = 1;
            return;
        }
        const double d = L[j * kRRLd + j];
        for (int i = j + 1 + tid; i < ns; i += nt) L[i * kRRLd + j] /= d;
        __syncthreads();
        const int r = ns - j - 1;
        for (int e = tid; e < r * r; e += nt) {
            const int i = j + 1 + e / r, l = j + 1 + e % r;
            if (l <= i) L[i * kRRLd + l] -= L[i * kRRLd + j] * L[l * kRRLd + j];
        }
        __syncthreads();
    }
    // ---- A <- L^-1 A (forward substitution, all columns at once)
    for (int i = 0; i < ns; ++i) {
        for (int c = tid; c < ns; c += nt) {
            double s = A[i * kRRLd + c];
            for (int p = 0; p < i; ++p) s -= L[i * kRRLd + p] * A[p * kRRLd + c];
            A[i * kRRLd + c] = s / L[i * kRRLd + i];
        }
        __syncthreads();
    }
    // ---- C <- L^-1 A^T  (= L^-1 H L^-T)
    for (int i = 0; i < ns; ++i) {
        for (int c = tid; c < ns; c += nt) {
            double s = A[c * kRRLd + i];
            for (int p = 0; p < i; ++p) s -= L[i * kRRLd + p] * C[p * kRRLd + c];
            C[i * kRRLd + c] = s / L[i * kRRLd + i];
        }
        __syncthreads();
    }
    for (int e = tid; e < ns * ns; e += nt) {
        const int i = e / ns, j = e % ns;
        if (j < i) {
            const double v = 0.5 * (C[i * kRRLd + j] + C[j * kRRLd + i]);
            C[i * kRRLd + j] = v;
            C[j * kRRLd + i] = v;
        }
    }
    // ---- V <- I (in A)
    for (int e = tid; e < ns * ns; e += nt) A[(e / ns) * kRRLd + e % ns] = (e / ns == e % ns) ? 1.0 : 0.0;
    __syncthreads();
    // ---- cyclic Jacobi, round-robin pairs over n2 = ns rounded up to even
    const int n2 = ns + (ns & 1);
    const int half = n2 / 2;
    double fro2 = 0.0;
    {
        double s = 0.0;
        for (int e = tid; e < ns * ns; e += nt) {
            const double v = C[(e / ns) * kRRLd + e % ns];
            s += v * v;
        }
        fro2 = rr_block_sum(s, red);
    }
    bool converged = false;
    for (int sweep = 0; sweep < 30 && !converged; ++sweep) {
        double off = 0.0;
        for (int e = tid; e < ns * ns; e += nt) {
            const int i = e / ns, j = e % ns;
            if (i != j) off += C[i * kRRLd + j] * C[i * kRRLd + j];
        }
        off = rr_block_sum(off, red);
        if (off <= 1e-28 * fro2) {  // off-diagonal norm <= 1e-14 of the Frobenius norm
            converged = true;
            break;
        }
        for (int round = 0; round < n2 - 1; ++round) {
            // pairs of this round: slot 0 pairs the fixed index n2-1 with `round`;
            // slot t pairs (round + t) and (round - t) mod (n2 - 1)
            for (int t = tid; t < half; t += nt) {
                int p, q;
                if (t == 0) {
                    p = round;
                    q = n2 - 1;
                } else {
                    p = (round + t) % (n2 - 1);
                    q = (round - t + (n2 - 1)) % (n2 - 1);
                }
                if (p > q) {
                    const int x = p;
                    p = q;
                    q = x;
                }
                double c = 1.0, s = 0.0;
                if (q < ns) {
                    const double apq = C[p * kRRLd + q];
                    if (apq != 0.0) {
                        const double app = C[p * kRRLd + p], aqq = C[q * kRRLd + q];
                        const double zeta = (aqq - app) / (2.0 * apq);
                        const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = c * tt;
                    }
                }
                pr[t] = p;
                qr[t] = q;
                cs[t] = c;
                sn[t] = s;
            }
            __syncthreads();
            // rows p, q of C
            for (int e = tid; e < half * ns; e += nt) {
                const int t = e / ns, j = e % ns;
                const int p = pr[t], q = qr[t];
                if (q >= ns || sn[t] == 0.0) continue;
                const double c = cs[t], s = sn[t];
                const double a = C[p * kRRLd + j], b = C[q * kRRLd + j];
                C[p * kRRLd + j] = c * a - s * b;
                C[q * kRRLd + j] = s * a + c * b;
            }
            __syncthreads();
            // columns p, q of C and of V
            for (int e = tid; e < half * ns; e += nt) {
                const int t = e / ns, j = e % ns;
                const int p = pr[t], q = qr[t];
                if (q >= ns || sn[t] == 0.0) continue;
                const double c = cs[t], s = sn[t];
                const double a = C[j * kRRLd + p], b = C[j * kRRLd + q];
                C[j * kRRLd + p] = c * a - s * b;
                C[j * kRRLd + q] = s * a + c * b;
                const double va = A[j * kRRLd + p], vb = A[j * kRRLd + q];
                A[j * kRRLd + p] = c * va - s * vb;
                A[j * kRRLd + q] = s * va + c * vb;
            }
            __syncthreads();
        }
    }
    if (!converged) {
        if (tid == 0) *status = 2;
        return;
    }
    // ---- lowest k eigenpairs in ascending order (rank of each diagonal entry)
    for (int i = tid; i < ns; i += nt) {
        const double v = C[i * kRRLd + i];
        int rank = 0;
        for (int j = 0; j < ns; ++j) {
            const double w = C[j * kRRLd + j];
            rank += (w < v || (w == v && j < i)) ? 1 : 0;
        }
        if (rank < k) {
            ev[rank] = v;
            pr[rank] = i;
        }
    }
    __syncthreads();
    // ---- Y = L^-T Z (backward substitution, k columns in parallel); Y [ns][k]
    for (int i = ns - 1; i >= 0; --i) {
        for (int c = tid; c < k; c += nt) {
            double s = A[i * kRRLd + pr[c]];
            for (int p = i + 1; p < ns; ++p) s -= L[p * kRRLd + i] * Y[p * k + c];
            Y[i * k + c] = s / L[i * kRRLd + i];
        }
        __syncthreads();
    }
    for (int c = tid; c < k; c += nt) theta[c] = ev[c];
    if (tid == 0) *status = 0;
}

void launch_rr_small(int ns, int k, const double* GA, const double* GB, double pivot_tol, double* Y, double* theta,
                     int* status, cudaStream_t s) {
    if (ns > kRRMax || k > ns || k < 1) fail(NAS_E_INVALID_ARG, "device Rayleigh-Ritz size");
    static std::mutex mu;
    static bool attr_set[64] = {false};
    int dev = 0;
    NAS_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= 64) fail(NAS_E_INVALID_ARG, "device id");
        if (!attr_set[dev]) {
            NAS_CUDA(cudaFuncSetAttribute(k_rr_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)rr_device_smem_bytes()));
            attr_set[dev] = true;
        }
    }
    k_rr_small<<<1, kRRThreads, rr_device_smem_bytes(), s>>>(ns, k, GA, GB, pivot_tol, Y, theta, status);
    NAS_CHECK_LAUNCH();
}

}  // namespace nas

// Device kernels of the LOBPCG solver for the small pencil F_A U = lambda F_B U
// of Algorithm 3 (F_A U = lambda F_B U, Sec. 3.3).  Both matrices have the arrow structure of the
// augmented basis {I phi_a} + {u^_j}: a sparse coarse block (CSR over the
// coarse unknowns), a dense border [nH][Na] and a dense corner [Na][Na].  The
// block vectors are row-major [m][w] with m = nH + Na.  Every sum runs in a
// fixed order (per-chunk partial sums, then an ordered final pass), so results
// are bit-reproducible.
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

// ---- both matrices of the pencil at once (same coarse CSR pattern): YA = A X, YB = B X
__global__ void k_arrow_rows2(ArrowDev A, ArrowDev B, int w, const double* X, double* YA, double* YB) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.nH * w) return;
    const int64_t i = t / w;
    const int j = (int)(t - i * w);
    double a = 0.0, b = 0.0;
    for (int p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
        const double x = X[(int64_t)A.col[p] * w + j];
        a += A.sval[p] * x;
        b += B.sval[p] * x;
    }
    const double* xa = X + A.nH * w + j;
    for (int q = 0; q < A.Na; ++q) {
        const double x = xa[(int64_t)q * w];
        a += A.Bd[i * A.Na + q] * x;
        b += B.Bd[i * A.Na + q] * x;
    }
    YA[t] = a;
    YB[t] = b;
}

// border rows of both: G = [Bd_A | Bd_B]^T X_H ([2 Na][w])
__global__ void k_arrow_border2(ArrowDev A, ArrowDev B, int w, const double* X, const double* G, double* YA,
                                double* YB) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.Na * w) return;
    const int a = t / w, j = t - (t / w) * w;
    double ya = G[t], yb = G[A.Na * w + t];
    const double* xa = X + A.nH * w + j;
    for (int q = 0; q < A.Na; ++q) {
        const double x = xa[(int64_t)q * w];
        ya += A.Cd[a * A.Na + q] * x;
        yb += B.Cd[a * A.Na + q] * x;
    }
    YA[(A.nH + a) * w + j] = ya;
    YB[(A.nH + a) * w + j] = yb;
}

void launch_arrow_apply2(const ArrowDev& A, const ArrowDev& B, int w, const double* X, double* YA, double* YB,
                         double* partial, double* G, cudaStream_t s) {
    if (A.ptr != B.ptr || A.col != B.col || A.nH != B.nH || A.Na != B.Na)
        fail(NAS_E_INVALID_ARG, "arrow pair: the two matrices must share the pattern");
    if (A.nH > 0) {
        k_arrow_rows2<<<grid_of(A.nH * w, 256), 256, 0, s>>>(A, B, w, X, YA, YB);
        NAS_CHECK_LAUNCH();
    }
    if (A.Na > 0) {
        ColBlocks L = ColBlocks::one(A.Bd, A.Na, A.Na);
        L.add(B.Bd, A.Na, A.Na);
        ColBlocks R = ColBlocks::one(X, w, w);
        launch_gram_tiles(A.nH, L, R, partial, G, s);
        k_arrow_border2<<<grid_of((int64_t)A.Na * w, 128), 128, 0, s>>>(A, B, w, X, G, YA, YB);
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

// ---- dst[i][q] = src[i][idx[q]] (src [m][k], dst [m][kq])
__global__ void k_gather_cols(int64_t m, int k, int kq, const int* idx, const double* src, double* dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * kq) return;
    const int64_t i = t / kq;
    const int q = (int)(t - i * kq);
    dst[t] = src[i * k + idx[q]];
}

void launch_gather_cols(int64_t m, int k, int kq, const int* idx, const double* src, double* dst, cudaStream_t s) {
    if (m * kq <= 0) return;
    k_gather_cols<<<grid_of(m * kq, 256), 256, 0, s>>>(m, k, kq, idx, src, dst);
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

}  // namespace nas

namespace nas {

// ---- preconditioner with a dense coarse block:
//   W[i][j] = sum_b T[i][b] R[b][j]   (i < nH; T FP32 [nH][nH], FP32 products and sums)
//   W[i][j] = Dinv[i] R[i][j]        (nH <= i < m)
// Stage 1, grid (row blocks of kPcRows, kPcSplit, column groups of kPcK):
// block (rb, sp, cg) multiplies 128 rows of T by 32 columns of the rows of R
// in its share of the b range, 32 b at a time:
// the 128 x 32 tile of T (coalesced row segments) and the 32 x 32 tile of R
// (converted to FP32) are staged in shared memory, and each thread keeps a
// 4 x 4 block of outputs in registers (rows 4 ty .. 4 ty + 3, columns
// 4 tx .. 4 tx + 3), reading four T values and four R values as float4 per
// step of b (16 multiply-adds per two vector loads).  Stage 2 adds the
// kPcSplit partial products in order.  FP32 is enough for a preconditioner
// (a fixed symmetric positive definite operator close to an inverse).
static const int kPcRows = 128;
static const int kPcK = 32;
static const int kPcSplit = 16;
static const int kPcLd = kPcK + 4;  // row pitch of the T tile: float4-aligned, conflict-free

__global__ void __launch_bounds__(256) k_dense_precond_part(int64_t nH, int k, const float* T, const double* R,
                                                            float* part) {
    __shared__ __align__(16) float Ts[kPcRows][kPcLd];
    __shared__ __align__(16) float Rs[kPcK][kPcK];
    const int64_t r0 = (int64_t)blockIdx.x * kPcRows;
    const int64_t span = (nH + kPcSplit - 1) / kPcSplit;
    const int64_t bbeg = (int64_t)blockIdx.y * span;
    const int64_t bend = bbeg + span < nH ? bbeg + span : nH;
    const int c0 = (int)blockIdx.z * kPcK;   // this block's group of kPcK columns
    const int tx = threadIdx.x % 8;   // columns c0 + 4 tx .. c0 + 4 tx + 3
    const int ty = threadIdx.x / 8;   // rows 4 ty .. 4 ty + 3
    float acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
    for (int64_t b0 = bbeg; b0 < bend; b0 += kPcK) {
        // T tile: element e -> (row e / 32, b e % 32); a warp reads 32 consecutive b of one row
#pragma unroll 4
        for (int e = threadIdx.x; e < kPcRows * kPcK; e += blockDim.x) {
            const int rr = e / kPcK, cc = e % kPcK;
            const int64_t i = r0 + rr, b = b0 + cc;
            Ts[rr][cc] = (i < nH && b < bend) ? T[i * nH + b] : 0.f;
        }
        for (int e = threadIdx.x; e < kPcK * kPcK; e += blockDim.x) {
            const int rr = e / kPcK, cc = e % kPcK;
            const int64_t bj = b0 + rr;
            const int cg = c0 + cc;
            Rs[rr][cc] = (bj < bend && cg < k) ? (float)R[bj * k + cg] : 0.f;
        }
        __syncthreads();
#pragma unroll 2
        for (int bb = 0; bb < kPcK; bb += 4) {
            float4 tv[4], rv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) tv[q] = *reinterpret_cast<const float4*>(&Ts[4 * ty + q][bb]);
#pragma unroll
            for (int u = 0; u < 4; ++u) rv[u] = *reinterpret_cast<const float4*>(&Rs[bb + u][4 * tx]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float t4[4] = {tv[q].x, tv[q].y, tv[q].z, tv[q].w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    acc[q][0] += t4[u] * rv[u].x;
                    acc[q][1] += t4[u] * rv[u].y;
                    acc[q][2] += t4[u] * rv[u].z;
                    acc[q][3] += t4[u] * rv[u].w;
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = r0 + 4 * ty + q;
        if (i >= nH) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = c0 + 4 * tx + c;
            if (j < k) part[((int64_t)blockIdx.y * nH + i) * k + j] = acc[q][c];
        }
    }
}

__global__ void k_dense_precond_sum(int64_t nH, int64_t m, int k, const float* part, const double* R,
                                    const double* Dinv, double* W) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * k) return;
    const int64_t i = t / k;
    if (i < nH) {
        float acc = 0.f;
        for (int sp = 0; sp < kPcSplit; ++sp) acc += part[(int64_t)sp * nH * k + t];
        W[t] = (double)acc;
    } else {
        W[t] = Dinv[i] * R[t];
    }
}

int64_t dense_precond_part_size(int64_t nH, int k) { return (int64_t)kPcSplit * nH * k; }

void launch_dense_precond(int64_t nH, int64_t m, int k, const float* T, const double* R, const double* Dinv,
                          float* part, double* W, cudaStream_t s) {
    if (k < 1 || k > 1024) fail(NAS_E_INVALID_ARG, "dense preconditioner: block width out of range");
    if (m <= 0) return;
    if (nH > 0) {
        dim3 grid((unsigned)((nH + kPcRows - 1) / kPcRows), kPcSplit, (unsigned)((k + kPcK - 1) / kPcK));
        k_dense_precond_part<<<grid, 256, 0, s>>>(nH, k, T, R, part);
        NAS_CHECK_LAUNCH();
    }
    k_dense_precond_sum<<<grid_of(m * k, 256), 256, 0, s>>>(nH, m, k, part, R, Dinv, W);
    NAS_CHECK_LAUNCH();
}

}  // namespace nas

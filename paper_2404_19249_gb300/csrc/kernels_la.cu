// Sparse and dense linear algebra kernels of the step: CSR SpMM with the N
// right-hand sides interleaved (row-major [n][N], so one row of X is one
// contiguous segment), block PCG updates with per-column scalars kept on the
// device, deterministic column-wise dot products and tall-skinny Gram
// products, the transposed transfer I^T, the reconstruction
// Psi = I u_H + U^ alpha, the two Galerkin gathers of A_H = I^T A I, and the
// Anderson-mixing reductions.  All reductions are two-stage with a fixed
// order (per-block partials, then one ordered pass), never atomics.
#include <algorithm>

#include "kernels.h"

namespace nas {

static const int kRedBlocks = 1216;  // 8 x 152 SMs: grid of the two-stage reductions

// ------------------------------------------------------------------ SpMV
// N == 1: 8 lanes per row, strided over the row's nonzeros, shuffle reduction
// in a fixed order.
__global__ void __launch_bounds__(256) k_spmv8(Csr A, const double* __restrict__ X, double* __restrict__ Y,
                                              double alpha, double beta) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t row = t >> 3;
    int lane = threadIdx.x & 7;
    bool valid = row < A.n_rows;
    double acc = 0.0;
    if (valid) {
        int p1 = A.rowptr[row + 1];
        for (int p = A.rowptr[row] + lane; p < p1; p += 8) acc += A.val[p] * X[A.col[p]];
    }
    acc += __shfl_down_sync(0xffffffffu, acc, 4, 8);
    acc += __shfl_down_sync(0xffffffffu, acc, 2, 8);
    acc += __shfl_down_sync(0xffffffffu, acc, 1, 8);
    if (valid && lane == 0) {
        double y = alpha * acc;
        if (beta != 0.0) y += beta * Y[row];
        Y[row] = y;
    }
}

void launch_spmm(const Csr& A, int N, const double* X, double* Y, double alpha, double beta,
                 cudaStream_t s) {
    if (A.n_rows <= 0) return;
    if (N == 1) {
        k_spmv8<<<grid_for(A.n_rows * 8, 256), 256, 0, s>>>(A, X, Y, alpha, beta);
        NAS_CHECK_LAUNCH();
    } else {
        launch_spmm_tuned(A, N, X, Y, alpha, beta, s);   // kernels_spmm.cu
    }
}

// ------------------------------------------------------------------ ordered reductions
// final pass: out[j] = sum_b partial[b][j] for j < width.  One warp per
// output: lane l sums b = l, l+32, ... in order, then a fixed shuffle tree, so
// the order is fixed and the loads of a lane are independent (no serial chain
// of nblocks dependent steps).
__global__ void k_reduce_partials(int nblocks, int64_t width, const double* partial, double* out) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (j >= width) return;  // warp-uniform
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(int64_t)b * width + j];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) out[j] = s;
}

static void reduce_partials(int nblocks, int64_t width, const double* partial, double* out, cudaStream_t s) {
    k_reduce_partials<<<grid_for(width * 32, 256), 256, 0, s>>>(nblocks, width, partial, out);
    NAS_CHECK_LAUNCH();
}

int64_t reduce_partial_size(int64_t width) { return (int64_t)kRedBlocks * width; }
int64_t gram_partial_size(int64_t width) { return (int64_t)kRedBlocks * width; }

struct ColDotArgs {
    const double* X[4];
    const double* Y[4];
};

// thread t of a block owns column c = t % N and row offset r = t / N
// (R = 256 / N rows per pass); blocks stride over rows.  Per block, column c
// is summed over r = 0..R-1 in order.
__global__ void __launch_bounds__(256) k_coldots(int64_t n, int N, int npairs, ColDotArgs a, const double* w,
                                                double* partial) {
    __shared__ double sh[4][256];
    int R = 256 / N;
    int t = threadIdx.x;
    int c = t % N, r = t / N;
    double acc[4] = {0, 0, 0, 0};
    if (r < R) {
        for (int64_t row = (int64_t)blockIdx.x * R + r; row < n; row += (int64_t)gridDim.x * R) {
            double wi = w ? w[row] : 1.0;
            int64_t idx = row * N + c;
            for (int k = 0; k < npairs; ++k) acc[k] += wi * a.X[k][idx] * a.Y[k][idx];
        }
    }
    for (int k = 0; k < npairs; ++k) sh[k][t] = acc[k];
    __syncthreads();
    if (t < N) {
        for (int k = 0; k < npairs; ++k) {
            double s = 0.0;
            for (int rr = 0; rr < R; ++rr) s += sh[k][rr * N + t];
            partial[(int64_t)blockIdx.x * npairs * N + k * N + t] = s;
        }
    }
}

void launch_coldots(int64_t n, int N, int npairs, const double* const* X, const double* const* Y,
                    const double* w, double* partial, double* out, cudaStream_t s) {
    if (N < 1 || N > 256 || npairs < 1 || npairs > 4) fail(NAS_E_INVALID_ARG, "coldots width");
    ColDotArgs a{};
    for (int k = 0; k < npairs; ++k) {
        a.X[k] = X[k];
        a.Y[k] = Y[k];
    }
    int R = 256 / N;
    int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (n + R - 1) / R));
    k_coldots<<<nb, 256, 0, s>>>(n, N, npairs, a, w, partial);
    NAS_CHECK_LAUNCH();
    int64_t width = (int64_t)npairs * N;
    reduce_partials(nb, width, partial, out, s);
}

// ------------------------------------------------------------------ PCG scalars and updates
__global__ void k_pcg_alpha(PcgCols c) {
    int j = threadIdx.x;
    if (j >= c.N) return;
    if (!c.active[j]) {
        c.alpha[j] = 0.0;
        return;
    }
    double pq = c.pq[j];
    if (!(pq > 0.0) || !isfinite(pq)) {
        *c.breakdown = 1;
        c.active[j] = 0;
        c.alpha[j] = 0.0;
        return;
    }
    c.alpha[j] = c.rz[j] / pq;
}

__global__ void k_pcg_beta(PcgCols c) {
    int j = threadIdx.x;
    if (j >= c.N) return;
    if (!c.active[j]) {
        c.beta[j] = 0.0;
        return;
    }
    double rzn = c.rz_new[j];
    if (!isfinite(rzn)) {
        *c.breakdown = 1;
        c.active[j] = 0;
        return;
    }
    c.beta[j] = c.rz[j] != 0.0 ? rzn / c.rz[j] : 0.0;
    c.rz[j] = rzn;
    if (c.rr[j] <= c.tol2 * c.bb[j]) c.active[j] = 0;
}

void launch_pcg_alpha(const PcgCols& c, cudaStream_t s) {
    k_pcg_alpha<<<1, 256, 0, s>>>(c);
    NAS_CHECK_LAUNCH();
}
void launch_pcg_beta(const PcgCols& c, cudaStream_t s) {
    k_pcg_beta<<<1, 256, 0, s>>>(c);
    NAS_CHECK_LAUNCH();
}

__global__ void k_pcg_update(int64_t n, int N, const double* alpha, const int* active, const double* P,
                             const double* Q, const double* Dinv, double* X, double* R, double* Z) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * N) return;
    int64_t i = t / N;
    int c = (int)(t - i * N);
    if (!active[c]) return;
    double a = alpha[c];
    X[t] += a * P[t];
    double r = R[t] - a * Q[t];
    R[t] = r;
    Z[t] = Dinv[i] * r;
}

void launch_pcg_update(int64_t n, int N, const double* alpha, const int* active, const double* P,
                       const double* Q, const double* Dinv, double* X, double* R, double* Z,
                       cudaStream_t s) {
    if (n <= 0) return;
    k_pcg_update<<<grid_for(n * N, 256), 256, 0, s>>>(n, N, alpha, active, P, Q, Dinv, X, R, Z);
    NAS_CHECK_LAUNCH();
}

__global__ void k_pcg_direction(int64_t n, int N, const double* beta, const int* active, const double* Z,
                                double* P) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * N) return;
    int c = (int)(t % N);
    if (!active[c]) return;
    P[t] = Z[t] + beta[c] * P[t];
}

void launch_pcg_direction(int64_t n, int N, const double* beta, const int* active, const double* Z,
                          double* P, cudaStream_t s) {
    if (n <= 0) return;
    k_pcg_direction<<<grid_for(n * N, 256), 256, 0, s>>>(n, N, beta, active, Z, P);
    NAS_CHECK_LAUNCH();
}

__global__ void k_scale_cols(int64_t n, int N, const double* sc, double* Y) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * N) return;
    Y[t] *= sc[t % N];
}

void launch_scale_cols(int64_t n, int N, const double* sc, double* Y, cudaStream_t s) {
    if (n <= 0) return;
    k_scale_cols<<<grid_for(n * N, 256), 256, 0, s>>>(n, N, sc, Y);
    NAS_CHECK_LAUNCH();
}

__global__ void k_scale_rows(int64_t n, int N, const double* Dinv, const double* R, double* Z) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * N) return;
    Z[t] = Dinv[t / N] * R[t];
}

void launch_scale_rows(int64_t n, int N, const double* Dinv, const double* R, double* Z, cudaStream_t s) {
    if (n <= 0) return;
    k_scale_rows<<<grid_for(n * N, 256), 256, 0, s>>>(n, N, Dinv, R, Z);
    NAS_CHECK_LAUNCH();
}

__global__ void k_sub_from(int64_t cnt, const double* B, double* R) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) R[t] = B[t] - R[t];
}

void launch_sub_from(int64_t cnt, const double* B, double* R, cudaStream_t s) {
    if (cnt <= 0) return;
    k_sub_from<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, B, R);
    NAS_CHECK_LAUNCH();
}

__global__ void k_axpby(int64_t cnt, double a, const double* x, double b, const double* y, double* out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) out[t] = a * x[t] + (y ? b * y[t] : 0.0);
}

void launch_axpby(int64_t cnt, double a, const double* x, double b, const double* y, double* out,
                  cudaStream_t s) {
    if (cnt <= 0) return;
    k_axpby<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, a, x, b, y, out);
    NAS_CHECK_LAUNCH();
}

__global__ void k_inv_diag(Csr A, double* Dinv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n_rows) return;
    double d = 0.0;
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p)
        if (A.col[p] == i) d = A.val[p];
    Dinv[i] = d != 0.0 ? 1.0 / d : 0.0;
}

void launch_inv_diag(const Csr& A, double* Dinv, cudaStream_t s) {
    if (A.n_rows <= 0) return;
    k_inv_diag<<<grid_for(A.n_rows, 256), 256, 0, s>>>(A, Dinv);
    NAS_CHECK_LAUNCH();
}

__global__ void k_combine3(int64_t nnz, double a, const double* v1, double b, const double* v2, double c,
                           const double* v3, double* out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    double s = a * v1[t] + b * v2[t];
    if (v3) s += c * v3[t];
    out[t] = s;
}

void launch_combine3(int64_t nnz, double a, const double* v1, double b, const double* v2, double c,
                     const double* v3, double* out, cudaStream_t s) {
    if (nnz <= 0) return;
    k_combine3<<<grid_for(nnz, 256), 256, 0, s>>>(nnz, a, v1, b, v2, c, v3, out);
    NAS_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ Gram X^T Y
// Blocks stride over 32-row tiles staged in shared memory; thread t owns
// entries ab = t, t+256, ... (at most 16), summed over the tile rows in order.
__global__ void __launch_bounds__(256) k_gram(int64_t n, int Nx, const double* X, int Ny, const double* Y,
                                             double* partial) {
    extern __shared__ double smem[];
    double* xs = smem;             // [32][Nx]
    double* ys = smem + 32 * Nx;   // [32][Ny]
    const int W = Nx * Ny;
    double acc[16];
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    for (int64_t r0 = (int64_t)blockIdx.x * 32; r0 < n; r0 += (int64_t)gridDim.x * 32) {
        int rows = (n - r0) < 32 ? (int)(n - r0) : 32;
        for (int j = threadIdx.x; j < 32 * Nx; j += blockDim.x)
            xs[j] = (j / Nx < rows) ? X[r0 * Nx + j] : 0.0;
        for (int j = threadIdx.x; j < 32 * Ny; j += blockDim.x)
            ys[j] = (j / Ny < rows) ? Y[r0 * Ny + j] : 0.0;
        __syncthreads();
        int k = 0;
        for (int ab = threadIdx.x; ab < W; ab += blockDim.x, ++k) {
            int a = ab / Ny, b = ab - a * Ny;
            double s = 0.0;
            for (int r = 0; r < 32; ++r) s += xs[r * Nx + a] * ys[r * Ny + b];
            acc[k] += s;
        }
        __syncthreads();
    }
    int k = 0;
    for (int ab = threadIdx.x; ab < W; ab += blockDim.x, ++k) partial[(int64_t)blockIdx.x * W + ab] = acc[k];
}

void launch_gram(int64_t n, int Nx, const double* X, int Ny, const double* Y, double* partial, double* G,
                 cudaStream_t s) {
    int64_t W = (int64_t)Nx * Ny;
    if (W < 1 || W > 16 * 256) fail(NAS_E_INVALID_ARG, "gram width");
    int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (n + 31) / 32));
    size_t sm = sizeof(double) * 32 * (Nx + Ny);
    k_gram<<<nb, 256, sm, s>>>(n, Nx, X, Ny, Y, partial);
    NAS_CHECK_LAUNCH();
    reduce_partials(nb, W, partial, G, s);
}

// Symmetric Gram G = X^T Y (known symmetric, e.g. U^T (A U) with A symmetric):
// only the N (N + 1) / 2 entries a <= b are summed, in packed order
// p = a N - a (a - 1) / 2 + (b - a); same tiles and per-entry order as k_gram.
__global__ void __launch_bounds__(256) k_gram_sym(int64_t n, int N, const double* X, const double* Y,
                                                 double* partial) {
    extern __shared__ double smem[];
    double* xs = smem;             // [32][N]
    double* ys = smem + 32 * N;    // [32][N]
    short2* tab = reinterpret_cast<short2*>(smem + 64 * N);   // packed index -> (a, b)
    const int P = N * (N + 1) / 2;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        int a = 0, off = 0;
        while (off + (N - a) <= p) {
            off += N - a;
            ++a;
        }
        tab[p] = make_short2((short)a, (short)(a + p - off));
    }
    double acc[16];
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    __syncthreads();
    for (int64_t r0 = (int64_t)blockIdx.x * 32; r0 < n; r0 += (int64_t)gridDim.x * 32) {
        int rows = (n - r0) < 32 ? (int)(n - r0) : 32;
        for (int j = threadIdx.x; j < 32 * N; j += blockDim.x) {
            xs[j] = (j / N < rows) ? X[r0 * N + j] : 0.0;
            ys[j] = (j / N < rows) ? Y[r0 * N + j] : 0.0;
        }
        __syncthreads();
        int k = 0;
        for (int p = threadIdx.x; p < P; p += blockDim.x, ++k) {
            const short2 ab = tab[p];
            double s = 0.0;
            for (int r = 0; r < 32; ++r) s += xs[r * N + ab.x] * ys[r * N + ab.y];
            acc[k] += s;
        }
        __syncthreads();
    }
    int k = 0;
    for (int p = threadIdx.x; p < P; p += blockDim.x, ++k) partial[(int64_t)blockIdx.x * P + p] = acc[k];
}

// packed upper triangle -> full symmetric [N][N]
__global__ void k_unpack_sym(int N, const double* packed, double* G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * N) return;
    int a = t / N, b = t % N;
    if (a > b) {
        const int tmp = a;
        a = b;
        b = tmp;
    }
    G[t] = packed[a * N - a * (a - 1) / 2 + (b - a)];
}

void launch_gram_sym(int64_t n, int N, const double* X, const double* Y, double* partial, double* G,
                     cudaStream_t s) {
    const int64_t P = (int64_t)N * (N + 1) / 2;
    if (N < 1 || P > 16 * 256) fail(NAS_E_INVALID_ARG, "gram width");
    int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (n + 31) / 32));
    size_t sm = sizeof(double) * 64 * N + sizeof(short2) * P;
    k_gram_sym<<<nb, 256, sm, s>>>(n, N, X, Y, partial);
    NAS_CHECK_LAUNCH();
    double* packed = partial + (int64_t)nb * P;   // the partial buffer holds kRedBlocks x N^2 >= (nb + 1) P
    reduce_partials(nb, P, partial, packed, s);
    k_unpack_sym<<<grid_for((int64_t)N * N, 256), 256, 0, s>>>(N, packed, G);
    NAS_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ transfer products
// one warp per output (a, c): lanes stride over the ~n/nH fine entries of
// coarse row a, then a fixed-order shuffle sum
// I^T Y, stage 1: one warp per piece of an I^T row, lane c holds column c
// (columns beyond 32 in further passes), entries in list order
__global__ void k_transpose_pieces(Pieces pc, const int32_t* trow, const double* tval, int N, const double* Y,
                                   double* partial) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (q >= pc.npieces) return;  // warp-uniform
    const int64_t b = pc.piece_start[q], e = pc.piece_start[q + 1];
    for (int c0 = 0; c0 < N; c0 += 32) {
        const int c = c0 + lane;
        double acc = 0.0;
        if (c < N)
            for (int64_t p = b; p < e; ++p) acc += tval[p] * Y[(int64_t)trow[p] * N + c];
        if (c < N) partial[q * N + c] = acc;
    }
}

// stage 2 of every piece reduction: out[a][c] = sum of the pieces of segment a, in order
__global__ void k_piece_sum(int64_t nseg, const int32_t* seg_piece, int N, const double* partial, double* out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nseg * N) return;
    const int64_t a = t / N;
    const int c = (int)(t - a * N);
    double acc = 0.0;
    for (int q = seg_piece[a]; q < seg_piece[a + 1]; ++q) acc += partial[(int64_t)q * N + c];
    out[t] = acc;
}

void launch_transpose_apply(const Pieces& pc, const int32_t* trow, const double* tval, int N, const double* Y,
                            double* partial, double* out, cudaStream_t s) {
    if (pc.nseg <= 0 || N <= 0) return;
    if (pc.npieces > 0) {
        k_transpose_pieces<<<grid_for(pc.npieces * 32, 256), 256, 0, s>>>(pc, trow, tval, N, Y, partial);
        NAS_CHECK_LAUNCH();
    }
    k_piece_sum<<<grid_for(pc.nseg * N, 256), 256, 0, s>>>(pc.nseg, pc.seg_piece, N, partial, out);
    NAS_CHECK_LAUNCH();
}

// I^T Y for FP32 Y [n][N] and FP32 weights (the FP32 block PCG's coarse
// restriction): per-piece sums in FP64, then the same ordered piece sums
__global__ void k_transpose_pieces_f32(Pieces pc, const int32_t* trow, const float* tval, int N, const float* Y,
                                       double* partial) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (q >= pc.npieces) return;  // warp-uniform
    const int64_t b = pc.piece_start[q], e = pc.piece_start[q + 1];
    for (int c0 = 0; c0 < N; c0 += 32) {
        const int c = c0 + lane;
        double acc = 0.0;
        if (c < N)
            for (int64_t p = b; p < e; ++p) acc += (double)tval[p] * (double)Y[(int64_t)trow[p] * N + c];
        if (c < N) partial[q * N + c] = acc;
    }
}

void launch_transpose_apply_f32(const Pieces& pc, const int32_t* trow, const float* tval, int N, const float* Y,
                                double* partial, double* out, cudaStream_t s) {
    if (pc.nseg <= 0 || N <= 0) return;
    if (pc.npieces > 0) {
        k_transpose_pieces_f32<<<grid_for(pc.npieces * 32, 256), 256, 0, s>>>(pc, trow, tval, N, Y, partial);
        NAS_CHECK_LAUNCH();
    }
    k_piece_sum<<<grid_for(pc.nseg * N, 256), 256, 0, s>>>(pc.nseg, pc.seg_piece, N, partial, out);
    NAS_CHECK_LAUNCH();
}

// Z[i][c] += sum_k w[i][k] Yc[icol[i][k]][c] (prolongation of a coarse block,
// columns of boundary coarse vertices (-1) skipped)
template <typename T>
__global__ void k_prolong_add(int64_t n, int N, const int32_t* icol, const T* ival, const double* Yc, T* Z) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * N) return;
    const int64_t i = t / N;
    const int c = (int)(t - i * N);
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int a = icol[4 * i + k];
        if (a >= 0) acc += (double)ival[4 * i + k] * Yc[(int64_t)a * N + c];
    }
    Z[t] += (T)acc;
}

void launch_prolong_add(int64_t n, int N, const int32_t* icol, const double* ival, const double* Yc, double* Z,
                        cudaStream_t s) {
    if (n <= 0) return;
    k_prolong_add<double><<<grid_for(n * N, 256), 256, 0, s>>>(n, N, icol, ival, Yc, Z);
    NAS_CHECK_LAUNCH();
}
void launch_prolong_add(int64_t n, int N, const int32_t* icol, const float* ival, const double* Yc, float* Z,
                        cudaStream_t s) {
    if (n <= 0) return;
    k_prolong_add<float><<<grid_for(n * N, 256), 256, 0, s>>>(n, N, icol, ival, Yc, Z);
    NAS_CHECK_LAUNCH();
}

__global__ void k_reconstruct(int64_t n, const int32_t* icol, const double* ival, int N, const double* U,
                              int64_t nH, int Na, const double* Uhat, double* Psi) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / N;
    if (i >= n) return;
    int c = (int)(t - i * N);
    double s = 0.0;
    for (int k = 0; k < 4; ++k) {
        int a = icol[4 * i + k];
        if (a >= 0) s += ival[4 * i + k] * U[(int64_t)a * N + c];
    }
    for (int j = 0; j < Na; ++j) s += Uhat[i * Na + j] * U[(nH + j) * N + c];
    Psi[t] = s;
}

void launch_reconstruct(int64_t n, const int32_t* icol, const double* ival, int N, const double* U,
                        int64_t nH, int Na, const double* Uhat, double* Psi, cudaStream_t s) {
    if (n <= 0) return;
    k_reconstruct<<<grid_for(n * N, 256), 256, 0, s>>>(n, icol, ival, N, U, nH, Na, Uhat, Psi);
    NAS_CHECK_LAUNCH();
}

__global__ void k_galerkin1(int64_t nw, const int64_t* ptr, const int32_t* con, const double* A,
                            const int32_t* col, const double* ival, double* W) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nw) return;
    double acc = 0.0;
    for (int64_t k = ptr[s]; k < ptr[s + 1]; ++k) {
        int q = con[k];
        int p = q >> 2;
        acc += A[p] * ival[(int64_t)col[p] * 4 + (q & 3)];
    }
    W[s] = acc;
}

void launch_galerkin1(int64_t nw, const int64_t* ptr, const int32_t* con, const double* A, const int32_t* col,
                      const double* ival, double* W, cudaStream_t s) {
    if (nw <= 0) return;
    k_galerkin1<<<grid_for(nw, 256), 256, 0, s>>>(nw, ptr, con, A, col, ival, W);
    NAS_CHECK_LAUNCH();
}

// one warp per piece of a coarse slot's gather list: lanes stride over the
// piece, then a fixed-order shuffle sum; k_piece_sum adds a slot's pieces
__global__ void k_galerkin2_pieces(Pieces pc, const int32_t* con, const double* W, const int32_t* wrow,
                                   const double* ival, double* partial) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (q >= pc.npieces) return;  // warp-uniform
    double acc = 0.0;
    for (int64_t k = pc.piece_start[q] + lane; k < pc.piece_start[q + 1]; k += 32) {
        const int r = con[k];
        const int sl = r >> 2;
        acc += ival[(int64_t)wrow[sl] * 4 + (r & 3)] * W[sl];
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) partial[q] = acc;
}

void launch_galerkin2(const Pieces& pc, const int32_t* con, const double* W, const int32_t* wrow,
                      const double* ival, double* partial, double* H, cudaStream_t s) {
    if (pc.nseg <= 0) return;
    if (pc.npieces > 0) {
        k_galerkin2_pieces<<<grid_for(pc.npieces * 32, 256), 256, 0, s>>>(pc, con, W, wrow, ival, partial);
        NAS_CHECK_LAUNCH();
    }
    k_piece_sum<<<grid_for(pc.nseg, 256), 256, 0, s>>>(pc.nseg, pc.seg_piece, 1, partial, H);
    NAS_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ Anderson
// Inner products of the history (Sec. 4, Anderson mixing) for m previous
// entries (m <= kAndMax - 1): with d_a = F_m - F_a, the matrix (d_a, d_b) for
// a <= b and the right-hand side (d_a, F_m), weighted by the quadrature
// weights.  The m (m + 1) / 2 + m distinct entries are summed in passes of
// at most kAndPass accumulators per thread (each pass re-reads the history);
// entry e of a pass is (a, b) = code[e], b < 0 meaning the right-hand side.
static const int kAndMax = 16;
static const int kAndPass = 20;
struct AndPass {
    const double* F[kAndMax];
    short2 code[kAndPass];
    int nent;      // entries in this pass
    int first;     // index of the pass's first entry in the full list
    int total;     // entries in the full list
};

__global__ void __launch_bounds__(256) k_anderson_dots(int64_t cnt, int m, AndPass a, const double* w,
                                                      double* partial) {
    __shared__ double sh[kAndPass][256];
    double acc[kAndPass];
#pragma unroll
    for (int k = 0; k < kAndPass; ++k) acc[k] = 0.0;
    const double* Fm = a.F[m];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double fm = Fm[i];
        const double wi = w[i];
        double d[kAndMax];
        for (int q = 0; q < m; ++q) d[q] = fm - a.F[q][i];
#pragma unroll
        for (int k = 0; k < kAndPass; ++k) {
            if (k < a.nent) {
                const short2 c = a.code[k];
                acc[k] += wi * d[c.x] * (c.y >= 0 ? d[c.y] : fm);
            }
        }
    }
    for (int k = 0; k < a.nent; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off)
            for (int k = 0; k < a.nent; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < a.nent; ++k) partial[(int64_t)blockIdx.x * a.total + a.first + k] = sh[k][0];
}

// out: the m x m matrix (row-major, both triangles) followed by the m right-hand sides
__global__ void k_anderson_expand(int m, const double* uniq, double* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * m + m) return;
    if (t < m * m) {
        int a = t / m, b = t % m;
        if (a > b) {
            const int x = a;
            a = b;
            b = x;
        }
        out[t] = uniq[a * m - a * (a - 1) / 2 + (b - a)];   // packed upper triangle
    } else {
        out[t] = uniq[m * (m + 1) / 2 + (t - m * m)];
    }
}

void launch_anderson_dots(int64_t cnt, int m, const double* const* F, const double* w, double* partial,
                          double* out, cudaStream_t s) {
    if (m < 1 || m > kAndMax - 1) fail(NAS_E_INVALID_ARG, "anderson depth");
    std::vector<short2> codes;
    for (int a = 0; a < m; ++a)
        for (int b = a; b < m; ++b) codes.push_back(make_short2((short)a, (short)b));
    for (int a = 0; a < m; ++a) codes.push_back(make_short2((short)a, (short)-1));
    const int total = (int)codes.size();
    int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (cnt + 255) / 256));
    for (int first = 0; first < total; first += kAndPass) {
        AndPass ap{};
        for (int q = 0; q <= m; ++q) ap.F[q] = F[q];
        ap.nent = std::min(kAndPass, total - first);
        ap.first = first;
        ap.total = total;
        for (int k = 0; k < ap.nent; ++k) ap.code[k] = codes[first + k];
        k_anderson_dots<<<nb, 256, 0, s>>>(cnt, m, ap, w, partial);
        NAS_CHECK_LAUNCH();
    }
    double* uniq = partial + (int64_t)nb * total;
    reduce_partials(nb, total, partial, uniq, s);
    k_anderson_expand<<<1, 512, 0, s>>>(m, uniq, out);
    NAS_CHECK_LAUNCH();
}

int64_t anderson_partial_size(int m) {
    const int total = m * (m + 1) / 2 + m;
    return ((int64_t)kRedBlocks + 1) * total;
}

struct MixArgs {
    const double* rin[kAndMax];
    const double* F[kAndMax];
    double alpha[kAndMax - 1];
};

__global__ void k_anderson_mix(int64_t cnt, int m, MixArgs a, double beta, double* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    double rm = a.rin[m][i], fm = a.F[m][i];
    double r = rm, f = fm;
    for (int j = 0; j < m; ++j) {
        r += a.alpha[j] * (a.rin[j][i] - rm);
        f += a.alpha[j] * (a.F[j][i] - fm);
    }
    out[i] = r + beta * f;
}

void launch_anderson_mix(int64_t cnt, int m, const double* const* rin, const double* const* F,
                         const double* alpha, double beta, double* rho_new, cudaStream_t s) {
    if (m < 0 || m > kAndMax - 1) fail(NAS_E_INVALID_ARG, "anderson depth");
    MixArgs a{};
    for (int j = 0; j <= m; ++j) {
        a.rin[j] = rin[j];
        a.F[j] = F[j];
    }
    for (int j = 0; j < m; ++j) a.alpha[j] = alpha[j];
    k_anderson_mix<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, m, a, beta, rho_new);
    NAS_CHECK_LAUNCH();
}

}  // namespace nas

namespace nas {

// ------------------------------------------------------------------ FP32 block PCG (mixed precision)
// The inner solve of the N shifted problems in FP32 storage and arithmetic;
// per-column scalars stay FP64 on the device (the same PcgCols logic), dot
// products accumulate in FP32 per thread and in FP64 across threads.

// out[k][c] = sum_i X_k[i][c] Y_k[i][c] (k < npairs <= 2), FP32 inputs
struct ColDotArgsF {
    const float* X[2];
    const float* Y[2];
};

__global__ void __launch_bounds__(256) k_coldots_f32(int64_t n, int N, int npairs, ColDotArgsF a, double* partial) {
    __shared__ double sh[2][256];
    const int R = 256 / N;
    const int t = threadIdx.x;
    const int c = t % N, r = t / N;
    float acc[2] = {0.f, 0.f};
    if (r < R) {
        for (int64_t row = (int64_t)blockIdx.x * R + r; row < n; row += (int64_t)gridDim.x * R) {
            const int64_t idx = row * N + c;
            for (int k = 0; k < npairs; ++k) acc[k] += a.X[k][idx] * a.Y[k][idx];
        }
    }
    for (int k = 0; k < npairs; ++k) sh[k][t] = (double)acc[k];
    __syncthreads();
    if (t < N) {
        for (int k = 0; k < npairs; ++k) {
            double s = 0.0;
            for (int rr = 0; rr < R; ++rr) s += sh[k][rr * N + t];
            partial[(int64_t)blockIdx.x * npairs * N + k * N + t] = s;
        }
    }
}

void launch_coldots_f32(int64_t n, int N, int npairs, const float* const* X, const float* const* Y,
                        double* partial, double* out, cudaStream_t s) {
    if (N < 1 || N > 256 || npairs < 1 || npairs > 2) fail(NAS_E_INVALID_ARG, "coldots width");
    ColDotArgsF a{};
    for (int k = 0; k < npairs; ++k) {
        a.X[k] = X[k];
        a.Y[k] = Y[k];
    }
    const int R = 256 / N;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (n + R - 1) / R));
    k_coldots_f32<<<nb, 256, 0, s>>>(n, N, npairs, a, partial);
    NAS_CHECK_LAUNCH();
    reduce_partials(nb, (int64_t)npairs * N, partial, out, s);
}

// X += alpha P, R -= alpha Q, Z = Dinv R (FP32 vectors, FP64 per-column alpha)
__global__ void k_pcg_update_f32(int64_t n, int N, const double* alpha, const int* active, const float* P,
                                 const float* Q, const float* Dinv, float* X, float* R, float* Z) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * N) return;
    const int64_t i = t / N;
    const int c = (int)(t - i * N);
    if (!active[c]) return;
    const float a = (float)alpha[c];
    X[t] += a * P[t];
    const float r = R[t] - a * Q[t];
    R[t] = r;
    Z[t] = Dinv[i] * r;
}

void launch_pcg_update_f32(int64_t n, int N, const double* alpha, const int* active, const float* P, const float* Q,
                           const float* Dinv, float* X, float* R, float* Z, cudaStream_t s) {
    if (n <= 0) return;
    k_pcg_update_f32<<<grid_for(n * N, 256), 256, 0, s>>>(n, N, alpha, active, P, Q, Dinv, X, R, Z);
    NAS_CHECK_LAUNCH();
}

__global__ void k_pcg_direction_f32(int64_t n, int N, const double* beta, const int* active, const float* Z,
                                    float* P) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * N) return;
    const int c = (int)(t % N);
    if (!active[c]) return;
    P[t] = Z[t] + (float)beta[c] * P[t];
}

void launch_pcg_direction_f32(int64_t n, int N, const double* beta, const int* active, const float* Z, float* P,
                              cudaStream_t s) {
    if (n <= 0) return;
    k_pcg_direction_f32<<<grid_for(n * N, 256), 256, 0, s>>>(n, N, beta, active, Z, P);
    NAS_CHECK_LAUNCH();
}

// Z = Dinv R (FP32)
__global__ void k_scale_rows_f32(int64_t n, int N, const float* Dinv, const float* R, float* Z) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * N) return;
    Z[t] = Dinv[t / N] * R[t];
}

void launch_scale_rows_f32(int64_t n, int N, const float* Dinv, const float* R, float* Z, cudaStream_t s) {
    if (n <= 0) return;
    k_scale_rows_f32<<<grid_for(n * N, 256), 256, 0, s>>>(n, N, Dinv, R, Z);
    NAS_CHECK_LAUNCH();
}

}  // namespace nas

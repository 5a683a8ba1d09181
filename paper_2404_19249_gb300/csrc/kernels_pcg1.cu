// Fused Jacobi-preconditioned CG for one right-hand side (the Hartree Poisson
// problem of Sec. 3.1), three kernels per iteration:
//   k_pcg1_spmv  : q = A p and per-block partial sums of p.q
//   k_pcg1_update: alpha = rz / (sum p.q); x += alpha p; r -= alpha q;
//                  z = D^-1 r; per-block partial sums of r.z and r.r
//   k_pcg1_dir   : beta = rz_new / rz; p = z + beta p; convergence test
// The scalars are not reduced by a separate launch: every block reduces the
// fixed-size partial array itself, in the same fixed order, so all blocks
// see bit-identical scalars and the result is deterministic.  The grid is a
// fixed number of blocks striding over the rows.  Kernels return at once
// when the solve is no longer active, so a captured graph of several
// iterations can run past convergence at negligible cost.
#include "kernels.h"

namespace nas {

static const int kPcgBlocks = 1216;  // 8 resident blocks x 152 SMs: one full wave (<= 32 registers)
static const int kPcgThreads = 256;

// Sum of part[0..G) in a fixed order, identical in every block.
__device__ __forceinline__ double block_sum_partials(const double* part, int G, double* sh) {
    double s = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) s += part[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void block_store_sum(double v, double* sh, double* out) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

template <int LPR>
__global__ void __launch_bounds__(kPcgThreads, 8) k_pcg1_spmv(Pcg1 s) {
    if (!*s.active) return;
    __shared__ double sh[kPcgThreads];
    const int lane = threadIdx.x % LPR;
    // warp-uniform loop: every lane of a warp runs the same trip count, so the
    // full-mask shuffles below are always executed by all 32 lanes
    const int64_t rows_per_warp = 32 / LPR;
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int64_t warp_stride = (int64_t)gridDim.x * (blockDim.x / 32) * rows_per_warp;
    double dot = 0.0;
    for (int64_t base = warp_id * rows_per_warp; base < s.n; base += warp_stride) {
        const int64_t row = base + (threadIdx.x % 32) / LPR;
        const bool valid = row < s.n;
        double acc = 0.0;
        if (valid) {
            const int p1 = s.rowptr[row + 1];
            for (int p = s.rowptr[row] + lane; p < p1; p += LPR) acc += s.val[p] * s.p[s.col[p]];
        }
#pragma unroll
        for (int off = LPR / 2; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, LPR > 1 ? LPR : 2);
        if (valid && lane == 0) {
            s.q[row] = acc;
            dot += s.p[row] * acc;
        }
    }
    block_store_sum(dot, sh, s.part_pq + blockIdx.x);
}

__global__ void __launch_bounds__(kPcgThreads, 8) k_pcg1_update(Pcg1 s, int par) {
    if (!*s.active) return;
    __shared__ double sh[kPcgThreads];
    const double pq = block_sum_partials(s.part_pq, gridDim.x, sh);
    const double rz = s.scal[par];
    if (!(pq > 0.0) || !isfinite(pq)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *s.breakdown = 1;
        return;
    }
    const double alpha = rz / pq;
    double srz = 0.0, srr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x) {
        s.x[i] += alpha * s.p[i];
        const double r = s.r[i] - alpha * s.q[i];
        s.r[i] = r;
        const double z = s.dinv[i] * r;
        s.z[i] = z;
        srz += r * z;
        srr += r * r;
    }
    block_store_sum(srz, sh, s.part_rz + blockIdx.x);
    __syncthreads();
    block_store_sum(srr, sh, s.part_rr + blockIdx.x);
}

__global__ void __launch_bounds__(kPcgThreads, 8) k_pcg1_dir(Pcg1 s, int par) {
    if (!*s.active || *s.breakdown) return;
    __shared__ double sh[kPcgThreads];
    const double rz_new = block_sum_partials(s.part_rz, gridDim.x, sh);
    const double rr = block_sum_partials(s.part_rr, gridDim.x, sh);
    const double rz = s.scal[par];
    const double beta = rz != 0.0 ? rz_new / rz : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x)
        s.p[i] = s.z[i] + beta * s.p[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.scal[par ^ 1] = rz_new;  // the next iteration reads the other slot
        s.scal[3] = rr;
        *s.iters += 1;
        if (!isfinite(rr)) *s.breakdown = 1;
        if (rr <= s.tol2 * s.scal[2] || !isfinite(rr)) *s.active = 0;
    }
}

int pcg1_blocks() { return kPcgBlocks; }

void launch_pcg1_iteration(const Pcg1& s, int par, int lpr, cudaStream_t st) {
    switch (lpr) {
        case 1: k_pcg1_spmv<1><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        case 2: k_pcg1_spmv<2><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        case 4: k_pcg1_spmv<4><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        case 8: k_pcg1_spmv<8><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        case 16: k_pcg1_spmv<16><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        default: k_pcg1_spmv<32><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
    }
    NAS_CHECK_LAUNCH();
    k_pcg1_update<<<kPcgBlocks, kPcgThreads, 0, st>>>(s, par);
    NAS_CHECK_LAUNCH();
    k_pcg1_dir<<<kPcgBlocks, kPcgThreads, 0, st>>>(s, par);
    NAS_CHECK_LAUNCH();
}

}  // namespace nas

// Fused Jacobi-preconditioned CG for one right-hand side (the Hartree Poisson
// problem of Sec. 3.1), three kernels per iteration:
//   k_pcg1_spmv  : q = A p and per-block partial sums of p.q
//   k_pcg1_update: alpha = rz / (sum p.q); x += alpha p; r -= alpha q;
//                  z = D^-1 r; per-block partial sums of r.z and r.r
//   k_pcg1_dir   : beta = rz_new / rz; p = z + beta p; convergence test
// With the two-level preconditioner z = D^-1 r + I K_H^-1 I^T r (I the
// nonnested transfer of the method, K_H = I^T K I), z and r.z are computed by
// four more kernels between update and dir: restriction I^T r (balanced piece
// sums, then per-row sums), the dense coarse solve with the precomputed
// K_H^-1, and prolongation.  k_pcg1_fused (below) runs the same seven phases
// inside one persistent cooperative launch.
// The scalars are not reduced by a separate launch: every block reduces the
// fixed-size partial array itself, in the same fixed order, so all blocks
// see bit-identical scalars and the result is deterministic.  The grid is a
// fixed number of blocks striding over the rows.  Kernels return at once
// when the solve is no longer active, so a captured graph of several
// iterations can run past convergence at negligible cost.
#include <algorithm>

#include "kernels.h"

namespace nas {

static const int kPcgBlocks = 1216;  // 8 resident blocks x 152 SMs: one full wave (<= 32 registers)
static const int kPcgThreads = 256;

// Sum of part[0..G) in a fixed order, identical in every block.
template <typename T>
__device__ __forceinline__ T block_sum_partials(const T* part, int G, T* sh) {
    T s = 0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) s += part[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    T r = sh[0];
    __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ void block_store_sum(T v, T* sh, T* out) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

template <typename T, int LPR>
__global__ void __launch_bounds__(kPcgThreads, 8) k_pcg1_spmv(Pcg1T<T> s) {
    if (!*s.active) return;
    __shared__ T sh[kPcgThreads];
    const int lane = threadIdx.x % LPR;
    // warp-uniform loop: every lane of a warp runs the same trip count, so the
    // full-mask shuffles below are always executed by all 32 lanes
    const int64_t rows_per_warp = 32 / LPR;
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int64_t warp_stride = (int64_t)gridDim.x * (blockDim.x / 32) * rows_per_warp;
    // read-only views (nothing this kernel writes aliases them), so the
    // loads may take the read-only path and be issued early
    const int32_t* __restrict__ rp = s.rowptr;
    const int32_t* __restrict__ cl = s.col;
    const T* __restrict__ va = s.val;
    const T* __restrict__ pv = s.p;
    T dot = 0;
    for (int64_t base = warp_id * rows_per_warp; base < s.n; base += warp_stride) {
        const int64_t row = base + (threadIdx.x % 32) / LPR;
        const bool valid = row < s.n;
        T acc = 0;
        if (valid) {
            // two independent accumulators: two gathers in flight per lane
            const int p1 = rp[row + 1];
            int p = rp[row] + lane;
            T a0 = 0, a1 = 0;
            for (; p + LPR < p1; p += 2 * LPR) {
                const int c0 = cl[p], c1 = cl[p + LPR];
                const T v0 = va[p], v1 = va[p + LPR];
                a0 += v0 * pv[c0];
                a1 += v1 * pv[c1];
            }
            if (p < p1) a0 += va[p] * pv[cl[p]];
            acc = a0 + a1;
        }
#pragma unroll
        for (int off = LPR / 2; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, LPR > 1 ? LPR : 2);
        if (valid && lane == 0) {
            s.q[row] = acc;
            dot += pv[row] * acc;
        }
    }
    block_store_sum(dot, sh, s.part_pq + blockIdx.x);
}

// q = A p from the sliced-ELL copy: one thread per row (slices of 32 rows, so
// a warp reads each of its rows' k-th entries as one coalesced segment), two
// accumulators; blocks stride over the rows; per-block partial sums of p.q
template <typename T>
__global__ void __launch_bounds__(kPcgThreads, 8) k_pcg1_spmv_sell(Pcg1T<T> s) {
    if (!*s.active) return;
    __shared__ T sh[kPcgThreads];
    const int64_t* __restrict__ sp = s.sell_ptr;
    const int32_t* __restrict__ cl = s.sell_col;
    const T* __restrict__ va = s.sell_val;
    const T* __restrict__ pv = s.p;
    T dot = 0;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < s.n;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slice = row >> 5;
        const int lane = (int)(row & 31);
        const int64_t b = sp[slice], e = sp[slice + 1];
        T a0 = 0, a1 = 0;
        int64_t idx = b + lane;
        for (; idx + 32 < e; idx += 64) {
            const int c0 = cl[idx], c1 = cl[idx + 32];
            const T v0 = va[idx], v1 = va[idx + 32];
            a0 += v0 * pv[c0];
            a1 += v1 * pv[c1];
        }
        if (idx < e) a0 += va[idx] * pv[cl[idx]];
        const T acc = a0 + a1;
        s.q[row] = acc;
        dot += pv[row] * acc;
    }
    block_store_sum(dot, sh, s.part_pq + blockIdx.x);
}

__global__ void k_sell_fill(int64_t n, int64_t nrows_pad, const int32_t* rowptr, const int32_t* col,
                            const double* val, const int64_t* sell_ptr, int32_t* sell_col, double* sell_val) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows_pad) return;
    const int64_t slice = r >> 5;
    const int lane = (int)(r & 31);
    const int64_t b = sell_ptr[slice];
    const int64_t w = (sell_ptr[slice + 1] - b) >> 5;
    const int64_t p0 = r < n ? rowptr[r] : 0;
    const int64_t len = r < n ? rowptr[r + 1] - p0 : 0;
    for (int64_t k = 0; k < w; ++k) {
        const int64_t idx = b + k * 32 + lane;
        if (k < len) {
            sell_col[idx] = col[p0 + k];
            sell_val[idx] = val[p0 + k];
        } else {
            sell_col[idx] = (int32_t)(r < n ? r : 0);
            sell_val[idx] = 0.0;
        }
    }
}

void launch_sell_fill(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                      const int64_t* sell_ptr, int64_t n_slices, int32_t* sell_col, double* sell_val, cudaStream_t st) {
    const int64_t rows = n_slices * 32;
    if (rows <= 0) return;
    k_sell_fill<<<(int)((rows + 255) / 256), 256, 0, st>>>(n, rows, rowptr, col, val, sell_ptr, sell_col, sell_val);
    NAS_CHECK_LAUNCH();
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads, 8) k_pcg1_update(Pcg1T<T> s, int par) {
    if (!*s.active) return;
    __shared__ T sh[kPcgThreads];
    const T pq = block_sum_partials(s.part_pq, gridDim.x, sh);
    const T rz = s.scal[par];
    if (!(pq > 0.0) || !isfinite(pq)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *s.breakdown = 1;
        return;
    }
    const T alpha = rz / pq;
    T srz = 0, srr = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x) {
        s.x[i] += alpha * s.p[i];
        const T r = s.r[i] - alpha * s.q[i];
        s.r[i] = r;
        srr += r * r;
        if (!s.two_level) {  // with the coarse correction, z and r.z come from k_pcg1_prolong
            const T z = s.dinv[i] * r;
            s.z[i] = z;
            srz += r * z;
        }
    }
    if (!s.two_level) block_store_sum(srz, sh, s.part_rz + blockIdx.x);
    __syncthreads();
    block_store_sum(srr, sh, s.part_rr + blockIdx.x);
}

// ---- two-level preconditioner z = D^-1 r + I K_H^-1 I^T r (coarse space of the method)
// Warp-level pieces shared by the per-phase kernels and the persistent form
// (same arithmetic in both): the sum of one balanced piece of an I^T row, and
// one row of the dense K_H^-1 times c (in T: FP64 storage for the FP64 solve,
// since a FP32 -> FP64 conversion costs a slot of the FP64 pipe like an FMA).
// Lanes stride by 32 with two independent accumulators (two gathers or loads
// in flight per lane), then a fixed-order shuffle sum; lane 0 holds the result.
template <typename T>
__device__ __forceinline__ T piece_sum(const int32_t* trow, const T* tval, const T* r, int64_t beg, int64_t end,
                                       int lane) {
    T a0 = 0, a1 = 0;
    int64_t p = beg + lane;
    for (; p + 32 < end; p += 64) {
        a0 += tval[p] * r[trow[p]];
        a1 += tval[p + 32] * r[trow[p + 32]];
    }
    if (p < end) a0 += tval[p] * r[trow[p]];
    T acc = a0 + a1;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    return acc;
}

template <typename T>
__device__ __forceinline__ T coarse_row_dot(const T* row, const T* c, int64_t nH, int lane) {
    T a0 = 0, a1 = 0;
    int64_t b = lane;
    for (; b + 32 < nH; b += 64) {
        a0 += row[b] * c[b];
        a1 += row[b + 32] * c[b + 32];
    }
    if (b < nH) a0 += row[b] * c[b];
    T acc = a0 + a1;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    return acc;
}

// c = I^T r in two stages: one warp per balanced piece of an I^T row, then
// each coarse row adds its pieces in order
template <typename T>
__global__ void __launch_bounds__(kPcgThreads) k_pcg1_restrict(Pcg1T<T> s) {
    if (!*s.active || *s.breakdown) return;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (q >= s.tpc.npieces) return;  // warp-uniform
    const T acc = piece_sum(s.trow, s.tval, s.r, s.tpc.piece_start[q], s.tpc.piece_start[q + 1], lane);
    if (lane == 0) s.cpart[q] = acc;
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads) k_pcg1_restrict_sum(Pcg1T<T> s) {
    if (!*s.active || *s.breakdown) return;
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.nH) return;
    T acc = 0;
    for (int q = s.tpc.seg_piece[a]; q < s.tpc.seg_piece[a + 1]; ++q) acc += s.cpart[q];
    s.cvec[a] = acc;
}

// y = K_H^-1 c (dense row-major inverse): one warp per row
template <typename T>
__global__ void __launch_bounds__(kPcgThreads) k_pcg1_coarse(Pcg1T<T> s) {
    if (!*s.active || *s.breakdown) return;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t a = warp; a < s.nH; a += nwarps) {
        const T acc = coarse_row_dot(s.khinv + a * s.nH, s.cvec, s.nH, lane);
        if (lane == 0) s.yvec[a] = acc;
    }
}

// z = D^-1 r + I y, with per-block partial sums of r.z
template <typename T>
__global__ void __launch_bounds__(kPcgThreads, 8) k_pcg1_prolong(Pcg1T<T> s) {
    if (!*s.active || *s.breakdown) return;
    __shared__ T sh[kPcgThreads];
    T srz = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x) {
        const T r = s.r[i];
        T z = s.dinv[i] * r;
        for (int k = 0; k < 4; ++k) {
            const int a = s.icol[4 * i + k];
            if (a >= 0) z += s.ival[4 * i + k] * s.yvec[a];
        }
        s.z[i] = z;
        srz += r * z;
    }
    block_store_sum(srz, sh, s.part_rz + blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads, 8) k_pcg1_dir(Pcg1T<T> s, int par) {
    if (!*s.active || *s.breakdown) return;
    __shared__ T sh[kPcgThreads];
    const T rz_new = block_sum_partials(s.part_rz, gridDim.x, sh);
    const T rr = block_sum_partials(s.part_rr, gridDim.x, sh);
    const T rz = s.scal[par];
    const T beta = rz != T(0) ? rz_new / rz : T(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x)
        s.p[i] = s.z[i] + beta * s.p[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.scal[par ^ 1] = rz_new;  // the next iteration reads the other slot
        s.scal[3] = rr;
        *s.iters += 1;
        if (!isfinite(rr)) *s.breakdown = 1;
        if (rr <= s.tol2 * s.scal[2] || !isfinite(rr)) *s.active = 0;  // scal[2] = tol^2 ||b||^2 (tol2 = 1)
    }
}

int pcg1_blocks() { return kPcgBlocks; }

// ---- persistent form of the two-level FP64 iteration (sliced-ELL matrix)
// One cooperative launch runs up to `chunk` whole iterations; the phases of an
// iteration (SpMV, update, restriction pieces, restriction sums, coarse solve,
// prolongation, new direction) are separated by grid-wide barriers instead of
// kernel boundaries, so the blocks stay resident and keep their caches warm.
// The grid is the per-phase kernels' grid (kPcgBlocks, one full wave) and
// every phase does the arithmetic of the kernel it replaces in the same order,
// with the same rows per thread and the same per-block partial sums, so both
// forms give bit-identical iterates.  Arrays written during the
// launch (p, q, r, z, x, the partial sums, cpart, cvec, yvec) are read with
// ordinary coherent loads; only the matrix, the transfer and the diagonal go
// through the read-only path.
static const int kFusedMinBlocks = 8;                       // per SM, <= 32 registers
static const unsigned long long kBarrierNs = 1000000000ull;  // 1 s wait limit

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch (every block resident).  bar[0]
// counts arrivals, bar[1] is the generation.  A wait longer than kBarrierNs
// sets *err and returns; once *err is set no barrier waits.  Returns the same
// value in every thread of the block: true while no error was flagged.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned nblocks, int* sh_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = *(volatile int*)err == 0;
        if (ok) {
            const unsigned g = ld_acquire_gpu(bar + 1);
            __threadfence();
            if (atomicAdd(bar, 1u) == nblocks - 1) {
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                const unsigned long long t0 = globaltimer_ns();
                while (ld_acquire_gpu(bar + 1) == g) {
                    if (globaltimer_ns() - t0 > kBarrierNs) {
                        atomicExch(err, 1);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        *sh_ok = ok;
    }
    __syncthreads();
    return *sh_ok != 0;
}

__global__ void __launch_bounds__(kPcgThreads, kFusedMinBlocks)
    k_pcg1_fused(Pcg1 s, unsigned* bar, int* err, int chunk) {
    __shared__ double sh[kPcgThreads];
    __shared__ int sh_ok;
    const unsigned G = gridDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)G * blockDim.x;
    const int lane = threadIdx.x % 32;
    const int64_t warp = tid / 32, nwarps = nth / 32;
    const int64_t* __restrict__ sp = s.sell_ptr;
    const int32_t* __restrict__ cl = s.sell_col;
    const double* __restrict__ va = s.sell_val;
    const double* __restrict__ dinv = s.dinv;
    const int32_t* __restrict__ trow = s.trow;
    const double* __restrict__ tval = s.tval;
    const int32_t* __restrict__ icol = s.icol;
    const double* __restrict__ ival = s.ival;
    const double* __restrict__ khinv = s.khinv;
    int par = 0;
    for (int it = 0; it < chunk; ++it) {
        // the flags change only before a barrier, so every block sees the same values
        if (!*(volatile int*)s.active || *(volatile int*)s.breakdown) break;
        // q = A p, partial sums of p.q
        {
            double dot = 0;
            for (int64_t row = tid; row < s.n; row += nth) {
                const int64_t slice = row >> 5;
                const int rl = (int)(row & 31);
                const int64_t b = sp[slice], e = sp[slice + 1];
                double a0 = 0, a1 = 0;
                int64_t idx = b + rl;
                for (; idx + 32 < e; idx += 64) {
                    const int c0 = cl[idx], c1 = cl[idx + 32];
                    const double v0 = va[idx], v1 = va[idx + 32];
                    a0 += v0 * s.p[c0];
                    a1 += v1 * s.p[c1];
                }
                if (idx < e) a0 += va[idx] * s.p[cl[idx]];
                const double acc = a0 + a1;
                s.q[row] = acc;
                dot += s.p[row] * acc;
            }
            block_store_sum(dot, sh, s.part_pq + blockIdx.x);
        }
        if (!grid_barrier(bar, err, G, &sh_ok)) return;
        // alpha = rz / p.q; x += alpha p; r -= alpha q; partial sums of r.r
        {
            const double pq = block_sum_partials(s.part_pq, (int)G, sh);
            const double rz = s.scal[par];
            if (!(pq > 0.0) || !isfinite(pq)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) *s.breakdown = 1;
                break;  // every block computed the same pq
            }
            const double alpha = rz / pq;
            double srr = 0;
            for (int64_t i = tid; i < s.n; i += nth) {
                s.x[i] += alpha * s.p[i];
                const double r = s.r[i] - alpha * s.q[i];
                s.r[i] = r;
                srr += r * r;
            }
            block_store_sum(srr, sh, s.part_rr + blockIdx.x);
        }
        if (!grid_barrier(bar, err, G, &sh_ok)) return;
        // I^T r: one warp per balanced piece
        for (int64_t q = warp; q < s.tpc.npieces; q += nwarps) {
            const double acc = piece_sum(trow, tval, s.r, s.tpc.piece_start[q], s.tpc.piece_start[q + 1], lane);
            if (lane == 0) s.cpart[q] = acc;
        }
        if (!grid_barrier(bar, err, G, &sh_ok)) return;
        for (int64_t a = tid; a < s.nH; a += nth) {
            double acc = 0;
            for (int q = s.tpc.seg_piece[a]; q < s.tpc.seg_piece[a + 1]; ++q) acc += s.cpart[q];
            s.cvec[a] = acc;
        }
        if (!grid_barrier(bar, err, G, &sh_ok)) return;
        // y = K_H^-1 c: one warp per row
        for (int64_t a = warp; a < s.nH; a += nwarps) {
            const double acc = coarse_row_dot(khinv + a * s.nH, s.cvec, s.nH, lane);
            if (lane == 0) s.yvec[a] = acc;
        }
        if (!grid_barrier(bar, err, G, &sh_ok)) return;
        // z = D^-1 r + I y, partial sums of r.z
        {
            double srz = 0;
            for (int64_t i = tid; i < s.n; i += nth) {
                const double r = s.r[i];
                double z = dinv[i] * r;
                for (int k = 0; k < 4; ++k) {
                    const int a = icol[4 * i + k];
                    if (a >= 0) z += ival[4 * i + k] * s.yvec[a];
                }
                s.z[i] = z;
                srz += r * z;
            }
            block_store_sum(srz, sh, s.part_rz + blockIdx.x);
        }
        if (!grid_barrier(bar, err, G, &sh_ok)) return;
        // beta = rz_new / rz; p = z + beta p; stop test
        {
            const double rz_new = block_sum_partials(s.part_rz, (int)G, sh);
            const double rr = block_sum_partials(s.part_rr, (int)G, sh);
            const double rz = s.scal[par];
            const double beta = rz != 0.0 ? rz_new / rz : 0.0;
            for (int64_t i = tid; i < s.n; i += nth) s.p[i] = s.z[i] + beta * s.p[i];
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                s.scal[par ^ 1] = rz_new;
                s.scal[3] = rr;
                *s.iters += 1;
                if (!isfinite(rr)) *s.breakdown = 1;
                if (rr <= s.tol2 * s.scal[2] || !isfinite(rr)) *s.active = 0;
            }
        }
        if (!grid_barrier(bar, err, G, &sh_ok)) return;
        par ^= 1;
    }
}

int pcg1_fused_blocks() {
    // computed once (a function-local static is initialised once even when
    // nas_batch_run's worker threads arrive here together)
    static const int blocks = [] {
        int dev = 0, sms = 0, coop = 0, per_sm = 0, b = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg1_fused, kPcgThreads, 0) == cudaSuccess &&
            (int64_t)per_sm * sms >= kPcgBlocks)
            b = kPcgBlocks;  // the per-phase kernels' grid: same partial sums, same iterates
        cudaGetLastError();
        return b;
    }();
    return blocks;
}

void launch_pcg1_fused(const Pcg1& s, unsigned* bar, int* err, int chunk, int blocks, cudaStream_t st) {
    if (blocks <= 0 || !s.two_level || !s.sell_ptr) fail(NAS_E_INVALID_ARG, "fused PCG: unsupported configuration");
    Pcg1 sv = s;
    void* args[4] = {(void*)&sv, (void*)&bar, (void*)&err, (void*)&chunk};
    NAS_CUDA(cudaLaunchCooperativeKernel((const void*)k_pcg1_fused, dim3((unsigned)blocks), dim3(kPcgThreads), args,
                                         0, st));
    ++g_launch_count;
}

template <typename T>
static void pcg1_coarse_correction(const Pcg1T<T>& s, cudaStream_t st) {
    const int warps_per_block = kPcgThreads / 32;
    const int gb = (int)std::min<int64_t>(4 * kPcgBlocks, (s.nH + warps_per_block - 1) / warps_per_block);
    if (s.tpc.npieces > 0) {
        k_pcg1_restrict<T><<<(int)((s.tpc.npieces + warps_per_block - 1) / warps_per_block), kPcgThreads, 0, st>>>(s);
        NAS_CHECK_LAUNCH();
    }
    k_pcg1_restrict_sum<T><<<(int)((s.nH + kPcgThreads - 1) / kPcgThreads), kPcgThreads, 0, st>>>(s);
    NAS_CHECK_LAUNCH();
    k_pcg1_coarse<T><<<gb, kPcgThreads, 0, st>>>(s);
    NAS_CHECK_LAUNCH();
    k_pcg1_prolong<T><<<kPcgBlocks, kPcgThreads, 0, st>>>(s);
    NAS_CHECK_LAUNCH();
}

template <typename T>
static void pcg1_iteration(const Pcg1T<T>& s, int par, int lpr, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                           cudaEvent_t ev1 = nullptr) {
    if (ev0) NAS_CUDA(cudaEventRecord(ev0, st));
    if (s.sell_ptr) lpr = 0;
    switch (lpr) {
        case 0: k_pcg1_spmv_sell<T><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        case 1: k_pcg1_spmv<T, 1><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        case 2: k_pcg1_spmv<T, 2><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        case 4: k_pcg1_spmv<T, 4><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        case 8: k_pcg1_spmv<T, 8><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        case 16: k_pcg1_spmv<T, 16><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
        default: k_pcg1_spmv<T, 32><<<kPcgBlocks, kPcgThreads, 0, st>>>(s); break;
    }
    NAS_CHECK_LAUNCH();
    if (ev1) NAS_CUDA(cudaEventRecord(ev1, st));
    k_pcg1_update<T><<<kPcgBlocks, kPcgThreads, 0, st>>>(s, par);
    NAS_CHECK_LAUNCH();
    if (s.two_level) pcg1_coarse_correction(s, st);
    k_pcg1_dir<T><<<kPcgBlocks, kPcgThreads, 0, st>>>(s, par);
    NAS_CHECK_LAUNCH();
}

void launch_pcg1_iteration(const Pcg1& s, int par, int lpr, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
    pcg1_iteration(s, par, lpr, st, ev0, ev1);
}
void launch_pcg1_iteration(const Pcg1f& s, int par, int lpr, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
    pcg1_iteration(s, par, lpr, st, ev0, ev1);
}
int pcg1_kernels_per_iteration(int two_level, int64_t npieces) {
    return two_level ? (npieces > 0 ? 7 : 6) : 3;
}
void launch_pcg1_coarse_correction(const Pcg1& s, cudaStream_t st) { pcg1_coarse_correction(s, st); }
void launch_pcg1_coarse_correction(const Pcg1f& s, cudaStream_t st) { pcg1_coarse_correction(s, st); }

// ---- mixed precision helpers
// start of an inner solve from e = 0: r given, z = M^-1 r (Jacobi part; the
// coarse part, if any, was added by the coarse-correction kernels), p = z,
// x = 0, partial sums of r.z (Jacobi only) and r.r
template <typename T>
__global__ void __launch_bounds__(kPcgThreads, 8) k_pcg1_start(Pcg1T<T> s) {
    __shared__ T sh[kPcgThreads];
    T srz = 0, srr = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x) {
        const T r = s.r[i];
        T z;
        if (s.two_level) {
            z = s.z[i];
        } else {
            z = s.dinv[i] * r;
            s.z[i] = z;
            srz += r * z;
        }
        s.p[i] = z;
        s.x[i] = 0;
        srr += r * r;
    }
    if (!s.two_level) block_store_sum(srz, sh, s.part_rz + blockIdx.x);
    __syncthreads();
    block_store_sum(srr, sh, s.part_rr + blockIdx.x);
}

void launch_pcg1_start(const Pcg1f& s, cudaStream_t st) {
    k_pcg1_start<float><<<kPcgBlocks, kPcgThreads, 0, st>>>(s);
    NAS_CHECK_LAUNCH();
}

__global__ void k_cast_to_f32(int64_t n, const double* a, float* b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_add_f32(int64_t n, const float* e, double* x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += (double)e[i];
}

void launch_cast_to_f32(int64_t n, const double* a, float* b, cudaStream_t st) {
    if (n <= 0) return;
    k_cast_to_f32<<<grid_for(n, 256), 256, 0, st>>>(n, a, b);
    NAS_CHECK_LAUNCH();
}

void launch_add_f32(int64_t n, const float* e, double* x, cudaStream_t st) {
    if (n <= 0) return;
    k_add_f32<<<grid_for(n, 256), 256, 0, st>>>(n, e, x);
    NAS_CHECK_LAUNCH();
}

}  // namespace nas

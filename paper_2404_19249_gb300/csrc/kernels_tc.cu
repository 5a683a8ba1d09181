// Tensor-core product W = T R for the LOBPCG preconditioner of the small
// problem (T = (I^T K I)^-1, the dense inverse coarse stiffness, FP32,
// nH x nH; R the block of residual rows, nH x k), on the 5th-generation
// tensor cores of sm_103a: tcgen05.mma with its accumulator in tensor memory.
//
// Precision: split TF32.  Each FP32 operand x is held as x_hi = tf32(x) and
// x_lo = tf32(x - x_hi); the product is accumulated as hi*hi + hi*lo + lo*hi
// (the lo*lo term is below FP32 rounding), in FP32 in tensor memory, which
// keeps FP32-level accuracy (Markidis et al. 2018; Ootomo and Yokota 2022).
// The preconditioner needs no more: it is a fixed SPD approximation of an
// inverse inside LOBPCG.
//
// Layout: the operands are staged by the CTA's threads in shared memory in
// the canonical K-major layout without swizzling: 8-row x 16-byte core
// matrices, the 8 core matrices of one 8-row group and one 32-element K tile
// contiguous (leading byte offset 128 between K-adjacent core matrices,
// stride byte offset 1024 between 8-row groups).  One tcgen05.mma of kind
// tf32 consumes K = 8 (two core matrices); a K tile of 32 takes four of them
// per split term.  A = T rows (K-major as T is stored), B = R^T: the
// staging loop reads R's rows (FP64), converts, splits and writes them
// transposed into the K-major layout; N is padded to a multiple of 16 (the
// MMA's N for M = 128) with zero columns.
//
// Work split: one CTA per 128-row tile of T and K range (split K, kTcSplit
// ranges), 128 threads; thread 0 issues the MMAs and commits them to an
// mbarrier; every wait on it is bounded (kTcSpin polls): on timeout the CTA
// records the error, frees its tensor memory and returns.  The CTA's FP32
// partial product goes to part[split][row][col], the layout of the FP32 SIMT
// kernel's stage 1, and the same stage 2 adds the splits in order.
#include <cuda_fp16.h>

#include <cstdint>

#include "kernels.h"

namespace nas {

namespace {

const int kTcM = 128;        // rows per CTA (MMA M)
const int kTcK = 32;         // K tile (floats)
const int kTcSplit = 12;     // K ranges
const int kTcThreads = 128;
const long long kTcSpin = 20000000;   // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// shared memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units), descriptor version 1 (bits 46-48), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// bounded wait for the phase with parity `par` to complete; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t par) {
    for (long long it = 0; it < kTcSpin; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, q;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(par)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace

__device__ int g_tc_error = 0;   // set when a CTA's mbarrier wait ran out (never expected)

__device__ __forceinline__ uint32_t canon_off(int r, int kk) {
    return (uint32_t)((r >> 3) * 1024 + (kk >> 2) * 128 + (r & 7) * 16 + (kk & 3) * 4);
}

// part[sp][i][j] = sum over b in K range sp of T[i][b] R[b][j], i in the CTA's
// 128 rows, j < k.  Dynamic shared memory: A_hi, A_lo (128 x 32 floats each),
// B_hi, B_lo (Npad x 32 floats each), 1024-byte aligned.
__global__ void __launch_bounds__(kTcThreads) k_tc_precond_part(int64_t nH, int k, int Npad, const float* T,
                                                               const double* R, float* part) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    unsigned char* base = tc_smem;
    // the dynamic area starts 1024-aligned (launch adds 1024 bytes of slack)
    base += (1024 - (smem_u32(base) & 1023)) & 1023;
    float* Ahi = reinterpret_cast<float*>(base);
    float* Alo = Ahi + kTcM * kTcK;
    float* Bhi = Alo + kTcM * kTcK;
    float* Blo = Bhi + Npad * kTcK;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int64_t row0 = (int64_t)blockIdx.x * kTcM;
    const int64_t span = (nH + kTcSplit - 1) / kTcSplit;
    const int64_t kb = (int64_t)blockIdx.y * span;
    const int64_t ke = kb + span < nH ? kb + span : nH;
    const uint32_t ncols = Npad <= 32 ? 32u : Npad <= 64 ? 64u : Npad <= 128 ? 128u : 256u;
    const uint32_t mb = smem_u32(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_tf32(kTcM, Npad);
    bool ok = true;
    uint32_t phase = 0;
    bool first = true;
    for (int64_t k0 = kb; k0 < ke && ok; k0 += kTcK) {
        // stage the A tile (rows of T) and the B tile (columns of R), split into
        // TF32 hi and lo parts, zero outside the matrix and the K range
        for (int idx = tid; idx < kTcM * kTcK; idx += kTcThreads) {
            const int r = idx / kTcK, kk = idx % kTcK;
            const int64_t i = row0 + r, b = k0 + kk;
            const float x = (i < nH && b < ke) ? T[i * nH + b] : 0.f;
            const float hi = __uint_as_float(tf32_bits(x));
            const float lo = __uint_as_float(tf32_bits(x - hi));
            const uint32_t o = canon_off(r, kk) / 4;
            Ahi[o] = hi;
            Alo[o] = lo;
        }
        for (int idx = tid; idx < Npad * kTcK; idx += kTcThreads) {
            const int kk = idx / Npad, j = idx % Npad;
            const int64_t b = k0 + kk;
            const float x = (j < k && b < ke) ? (float)R[b * k + j] : 0.f;
            const float hi = __uint_as_float(tf32_bits(x));
            const float lo = __uint_as_float(tf32_bits(x - hi));
            const uint32_t o = canon_off(j, kk) / 4;
            Bhi[o] = hi;
            Blo[o] = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
            for (int ks = 0; ks < kTcK / 8; ++ks) {
                const uint32_t off = (uint32_t)ks * 256;   // K = 8 tf32 = two 16-byte core matrices
                mma_tf32(tmem, smem_desc(ah + off, 128, 1024), smem_desc(bh + off, 128, 1024), idesc, first ? 0u : 1u);
                first = false;
                mma_tf32(tmem, smem_desc(ah + off, 128, 1024), smem_desc(bl + off, 128, 1024), idesc, 1u);
                mma_tf32(tmem, smem_desc(al + off, 128, 1024), smem_desc(bh + off, 128, 1024), idesc, 1u);
            }
            mma_commit(mb);
        }
        first = false;
        // the tile buffers are reused: wait until the MMAs that read them are done
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        ok = __syncthreads_and(ok) != 0;
    }
    if (!ok) {
        atomicExch(&g_tc_error, 1);
        mbar_wait(mb, phase ^ 1u);   // bounded second wait for the MMAs in flight
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && kb < ke) {
        // accumulator rows 32 w .. 32 w + 31 live in tensor memory lanes of warp w
        const int64_t i = row0 + 32 * warp + lane;
        for (int c0 = 0; c0 < Npad; c0 += 16) {
            uint32_t v[16];
            const uint32_t addr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (i < nH)
                for (int q = 0; q < 16; ++q) {
                    const int j = c0 + q;
                    if (j < k) part[((int64_t)blockIdx.y * nH + i) * k + j] = __uint_as_float(v[q]);
                }
        }
    } else if (ok) {
        // empty K range: this split contributes zeros
        const int64_t i = row0 + 32 * warp + lane;
        if (i < nH)
            for (int j = 0; j < k; ++j) part[((int64_t)blockIdx.y * nH + i) * k + j] = 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// W[i][j] = sum_sp part[sp][i][j] (i < nH, splits in order); W[i][j] = Dinv[i] R[i][j] (nH <= i < m)
__global__ void k_tc_precond_sum(int64_t nH, int64_t m, int k, const float* part, const double* R,
                                 const double* Dinv, double* W) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * k) return;
    const int64_t i = t / k;
    if (i < nH) {
        float acc = 0.f;
        for (int sp = 0; sp < kTcSplit; ++sp) acc += part[(int64_t)sp * nH * k + t];
        W[t] = (double)acc;
    } else {
        W[t] = Dinv[i] * R[t];
    }
}

void launch_dense_precond_tc(int64_t nH, int64_t m, int k, const float* T, const double* R, const double* Dinv,
                             float* part, double* W, cudaStream_t s) {
    if (k < 1 || k > 256) fail(NAS_E_INVALID_ARG, "tensor-core preconditioner: block width out of range");
    if (m <= 0) return;
    if (nH > 0) {
        const int Npad = (k + 15) / 16 * 16;
        const size_t smem = 1024 + sizeof(float) * (size_t)kTcK * (2 * kTcM + 2 * Npad);
        NAS_CUDA(cudaFuncSetAttribute(k_tc_precond_part, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        dim3 grid((unsigned)((nH + kTcM - 1) / kTcM), kTcSplit);
        k_tc_precond_part<<<grid, kTcThreads, smem, s>>>(nH, k, Npad, T, R, part);
        NAS_CHECK_LAUNCH();
    }
    k_tc_precond_sum<<<grid_for(m * k, 256), 256, 0, s>>>(nH, m, k, part, R, Dinv, W);
    NAS_CHECK_LAUNCH();
}

int64_t dense_precond_tc_part_size(int64_t nH, int k) { return (int64_t)kTcSplit * nH * k; }

// ---------------------------------------------------------------------------
// Reconstruction Psi = I u_H + U^ alpha (the density update of Algorithm 3)
// with the dense part U^ alpha (n x Na times Na x N; Na, N <= 64) on the
// tensor cores at FP64 accuracy, by an error-free split into small integers
// (the scheme of Ozaki, Ogita, Oishi and Rump, 2012, in its integer-slice
// form):
//  * row i of U^ is written in fixed point against the largest binary
//    exponent of the row, x = sign M 2^(E_i - 1075) with M the 53-bit
//    significand shifted right by E_i - e(x) (truncated), and the top 49 bits
//    of M are cut into seven 7-bit slices, M ~ sum_s a_s 2^(46 - 7 s); column j
//    of alpha likewise against its own exponent F_j (slices b_t);
//  * slices are integers below 128 in magnitude, exact in FP16; a product of
//    two is below 2^14, a sum over K <= 64 below 2^20, and
//    D_d = sum_{s+t=d} A_s B_t (d = 0..6, at most 7 terms) below 2^23, so an
//    FP32 accumulator in tensor memory holds it exactly;
//  * the epilogue adds acc = sum_d D_d 2^(7 (6 - d)) in int64 (|acc| < 2^63,
//    exact) and rounds once: (double) acc 2^(E_i - 1050) 2^(F_j - 1050).
// The slices s + t > 6 and the truncated bits are dropped: per product the
// error is below 2^-45.8 max_k |U^_ik| max_k |alpha_kj|, per entry below
// 2^-39.8 of it for K = 64, within a factor 4 of FP64's own worst-case
// dot-product bound (K^2 2^-53 = 2^-41).  The FP64 pipe keeps only the conversion, the
// scaling and the four terms of I u_H, about 7 of the 68 FP64 operations per
// entry of the SIMT kernel.
//
// One persistent CTA per SM (256 threads; 168 KB of slices in shared memory,
// the same canonical no-swizzle K-major layout as above with 64-element rows);
// alpha's slices are staged once per CTA.  Per 128-row tile: two threads slice
// each row (one K half each) into the seven A slices, thread 0 issues the
// 28 x (Na/16) MMAs (kind::f16, M = 128, N = Npad) into seven accumulators and
// commits them to an mbarrier (bounded wait), and the same two threads read
// the row's accumulators (tensor-memory lane = row), alternate 16-column
// chunks each.  With four warps per SM the kernel was latency-bound (6 % of
// the warp slots, 8 % issue-active, FP64 pipe 28 % busy under ncu).
namespace {

const int kOzM = 128;                           // rows per tile (MMA M)
const int kOzK = 64;                            // K capacity: rows of 8 core matrices of 8 FP16
const int kOzS = 7;                             // slices per operand
const int kOzThreads = 256;                     // two threads per tile row
const uint32_t kOzSliceA = kOzM * kOzK * 2;     // bytes per A slice
const uint32_t kOzSliceB = 64 * kOzK * 2;       // bytes per B slice (N <= 64)

// kind::f16: D FP32 (bits 4-5 = 1), A and B FP16 (bits 7-9, 10-12 = 0), K-major
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// byte offset of FP16 element (r, k) of a K-major tile with 64-element rows
__device__ __forceinline__ uint32_t canon16(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ int biased_exp(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// 2^e as a double for -1074 <= e <= 1023 (0 below)
__device__ __forceinline__ double pow2(int e) {
    if (e >= -1022) return __longlong_as_double((long long)(e + 1023) << 52);
    if (e >= -1074) return __longlong_as_double(1LL << (e + 1074));
    return 0.0;
}

// significand of x aligned to the biased exponent E >= e(x) (zero and
// subnormal x give 0), and its sign
__device__ __forceinline__ unsigned long long fixed53(double x, int E, bool* neg) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    *neg = bits < 0;
    if (ex == 0 || E - ex >= 53) return 0ULL;
    return ((unsigned long long)(bits & 0xFFFFFFFFFFFFFLL) | (1ULL << 52)) >> (E - ex);
}

// FP16 bit pattern of slice s (bits 46 - 7 s .. 52 - 7 s of M) with its sign
__device__ __forceinline__ uint32_t slice_h(unsigned long long M, bool neg, int s) {
    const int a = (int)((M >> (46 - 7 * s)) & 127ULL);
    return (uint32_t)__half_as_ushort(__int2half_rn(neg ? -a : a));
}

// the 8 values x[0..7] (K positions k0..k0+7 of tile row r) as 7 slices
__device__ __forceinline__ void stage8(const double* x, int E, unsigned char* slab, uint32_t slice_bytes, int r,
                                       int k0) {
    unsigned long long M[8];
    bool neg[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) M[q] = fixed53(x[q], E, &neg[q]);
#pragma unroll
    for (int s = 0; s < kOzS; ++s) {
        uint4 v;
        v.x = slice_h(M[0], neg[0], s) | (slice_h(M[1], neg[1], s) << 16);
        v.y = slice_h(M[2], neg[2], s) | (slice_h(M[3], neg[3], s) << 16);
        v.z = slice_h(M[4], neg[4], s) | (slice_h(M[5], neg[5], s) << 16);
        v.w = slice_h(M[6], neg[6], s) | (slice_h(M[7], neg[7], s) << 16);
        *reinterpret_cast<uint4*>(slab + (size_t)s * slice_bytes + canon16(r, k0)) = v;
    }
}

}  // namespace

// Psi[i][j] = sum_k ival[i][k] U[icol[i][k]][j] + sum_c Uhat[i][c] U[nH + c][j]
// (alpha = U[nH..nH+Na)) with the second sum on the tensor cores as above.
// Dynamic shared memory: 7 A slices (128 x 64 FP16) and 7 B slices (64 x 64
// FP16), 1024-byte aligned.
__global__ void __launch_bounds__(kOzThreads) k_tc_reconstruct(int64_t n, const int32_t* icol, const double* ival,
                                                              int N, int Npad, uint32_t ncols, const double* U,
                                                              int64_t nH, int Na, const double* Uhat,
                                                              double* Psi) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ double colscale[64];   // 2^(F_j - 1050), 0 for an all-zero column
    __shared__ int epart[2][kOzM];     // the two half-row maxima of the row exponent
    unsigned char* base = oz_smem;
    base += (1024 - (smem_u32(base) & 1023)) & 1023;
    unsigned char* As = base;
    unsigned char* Bs = base + (size_t)kOzS * kOzSliceA;
    // thread tid works on tile row r = tid % 128: K half h = tid / 128 when
    // staging, and in the epilogue (warps w and w + 4 share tensor-memory lanes
    // 32 (w % 4) ..) the 16-column chunks c with c % 2 == h
    const int tid = threadIdx.x, warp = tid >> 5, r = tid & (kOzM - 1), h = tid >> 7;
    const uint32_t mb = smem_u32(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // alpha's slices: thread j < Npad stages column j (row j of the K-major B tile)
    const double* alpha = U + nH * (int64_t)N;
    if (tid < Npad) {
        const int j = tid;
        int F = 0;
        if (j < N)
            for (int c = 0; c < Na; ++c) F = max(F, biased_exp(alpha[(int64_t)c * N + j]));
        colscale[j] = F ? pow2(F - 1050) : 0.0;
        for (int k0 = 0; k0 < kOzK; k0 += 8) {
            double x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = k0 + q;
                x[q] = (j < N && c < Na) ? alpha[(int64_t)c * N + j] : 0.0;
            }
            stage8(x, F, Bs, kOzSliceB, j, k0);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_f16(kOzM, Npad);
    const int nks = (Na + 15) / 16;
    const int64_t ntiles = (n + kOzM - 1) / kOzM;
    bool ok = true;
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * kOzM + r;
        // row i of U^ in seven slices (zeros past the last row): this thread
        // takes K positions [32 h, 32 h + 32); the row exponent is the max of
        // the two halves' maxima
        const int kb = (kOzK / 2) * h;
        int E = 0;
        if (i < n)
            for (int c = kb; c < kb + kOzK / 2 && c < Na; ++c) E = max(E, biased_exp(Uhat[i * Na + c]));
        epart[h][r] = E;
        __syncthreads();
        E = max(epart[0][r], epart[1][r]);
        for (int k0 = kb; k0 < kb + kOzK / 2; k0 += 8) {
            double x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = k0 + q;
                x[q] = (i < n && c < Na) ? Uhat[i * Na + c] : 0.0;
            }
            stage8(x, E, As, kOzSliceA, r, k0);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
            for (int d = 0; d < kOzS; ++d)
                for (int sa = 0; sa <= d; ++sa)
                    for (int ks = 0; ks < nks; ++ks) {
                        const uint32_t off = (uint32_t)ks * 256;   // K = 16 FP16 = two core matrices
                        mma_f16(tmem + (uint32_t)(d * Npad), smem_desc(a0 + sa * kOzSliceA + off, 128, 1024),
                                smem_desc(b0 + (d - sa) * kOzSliceB + off, 128, 1024), idesc,
                                (sa | ks) ? 1u : 0u);
                    }
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: tensor-memory lane r (lanes 32 (warp % 4) ..) holds row i
        const double rs = E ? pow2(E - 1050) : 0.0;
        int a4[4] = {-1, -1, -1, -1};
        double w4[4] = {0.0, 0.0, 0.0, 0.0};
        if (i < n)
            for (int k = 0; k < 4; ++k) {
                a4[k] = icol[4 * i + k];
                w4[k] = ival[4 * i + k];
            }
        for (int c0 = 16 * h; c0 < Npad; c0 += 32) {
            long long acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0;
            for (int d = 0; d < kOzS; ++d) {
                uint32_t v[16];
                const uint32_t addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(d * Npad + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                    "%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const long long w = 1LL << (7 * (kOzS - 1 - d));
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] += (long long)__float2int_rn(__uint_as_float(v[q])) * w;
            }
            if (i < n)
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = c0 + q;
                    if (j < N) {
                        double iu = 0.0;
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (a4[k] >= 0) iu += w4[k] * U[(int64_t)a4[k] * N + j];
                        Psi[i * N + j] = fma((double)acc[q] * rs, colscale[j], iu);
                    }
                }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (!ok) {
        atomicExch(&g_tc_error, 1);
        mbar_wait(mb, phase ^ 1u);   // bounded second wait for the MMAs in flight
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

bool reconstruct_tc_supported(int N, int Na) { return N >= 1 && N <= 64 && Na >= 1 && Na <= kOzK; }

void launch_reconstruct_tc(int64_t n, const int32_t* icol, const double* ival, int N, const double* U,
                           int64_t nH, int Na, const double* Uhat, double* Psi, cudaStream_t s) {
    if (n <= 0) return;
    if (!reconstruct_tc_supported(N, Na)) fail(NAS_E_INVALID_ARG, "tensor-core reconstruction: N or Na out of range");
    const int sms = tc_sm_count();
    const int Npad = (N + 15) / 16 * 16;
    const int need = kOzS * Npad;
    const uint32_t ncols = need <= 32 ? 32u : need <= 64 ? 64u : need <= 128 ? 128u : need <= 256 ? 256u : 512u;
    const size_t smem = 1024 + (size_t)kOzS * (kOzSliceA + kOzSliceB);
    NAS_CUDA(cudaFuncSetAttribute(k_tc_reconstruct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t ntiles = (n + kOzM - 1) / kOzM;
    const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
    k_tc_reconstruct<<<grid, kOzThreads, smem, s>>>(n, icol, ival, N, Npad, ncols, U, nH, Na, Uhat, Psi);
    NAS_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Gram matrices G = X^T Y (X, Y [n][N], N <= 64) of the blocks of Sec. 3.3
// (gamma = U^T M U^, beta = U^T A U^, known symmetric), on the tensor cores by
// the same error-free integer slices.  The rows are taken in chunks of 64:
// per chunk, column c of X is written in fixed point against the largest
// exponent of that column within the chunk (E_c), column c' of Y likewise
// (F_c'), and D_d = sum_{s+t=d} A_s B_t over the chunk's 64 rows is exact in
// FP32 (|D_d| < 7 x 64 x 2^14 < 2^23).  The epilogue turns the chunk's
// product into one FP64 number per entry, acc 2^(E_c + F_c' - 2100) with
// acc = sum_d D_d 2^(7 (6 - d)) (exact int64), and adds it to the entry's
// FP64 running sum; so every chunk is rounded once and the chunks are added
// in FP64, as a blocked FP64 sum would.  A is X^T (the N columns of the chunk
// as rows, zero rows up to the MMA's M = 128), B is Y^T (N rows).  One
// persistent CTA per SM (256 threads) takes chunks blockIdx.x, + gridDim.x, ...;
// its 64 x 64 partial sums go to part[blockIdx.x], and k_tc_gram_finish adds
// the CTA partials in a fixed order and mirrors the upper triangle, so G is
// exactly symmetric and repeated calls are bit-identical.
__global__ void __launch_bounds__(kOzThreads) k_tc_gram(int64_t n, int N, int Npad, uint32_t ncols, const double* X,
                                                       const double* Y, double* part) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int emax[4][64], fmax[4][64];   // per row group: the columns' exponent maxima
    __shared__ int ech[64], fch[64];           // the chunk's column exponents E_c, F_c'
    unsigned char* base = oz_smem;
    base += (1024 - (smem_u32(base) & 1023)) & 1023;
    unsigned char* As = base;
    unsigned char* Bs = base + (size_t)kOzS * kOzSliceA;
    // staging: thread (c, g) takes column c of the chunk's rows [16 g, 16 g + 16)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, c = tid & 63, g = tid >> 6;
    const uint32_t mb = smem_u32(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // rows 64..127 of the A slices stay zero
    {
        uint4* p = reinterpret_cast<uint4*>(As);
        const int words = (int)(kOzS * kOzSliceA / 16);
        for (int w = tid; w < words; w += kOzThreads) p[w] = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_f16(kOzM, Npad);
    // epilogue: warps w with w % 4 < 2 read tensor-memory lanes m = 32 (w % 4) + lane
    // (the columns of X), the 16-column chunks 16 h and 16 h + 32 (h = w / 4)
    const bool ep = (warp & 3) < 2;
    const int m = 32 * (warp & 3) + lane, h = warp >> 2;
    double sum[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) sum[q] = 0.0;
    const int64_t nchunks = (n + 63) / 64;
    bool ok = true;
    uint32_t phase = 0;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t r0 = ch * 64 + 16 * g;
        double xv[16], yv[16];
        int ex = 0, ey = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const bool in = c < N && r0 + q < n;
            xv[q] = in ? X[(r0 + q) * N + c] : 0.0;
            yv[q] = in ? Y[(r0 + q) * N + c] : 0.0;
            ex = max(ex, biased_exp(xv[q]));
            ey = max(ey, biased_exp(yv[q]));
        }
        emax[g][c] = ex;
        fmax[g][c] = ey;
        __syncthreads();
        const int E = max(max(emax[0][c], emax[1][c]), max(emax[2][c], emax[3][c]));
        const int F = max(max(fmax[0][c], fmax[1][c]), max(fmax[2][c], fmax[3][c]));
        if (g == 0) {
            ech[c] = E;
            fch[c] = F;
        }
        stage8(xv, E, As, kOzSliceA, c, 16 * g);
        stage8(xv + 8, E, As, kOzSliceA, c, 16 * g + 8);
        stage8(yv, F, Bs, kOzSliceB, c, 16 * g);
        stage8(yv + 8, F, Bs, kOzSliceB, c, 16 * g + 8);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
            for (int d = 0; d < kOzS; ++d)
                for (int sa = 0; sa <= d; ++sa)
                    for (int ks = 0; ks < kOzK / 16; ++ks) {
                        const uint32_t off = (uint32_t)ks * 256;
                        mma_f16(tmem + (uint32_t)(d * Npad), smem_desc(a0 + sa * kOzSliceA + off, 128, 1024),
                                smem_desc(b0 + (d - sa) * kOzSliceB + off, 128, 1024), idesc,
                                (sa | ks) ? 1u : 0u);
                    }
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ep) {
            const int Em = ech[m];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int c0 = 16 * h + 32 * half;
                if (c0 >= Npad) break;
                long long acc[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = 0;
                for (int d = 0; d < kOzS; ++d) {
                    uint32_t v[16];
                    const uint32_t addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(d * Npad + c0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                        "%14,%15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15])
                        : "r"(addr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const long long w = 1LL << (7 * (kOzS - 1 - d));
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc[q] += (long long)__float2int_rn(__uint_as_float(v[q])) * w;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int Fj = fch[c0 + q];
                    if (Em && Fj) sum[16 * half + q] = fma((double)acc[q], pow2(Em + Fj - 2100), sum[16 * half + q]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (!ok) {
        atomicExch(&g_tc_error, 1);
        mbar_wait(mb, phase ^ 1u);
    }
    if (ep && m < N)
#pragma unroll
        for (int half = 0; half < 2; ++half)
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = 16 * h + 32 * half + q;
                if (j < N) part[((int64_t)blockIdx.x * N + m) * N + j] = sum[16 * half + q];
            }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// G[a][b] = G[b][a] = sum over CTAs (in order) of part[cta][a][b], a <= b
__global__ void k_tc_gram_finish(int nb, int N, const double* part, double* G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * N) return;
    const int a = t / N, b = t % N;
    if (a > b) return;
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += part[((int64_t)k * N + a) * N + b];
    G[a * N + b] = s;
    G[b * N + a] = s;
}

bool gram_tc_supported(int N) { return N >= 1 && N <= 64; }

int tc_sm_count() {
    static const int sms = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess)
            v = 0;
        cudaGetLastError();
        return v > 0 ? v : 1;
    }();
    return sms;
}

void launch_gram_sym_tc(int64_t n, int N, const double* X, const double* Y, double* partial, double* G,
                        cudaStream_t s) {
    if (!gram_tc_supported(N)) fail(NAS_E_INVALID_ARG, "tensor-core Gram: N out of range");
    const int Npad = (N + 15) / 16 * 16;
    const int need = kOzS * Npad;
    const uint32_t ncols = need <= 32 ? 32u : need <= 64 ? 64u : need <= 128 ? 128u : need <= 256 ? 256u : 512u;
    const size_t smem = 1024 + (size_t)kOzS * (kOzSliceA + kOzSliceB);
    const int64_t nchunks = (n + 63) / 64;
    if (nchunks == 0) {
        NAS_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * N * N, s));
        return;
    }
    const int grid = (int)(nchunks < tc_sm_count() ? nchunks : tc_sm_count());
    NAS_CUDA(cudaFuncSetAttribute(k_tc_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_gram<<<grid, kOzThreads, smem, s>>>(n, N, Npad, ncols, X, Y, partial);
    NAS_CHECK_LAUNCH();
    k_tc_gram_finish<<<grid_for((int64_t)N * N, 256), 256, 0, s>>>(grid, N, partial, G);
    NAS_CHECK_LAUNCH();
}

bool tc_error_take(cudaStream_t s) {
    int v = 0, zero = 0;
    NAS_CUDA(cudaMemcpyFromSymbolAsync(&v, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    NAS_CUDA(cudaStreamSynchronize(s));
    if (v) NAS_CUDA(cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    return v != 0;
}

}  // namespace nas

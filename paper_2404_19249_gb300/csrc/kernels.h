// Launchers of the nas GPU kernels (internal).  All kernels are FP64 and
// deterministic: every sum is taken in a fixed order (no floating-point
// atomics), so two runs on the same input give bit-identical results.
#pragma once

#include <string>

#include "common.h"

namespace nas {

// ------------------------------------------------------------ quadrature tables
// Upload the reference-element tables (quadrature points/weights, basis
// values, products and gradients) of the fine-space order to constant memory.
void fem_set_order(int order, int device);

// ------------------------------------------------------------ point location
struct LocateArgs {
    int64_t n_points;
    const int32_t* point_node;   // node id of each point
    const double* point_xyz;     // node coordinates [nnode][3]
    const double* cxyz;          // coarse vertices [nvc][3]
    const int32_t* ctet;         // coarse tets [nec][4]
    const int32_t* coarse_dof_of_node;  // [nvc] coarse dof or -1
    const int64_t* bptr;         // bucket CSR
    const int32_t* btet;
    double org[3], inv_h[3];
    int nb[3];
    int32_t* elem;               // out [n_points]
    int32_t* icol;               // out [n_points][4]
    double* ival;                // out [n_points][4]
    int* error_flag;             // set to 1 if a point is in no tetrahedron
};
void launch_locate(const LocateArgs& a, cudaStream_t s);

// ------------------------------------------------------------ element kernels
struct Mesh {
    int64_t ne;
    int nloc, nq;
    const double* vxyz;    // vertex coordinates [nv][3]
    const int32_t* elem;   // [ne][nloc] node ids; the first 4 are the vertices
};

// detJ > 0 check and quadrature weights Wq[e][q] = w_q |det J_e|
void launch_geometry(const Mesh& m, double* Wq, int* error_flag, cudaStream_t s);
// element stiffness matrices L[e][a][b] = sum_q Wq grad phi_a . grad phi_b
void launch_local_stiffness(const Mesh& m, double* L, cudaStream_t s);
// element mass matrices L[e][a][b] = sum_q Wq c_q phi_a phi_b (coef == nullptr: c = 1)
void launch_local_mass(const Mesh& m, const double* Wq, const double* coef, double* L, cudaStream_t s);
// external potential at quadrature points
struct Nuclei {
    int count;
    const double* R;   // device [count][3]
    const double* Z;   // device [count]
    int potential;     // nas_potential
    double smooth_a, omega;
};
void launch_vext(const Mesh& m, const Nuclei& nuc, double* vq, cudaStream_t s);
// nodal values (all nodes) -> values at quadrature points [ne][nq]
void launch_nodal_to_quad(const Mesh& m, const double* nodal, double* out, cudaStream_t s);
// LDA (Slater exchange + Perdew-Zunger correlation) pointwise; eps or vxc may be null
void launch_lda(int64_t cnt, const double* rho, double* eps, double* vxc, cudaStream_t s);
// coefficient of the nonlinear mass matrix: c = V_H(q) + V_xc(rho_in(q)), also
// storing eps_xc and V_xc at the quadrature points (xc = 0: V_H only)
void launch_nl_coef(const Mesh& m, const double* VH_nodal, const double* rho, int xc,
                    double* coef, double* eps, double* vxc, cudaStream_t s);
// rho[e][q] = sum_c occ[c] psi_c(x_q)^2, psi from dof values Psi[n][N]
void launch_density(const Mesh& m, const int32_t* dof_of_node, const double* Psi, int N,
                    const double* occ, double* rho, cudaStream_t s);
// the same density from pattern pairs: D on the fine pattern's upper entries
// (b >= a) once, then each element's quadrature points from its pairs' slots.
// slot [ne][10 | 55] is built once per mesh by launch_pair_slots (false if an
// interior pair is missing from the pattern); D holds nnz doubles; N <= 128
int64_t density_pair_count(const Mesh& m);
bool launch_pair_slots(const Mesh& m, const int32_t* dof_of_node, const int32_t* rowptr, const int32_t* col,
                       int32_t* slot, int* err, cudaStream_t s);
void launch_density_pairs(const Mesh& m, int64_t n, const int32_t* rowptr, const int32_t* col, const double* Psi,
                          int N, const double* occ, const int32_t* slot, double* D, double* rho, cudaStream_t s);
// element load vectors Lv[e][a] = sum_q Wq f_q phi_a
void launch_local_load(const Mesh& m, const double* Wq, const double* f, double* Lv, cudaStream_t s);
// out[s] = scale * sum_{k in [ptr[s],ptr[s+1])} src[idx[k]]
void launch_gather(int64_t nslots, const int64_t* ptr, const int32_t* idx, const double* src,
                   double scale, double* out, cudaStream_t s);
// charge moments: out[0] = int rho, out[1..3] = int x rho, out[4..9] = int x_i x_j rho
// (i<=j: xx, xy, xz, yy, yz, zz); quadrature positions recomputed from vertices.
void launch_moments(const Mesh& m, const double* Wq, const double* rho, double* partial,
                    double* out, cudaStream_t s);
// boundary values of V_H (monopole + optional quadrupole) written into V_nodal
// at the boundary nodes and into wB[nb]
void launch_boundary_values(int64_t nb, const int32_t* bnd_node, const double* node_xyz,
                            const double* moments, int multipole, double* wB, double* V_nodal,
                            cudaStream_t s);
// out[e][q] = sum_c A_c(x_q) U_c(x_q) for dof values A, U [n][N]
void launch_pair_density(const Mesh& m, const int32_t* dof_of_node, const double* A, const double* U, int N,
                         double* out, cudaStream_t s);
// out[k][c] = sum_{e,q} W_eq w_eq dV_ext/dp_(k,c)(x_q), p = (R_k x, y, z, Z_k);
// partial: scratch of 1216*32 doubles (Coulomb or smoothed Coulomb)
void launch_vext_grad(const Mesh& m, const Nuclei& nuc, const double* Wq, const double* w, double* partial,
                      double* out, cudaStream_t s);
// gather nodal values at the dofs: x[i] = V_nodal[dof_node[i]]
void launch_nodal_to_dof(int64_t n, const int32_t* dof_node, const double* V_nodal, double* x,
                         cudaStream_t s);
// scatter dof values into nodal array: V_nodal[dof_node[i]] = x[i]
void launch_dof_to_nodal(int64_t n, const int32_t* dof_node, const double* x, double* V_nodal,
                         cudaStream_t s);

// ------------------------------------------------------------ sparse / dense linear algebra
struct Csr {
    int64_t n_rows;
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
    int64_t rowptr_nnz = 0;   // nnz (host-side bookkeeping for byte counts)
};
// Y = alpha * A X (+ beta Y), X [ncols][N], Y [n_rows][N]
// SpMM with N > 1 interleaved right-hand sides through the layout autotuner
// (kernels_spmm.cu); N = 1 takes the 8-lanes-per-row SpMV
void launch_spmm_tuned(const Csr& A, int N, const double* X, double* Y, double alpha, double beta, cudaStream_t s);
// autotuner control and record (kernels_spmm.cu)
void spmm_set_tuning(bool on);
void spmm_force_layout(const int32_t* rowptr, int64_t n, int N, int bytes, int id);
std::string spmm_tuning_report();
int spmm_num_layouts();
const char* spmm_layout_name(int id);
void launch_spmm_layout(int id, int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, int N,
                        const double* X, double* Y, cudaStream_t s);
void launch_spmm_layout(int id, int64_t n, const int32_t* rowptr, const int32_t* col, const float* val, int N,
                        const float* X, float* Y, cudaStream_t s);
void launch_spmm(const Csr& A, int N, const double* X, double* Y, double alpha, double beta,
                 cudaStream_t s);

// Deterministic column-wise weighted dot products: out[k][c] = sum_i w_i X_k[i][c] Y_k[i][c]
// for k < npairs (w == nullptr: w_i = 1).  partial: scratch of
// reduce_partial_size(N*npairs) doubles.
int64_t reduce_partial_size(int64_t width);
void launch_coldots(int64_t n, int N, int npairs, const double* const* X, const double* const* Y,
                    const double* w, double* partial, double* out, cudaStream_t s);

// Block PCG vector updates with per-column scalars held on the device.
struct PcgCols {
    int N;
    double* rz;      // [N] r.z of the current iterate
    double* pq;      // [N]
    double* rz_new;  // [N]
    double* rr;      // [N]
    double* bb;      // [N] ||b||^2
    double* alpha;   // [N]
    double* beta;    // [N]
    int* active;     // [N]
    int* breakdown;  // [1]
    double tol2;     // tol^2
};
// alpha_c = rz_c / pq_c for active columns (pq <= 0 or non-finite -> breakdown)
void launch_pcg_alpha(const PcgCols& c, cudaStream_t s);
// beta_c = rz_new_c / rz_c; rz <- rz_new; deactivate converged columns
void launch_pcg_beta(const PcgCols& c, cudaStream_t s);
// X += alpha P, R -= alpha Q, Z = Dinv R (per column alpha, inactive columns untouched)
void launch_pcg_update(int64_t n, int N, const double* alpha, const int* active, const double* P,
                       const double* Q, const double* Dinv, double* X, double* R, double* Z,
                       cudaStream_t s);
// P = Z + beta P (active columns)
void launch_pcg_direction(int64_t n, int N, const double* beta, const int* active, const double* Z,
                          double* P, cudaStream_t s);
// Y[i][c] *= s[c]
void launch_scale_cols(int64_t n, int N, const double* s_dev, double* Y, cudaStream_t s);
// Z = Dinv R
void launch_scale_rows(int64_t n, int N, const double* Dinv, const double* R, double* Z,
                       cudaStream_t s);
// R = B - R (elementwise), used after R = A X
void launch_sub_from(int64_t cnt, const double* B, double* R, cudaStream_t s);
// out = a*x + b*y elementwise
void launch_axpby(int64_t cnt, double a, const double* x, double b, const double* y, double* out,
                  cudaStream_t s);
// Dinv[i] = 1 / A_ii
void launch_inv_diag(const Csr& A, double* Dinv, cudaStream_t s);
// val_out = a*v1 + b*v2 + c*v3 (CSR value arrays with a common pattern; v3 may be null)
void launch_combine3(int64_t nnz, double a, const double* v1, double b, const double* v2, double c,
                     const double* v3, double* out, cudaStream_t s);

// G[a][b] = sum_i X[i][a] Y[i][b]  (X [n][Nx], Y [n][Ny]) deterministic; partial scratch
// of gram_partial_size(Nx*Ny) doubles
int64_t gram_partial_size(int64_t width);
// G = X^T Y for a product known to be symmetric (X, Y [n][N]): the upper
// triangle is summed and mirrored, so G is exactly symmetric; partial holds
// reduce_partial_size(N * N) doubles
void launch_gram_sym(int64_t n, int N, const double* X, const double* Y, double* partial, double* G,
                     cudaStream_t s);
void launch_gram(int64_t n, int Nx, const double* X, int Ny, const double* Y, double* partial,
                 double* G, cudaStream_t s);
// launch_gram_sym on the tensor cores (error-free integer slices per 64-row
// chunk, FP64 sums across chunks; kernels_tc.cu); 1 <= N <= 64; partial holds
// (number of SMs) x N^2 doubles
bool gram_tc_supported(int N);
void launch_gram_sym_tc(int64_t n, int N, const double* X, const double* Y, double* partial, double* G,
                        cudaStream_t s);
// multiprocessors of the current device (queried once)
int tc_sm_count();

// Balanced pieces of a segmented list (see PieceMap on the host): pieces of
// segment a are [seg_piece[a], seg_piece[a+1]); piece q covers list entries
// [piece_start[q], piece_start[q+1]).
struct Pieces {
    int64_t nseg = 0, npieces = 0;
    const int32_t* seg_piece = nullptr;
    const int64_t* piece_start = nullptr;
};
// out[a][c] = sum_{p in segment a} tval[p] Y[trow[p]][c]   (I^T Y over the I^T
// rows split into pieces); partial: scratch of npieces * N doubles
// FP32 Y and weights, FP64 piece sums and result
void launch_transpose_apply_f32(const Pieces& pc, const int32_t* trow, const float* tval, int N, const float* Y,
                                double* partial, double* out, cudaStream_t s);
// Z += I Yc for a coarse block Yc [nH][N] (FP64), Z [n][N] FP64 or FP32
void launch_prolong_add(int64_t n, int N, const int32_t* icol, const double* ival, const double* Yc, double* Z,
                        cudaStream_t s);
void launch_prolong_add(int64_t n, int N, const int32_t* icol, const float* ival, const double* Yc, float* Z,
                        cudaStream_t s);
void launch_transpose_apply(const Pieces& pc, const int32_t* trow, const double* tval, int N, const double* Y,
                            double* partial, double* out, cudaStream_t s);
// Psi[i][c] = sum_k ival[i][k] uH[icol[i][k]][c] + sum_j Uhat[i][j] alpha[j][c]
// U = [uH ; alpha] is [(nH + Na)][N] on the device; Na may be 0.
void launch_reconstruct(int64_t n, const int32_t* icol, const double* ival, int N, const double* U,
                        int64_t nH, int Na, const double* Uhat, double* Psi, cudaStream_t s);
// the same with the dense part on the tensor cores (error-free integer
// slices, FP64 accuracy; kernels_tc.cu); needs 1 <= N <= 64 and 1 <= Na <= 64
bool reconstruct_tc_supported(int N, int Na);
void launch_reconstruct_tc(int64_t n, const int32_t* icol, const double* ival, int N, const double* U,
                           int64_t nH, int Na, const double* Uhat, double* Psi, cudaStream_t s);
// Galerkin stage 1: W[s] = sum_{q in list} A[q>>2] * ival[col[q>>2]*4 + (q&3)]
void launch_galerkin1(int64_t nw, const int64_t* ptr, const int32_t* con, const double* A,
                      const int32_t* col, const double* ival, double* W, cudaStream_t s);
// Galerkin stage 2: H[t] = sum_{r in list t} ival[wrow[r>>2]*4 + (r&3)] * W[r>>2]
// over the lists split into pieces; partial: scratch of npieces doubles
void launch_galerkin2(const Pieces& pc, const int32_t* con, const double* W, const int32_t* wrow,
                      const double* ival, double* partial, double* H, cudaStream_t s);

// ------------------------------------------------------------ small pencil on the device
// Arrow-structured symmetric matrix of the small problem (the 2 x 2 block form of F_A, F_B in Sec. 3.3):
// [[S, Bd], [Bd^T, Cd]], S sparse nH x nH (CSR, full symmetric storage),
// Bd dense [nH][Na], Cd dense [Na][Na]; all pointers on the device.
struct ArrowDev {
    int64_t nH = 0;
    int Na = 0;
    const int32_t* ptr = nullptr;
    const int32_t* col = nullptr;
    const double* sval = nullptr;
    const double* Bd = nullptr;
    const double* Cd = nullptr;
};
// A matrix given as up to six column blocks side by side: column a of the
// whole is column (a - offset) of block u, block u row-major with row stride ld[u].
struct ColBlocks {
    static const int kMax = 6;
    const double* p[kMax] = {};
    int ld[kMax] = {};
    int w[kMax] = {};
    int nblk = 0;
    __host__ __device__ int ncols() const {
        int c = 0;
        for (int u = 0; u < nblk; ++u) c += w[u];
        return c;
    }
    static ColBlocks one(const double* a, int ld, int w) {
        ColBlocks c;
        c.p[0] = a;
        c.ld[0] = ld;
        c.w[0] = w;
        c.nblk = 1;
        return c;
    }
    void add(const double* a, int ldv, int wv) {
        if (nblk >= kMax) return;  // callers never exceed kMax blocks
        p[nblk] = a;
        ld[nblk] = ldv;
        w[nblk] = wv;
        ++nblk;
    }
};
// Y = F X for X, Y [m][w]; partial: gram_tiles_partial_size(nH, Na, w) doubles,
// G: Na*w doubles of scratch
void launch_arrow_apply(const ArrowDev& F, int w, const double* X, double* Y, double* partial, double* G,
                        cudaStream_t s);
// YA = A X and YB = B X for two arrow matrices with the same pattern (X read
// once); partial: gram_tiles_partial_size(nH, 2 Na, w), G: 2 Na w doubles
void launch_arrow_apply2(const ArrowDev& A, const ArrowDev& B, int w, const double* X, double* YA, double* YB,
                         double* partial, double* G, cudaStream_t s);
// G[a][b] = sum_{i<m} L(i,a) R(i,b) (deterministic); partial scratch of
// gram_tiles_partial_size(m, ncols(L), ncols(R)) doubles
int64_t gram_tiles_partial_size(int64_t m, int La, int Rb);
void launch_gram_tiles(int64_t m, const ColBlocks& L, const ColBlocks& R, double* partial, double* G,
                       cudaStream_t s);
// Y[i][j] = alpha sum_a S(i,a) C[a][j] + beta Y[i][j], C row-major [ncols(S)][kout]
void launch_cols_mult(int64_t m, const ColBlocks& S, const double* C, int kout, double alpha, double beta,
                      double* Y, cudaStream_t s);
// dst[i][q] = src[i][idx[q]]: columns idx[0..kq) of src [m][k] into dst [m][kq]
void launch_gather_cols(int64_t m, int k, int kq, const int* idx, const double* src, double* dst, cudaStream_t s);
// R = AX - BX diag(theta) for [m][k] arrays (theta on the device)
void launch_eig_resid(int64_t m, int k, const double* AX, const double* BX, const double* theta, double* R,
                      cudaStream_t s);
// columns of A1, A2, A3 ([m][k], any may be null) scaled by 1/sqrt(nrm[j])
void launch_inv_sqrt_scale(int64_t m, int k, const double* nrm, double* A1, double* A2, double* A3,
                           cudaStream_t s);
// LOBPCG preconditioner with a dense coarse block: W = T R on the first nH rows
// (T FP32 [nH][nH], e.g. the inverse coarse stiffness), W = Dinv R on the
// remaining m - nH rows; R, W [m][k] FP64, k <= 32; part: FP32 scratch of
// dense_precond_part_size(nH, k)
int64_t dense_precond_part_size(int64_t nH, int k);
// the same product on the tensor cores (kernels_tc.cu): tcgen05.mma of kind
// tf32 with split-TF32 operands (FP32-level accuracy), FP32 accumulator in
// tensor memory; k <= 256; part holds dense_precond_tc_part_size doubles' worth
// of floats
void launch_dense_precond_tc(int64_t nH, int64_t m, int k, const float* T, const double* R, const double* Dinv,
                             float* part, double* W, cudaStream_t s);
int64_t dense_precond_tc_part_size(int64_t nH, int k);
// true if a tensor-core CTA gave up waiting on its mbarrier since the last
// call (the flag is cleared); synchronises s
bool tc_error_take(cudaStream_t s);
void launch_dense_precond(int64_t nH, int64_t m, int k, const float* T, const double* R, const double* Dinv,
                          float* part, double* W, cudaStream_t s);
// T[i] = 1 / (A_ii - sigma B_ii), diag_slot[i] = CSR slot of (i, i) in the coarse block
void launch_eig_precond(const ArrowDev& A, const ArrowDev& B, const int32_t* diag_slot, double sigma, double* T,
                        cudaStream_t s);

// Fused single right-hand-side PCG (Poisson): device state of one solve, in
// FP64 (Pcg1) or FP32 (Pcg1f, the inner solver of the mixed-precision mode).
template <typename T>
struct Pcg1T {
    int64_t n;
    const int32_t* rowptr;
    const int32_t* col;
    const T* val;
    const T* dinv;
    T *x, *r, *z, *p, *q;
    T *part_pq, *part_rz, *part_rr;  // [pcg1_blocks()] per-block partial sums
    T* scal;                          // [0],[1] rz (by iteration parity), [2] stop threshold, [3] r.r
    int* active;                      // cleared when ||r||^2 <= tol2 scal[2]
    int* breakdown;
    int* iters;
    T tol2;
    // optional two-level preconditioner z = D^-1 r + I K_H^-1 I^T r
    int two_level = 0;
    int64_t nH = 0;
    Pieces tpc;                      // I^T rows (coarse) split into balanced pieces
    const int32_t* trow = nullptr;   // I^T entries: fine row and weight
    const T* tval = nullptr;
    T* cpart = nullptr;              // [tpc.npieces] piece sums of I^T r
    const int32_t* icol = nullptr;   // I as ELL [n][4]
    const T* ival = nullptr;
    const T* khinv = nullptr;        // dense K_H^-1 [nH][nH]
    T* cvec = nullptr;               // [nH]
    T* yvec = nullptr;               // [nH]
    // optional sliced-ELL copy of the matrix (32 rows per slice, column-major
    // within a slice, zero-padded to the slice's longest row); used for q = A p
    // when sell_ptr is set
    const int64_t* sell_ptr = nullptr;  // [n_slices + 1] entry offsets
    const int32_t* sell_col = nullptr;
    const T* sell_val = nullptr;
};
using Pcg1 = Pcg1T<double>;
using Pcg1f = Pcg1T<float>;
int pcg1_blocks();
// one PCG iteration (3 kernels, 7 with the two-level preconditioner);
// par = iteration parity (selects the rz slot).  ev0/ev1 (optional) are
// recorded right before and after the SpMV kernel.
void launch_pcg1_iteration(const Pcg1& s, int par, int lanes_per_row, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                           cudaEvent_t ev1 = nullptr);
void launch_pcg1_iteration(const Pcg1f& s, int par, int lanes_per_row, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                           cudaEvent_t ev1 = nullptr);
int pcg1_kernels_per_iteration(int two_level, int64_t npieces);
// Persistent (cooperative) form of the two-level FP64 iteration with the
// sliced-ELL matrix: one launch runs up to `chunk` iterations (starting at
// parity 0) with grid-wide barriers between the phases; bar = two zeroed
// unsigned counters, err = flag set if a barrier wait exceeded its limit.
// pcg1_fused_blocks() is the co-resident grid size (0: no cooperative launch).
int pcg1_fused_blocks();
void launch_pcg1_fused(const Pcg1& s, unsigned* bar, int* err, int chunk, int blocks, cudaStream_t st);
// sliced ELL (32 rows per slice) of a CSR matrix: sell_ptr from the host,
// columns and values filled on the device (padding: column = row, value 0)
void launch_sell_fill(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                      const int64_t* sell_ptr, int64_t n_slices, int32_t* sell_col, double* sell_val, cudaStream_t st);
// z = D^-1 r + I K_H^-1 I^T r and partial sums of r.z (two-level only)
void launch_pcg1_coarse_correction(const Pcg1& s, cudaStream_t st);
void launch_pcg1_coarse_correction(const Pcg1f& s, cudaStream_t st);
// FP32 inner solve start from e = 0 (p = z, x = 0, partial sums of r.z, r.r)
void launch_pcg1_start(const Pcg1f& s, cudaStream_t st);
void launch_cast_to_f32(int64_t n, const double* a, float* b, cudaStream_t st);
// FP32 block PCG pieces (mixed precision, the N shifted problems): SpMM with
// N interleaved columns; column dots (FP32 products, FP64 across threads);
// updates with FP64 per-column scalars
void launch_spmm_f32(int64_t n_rows, const int32_t* rowptr, const int32_t* col, const float* val, int N,
                     const float* X, float* Y, cudaStream_t s);
void launch_coldots_f32(int64_t n, int N, int npairs, const float* const* X, const float* const* Y,
                        double* partial, double* out, cudaStream_t s);
void launch_pcg_update_f32(int64_t n, int N, const double* alpha, const int* active, const float* P, const float* Q,
                           const float* Dinv, float* X, float* R, float* Z, cudaStream_t s);
void launch_pcg_direction_f32(int64_t n, int N, const double* beta, const int* active, const float* Z, float* P,
                              cudaStream_t s);
void launch_scale_rows_f32(int64_t n, int N, const float* Dinv, const float* R, float* Z, cudaStream_t s);
void launch_add_f32(int64_t n, const float* e, double* x, cudaStream_t st);

// Anderson: given F^0..F^m (pointers), w, compute the k x k matrix
// A[a][b] = (F^m - F^a, F^m - F^b) and rhs[a] = (F^m - F^a, F^m), k = m;
// out = [A (k*k), rhs (k)] deterministic
// partial-sum buffer size (doubles) of launch_anderson_dots for m previous entries
int64_t anderson_partial_size(int m);
void launch_anderson_dots(int64_t cnt, int m, const double* const* F, const double* w,
                          double* partial, double* out, cudaStream_t s);
// rho_new = rin_m + sum_a alpha_a (rin_a - rin_m) + beta (F_m + sum_a alpha_a (F_a - F_m))
void launch_anderson_mix(int64_t cnt, int m, const double* const* rin, const double* const* F,
                         const double* alpha, double beta, double* rho_new, cudaStream_t s);

}  // namespace nas

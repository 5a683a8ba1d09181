// Element-level finite element kernels (Sec. 2 discretisation, Sec. 3.1
// potentials, Sec. 3.3, the matrices A_h^L and A_h^NL): geometry, element matrices, potentials
// and densities at quadrature points.  One thread per element; reference
// element tables live in constant memory (every thread of a warp reads the
// same entry at the same time, a broadcast).
//
// Quadrature (the paper leaves it open): P1 uses the symmetric 4-point
// degree-2 rule, P2 the symmetric 14-point degree-5 rule with orbits
// (a,a,a,1-3a) x4, (b,b,b,1-3b) x4, (c,c,1/2-c,1/2-c) x6 whose parameters
// solve the moment equations of all monomials of degree <= 5.
#include <cmath>
#include <mutex>

#include "kernels.h"

namespace nas {

template <int ORDER> struct El;
template <> struct El<1> { static constexpr int NLOC = 4, NQ = 4, NP = 10; };
template <> struct El<2> { static constexpr int NLOC = 10, NQ = 14, NP = 55; };

struct Tables1 { double bary[4][4]; double w[4]; double phi[4][4]; double pp[4][10]; double dphi[4][4][3]; };
struct Tables2 { double bary[14][4]; double w[14]; double phi[14][10]; double pp[14][55]; double dphi[14][10][3]; };

__constant__ Tables1 c_t1;
__constant__ Tables2 c_t2;

template <int ORDER> __device__ __forceinline__ const double* T_w();
template <> __device__ __forceinline__ const double* T_w<1>() { return c_t1.w; }
template <> __device__ __forceinline__ const double* T_w<2>() { return c_t2.w; }
template <int ORDER> __device__ __forceinline__ double T_bary(int q, int k);
template <> __device__ __forceinline__ double T_bary<1>(int q, int k) { return c_t1.bary[q][k]; }
template <> __device__ __forceinline__ double T_bary<2>(int q, int k) { return c_t2.bary[q][k]; }
template <int ORDER> __device__ __forceinline__ double T_phi(int q, int a);
template <> __device__ __forceinline__ double T_phi<1>(int q, int a) { return c_t1.phi[q][a]; }
template <> __device__ __forceinline__ double T_phi<2>(int q, int a) { return c_t2.phi[q][a]; }
template <int ORDER> __device__ __forceinline__ double T_pp(int q, int p);
template <> __device__ __forceinline__ double T_pp<1>(int q, int p) { return c_t1.pp[q][p]; }
template <> __device__ __forceinline__ double T_pp<2>(int q, int p) { return c_t2.pp[q][p]; }
template <int ORDER> __device__ __forceinline__ double T_dphi(int q, int a, int d);
template <> __device__ __forceinline__ double T_dphi<1>(int q, int a, int d) { return c_t1.dphi[q][a][d]; }
template <> __device__ __forceinline__ double T_dphi<2>(int q, int a, int d) { return c_t2.dphi[q][a][d]; }

// ------------------------------------------------------------------ host tables
static const int kEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const double kDL[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

static void basis(int order, const double* L, double* phi, double (*dphi)[3]) {
    if (order == 1) {
        for (int a = 0; a < 4; ++a) {
            phi[a] = L[a];
            for (int d = 0; d < 3; ++d) dphi[a][d] = kDL[a][d];
        }
        return;
    }
    for (int i = 0; i < 4; ++i) {
        phi[i] = L[i] * (2.0 * L[i] - 1.0);
        for (int d = 0; d < 3; ++d) dphi[i][d] = (4.0 * L[i] - 1.0) * kDL[i][d];
    }
    for (int k = 0; k < 6; ++k) {
        int i = kEdge[k][0], j = kEdge[k][1];
        phi[4 + k] = 4.0 * L[i] * L[j];
        for (int d = 0; d < 3; ++d) dphi[4 + k][d] = 4.0 * (L[j] * kDL[i][d] + L[i] * kDL[j][d]);
    }
}

template <class T>
static void fill_tables(T& t, int order, int nq, int nloc, const double (*bary)[4], const double* w) {
    for (int q = 0; q < nq; ++q) {
        for (int k = 0; k < 4; ++k) t.bary[q][k] = bary[q][k];
        t.w[q] = w[q];
        double phi[10], dphi[10][3];
        basis(order, bary[q], phi, dphi);
        int p = 0;
        for (int a = 0; a < nloc; ++a) {
            t.phi[q][a] = phi[a];
            for (int d = 0; d < 3; ++d) t.dphi[q][a][d] = dphi[a][d];
            for (int b = a; b < nloc; ++b) t.pp[q][p++] = phi[a] * phi[b];
        }
    }
}

void fem_set_order(int /*order*/, int device) {
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0 || device >= 64) fail(NAS_E_INVALID_ARG, "device id");
    if (done[device]) return;
    // P1: 4 points (b,b,b,a) with a = (5+3 sqrt5)/20, b = (5-sqrt5)/20, w = 1/24
    Tables1 t1;
    {
        double a = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, b = (5.0 - std::sqrt(5.0)) / 20.0;
        double bary[4][4], w[4];
        for (int q = 0; q < 4; ++q) {
            for (int k = 0; k < 4; ++k) bary[q][k] = (k == q) ? a : b;
            w[q] = 1.0 / 24.0;
        }
        fill_tables(t1, 1, 4, 4, bary, w);
    }
    // P2: 14 points, degree 5
    Tables2 t2;
    {
        const double a = 0.09273525031089122640232391, b = 0.3108859192633006097973457,
                     c = 0.04550370412564964949188053;
        const double w1 = 0.01224884051939365825728503, w2 = 0.01878132095300264179986428,
                     w3 = 0.007091003462846911073011571;
        double bary[14][4], w[14];
        int q = 0;
        const double tv[2] = {a, b}, tw[2] = {w1, w2};
        for (int o = 0; o < 2; ++o)
            for (int k = 0; k < 4; ++k, ++q) {
                for (int j = 0; j < 4; ++j) bary[q][j] = tv[o];
                bary[q][k] = 1.0 - 3.0 * tv[o];
                w[q] = tw[o];
            }
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j, ++q) {
                for (int k = 0; k < 4; ++k) bary[q][k] = 0.5 - c;
                bary[q][i] = c;
                bary[q][j] = c;
                w[q] = w3;
            }
        fill_tables(t2, 2, 14, 10, bary, w);
    }
    NAS_CUDA(cudaMemcpyToSymbol(c_t1, &t1, sizeof(t1)));
    NAS_CUDA(cudaMemcpyToSymbol(c_t2, &t2, sizeof(t2)));
    done[device] = true;
}

// ------------------------------------------------------------------ device helpers
struct Jac {
    double J[3][3];  // columns v1-v0, v2-v0, v3-v0
    double det;
};

__device__ __forceinline__ void load_vertices(const Mesh& m, int64_t e, double v[4][3]) {
    for (int k = 0; k < 4; ++k) {
        int u = m.elem[e * m.nloc + k];
        v[k][0] = m.vxyz[3 * u];
        v[k][1] = m.vxyz[3 * u + 1];
        v[k][2] = m.vxyz[3 * u + 2];
    }
}

__device__ __forceinline__ void jacobian(const double v[4][3], Jac& j) {
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) j.J[r][c] = v[c + 1][r] - v[0][r];
    j.det = j.J[0][0] * (j.J[1][1] * j.J[2][2] - j.J[1][2] * j.J[2][1]) -
            j.J[0][1] * (j.J[1][0] * j.J[2][2] - j.J[1][2] * j.J[2][0]) +
            j.J[0][2] * (j.J[1][0] * j.J[2][1] - j.J[1][1] * j.J[2][0]);
}

// G = J^{-T}: grad_x phi = G grad_ref phi
__device__ __forceinline__ void inv_transpose(const Jac& j, double G[3][3]) {
    const double (*J)[3] = j.J;
    double id = 1.0 / j.det;
    // cofactor matrix C; J^{-1} = C^T / det, so J^{-T} = C / det
    G[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
    G[0][1] = -(J[1][0] * J[2][2] - J[1][2] * J[2][0]) * id;
    G[0][2] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
    G[1][0] = -(J[0][1] * J[2][2] - J[0][2] * J[2][1]) * id;
    G[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    G[1][2] = -(J[0][0] * J[2][1] - J[0][1] * J[2][0]) * id;
    G[2][0] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    G[2][1] = -(J[0][0] * J[1][2] - J[0][2] * J[1][0]) * id;
    G[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
}

// Slater exchange + Perdew-Zunger correlation (Sec. 3.1, the exchange and correlation potentials);
// rho <= 1e-30 gives 0; r_s = 1 takes the r_s >= 1 branch.
__device__ __forceinline__ void lda_point(double rho, double& eps, double& v) {
    if (!(rho > 1e-30)) {
        eps = 0.0;
        v = 0.0;
        return;
    }
    const double A = 0.0311, B = -0.048, GAMMA = -0.1423, BETA1 = 1.0529, BETA2 = 0.3334,
                 C = 0.0020, D = -0.0116;
    // one cube root per point (sm_103 issues 2 FP64 FMA per clock per SM):
    // v_x = -(3 rho / pi)^(1/3) = -CX rho^(1/3), eps_x = 3/4 v_x,
    // r_s = (3 / (4 pi rho))^(1/3) = CRS / rho^(1/3)
    const double CX = 0.9847450218426965411790, CRS = 0.6203504908994000166680;
    const double r13 = cbrt(rho);
    const double v_x = -CX * r13;
    const double eps_x = 0.75 * v_x;
    const double rs = CRS / r13;
    double eps_c, v_c;
    if (rs < 1.0) {
        double ln = log(rs);
        eps_c = A * ln + B + C * rs * ln + D * rs;
        v_c = A * ln + (B - A / 3.0) + (2.0 / 3.0) * C * rs * ln + (1.0 / 3.0) * (2.0 * D - C) * rs;
    } else {
        double sq = sqrt(rs);
        double inv_den = 1.0 / (1.0 + BETA1 * sq + BETA2 * rs);
        eps_c = GAMMA * inv_den;
        v_c = eps_c * (1.0 + (7.0 / 6.0) * BETA1 * sq + (4.0 / 3.0) * BETA2 * rs) * inv_den;
    }
    eps = eps_x + eps_c;
    v = v_x + v_c;
}

// ------------------------------------------------------------------ kernels
template <int ORDER>
__global__ void k_geometry(Mesh m, double* Wq, int* err) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    double v[4][3];
    load_vertices(m, e, v);
    Jac j;
    jacobian(v, j);
    if (!(j.det > 0.0)) atomicExch(err, 1);
    constexpr int NQ = El<ORDER>::NQ;
    for (int q = 0; q < NQ; ++q) Wq[e * NQ + q] = T_w<ORDER>()[q] * j.det;
}

template <int ORDER>
__global__ void __launch_bounds__(128) k_local_stiffness(Mesh m, double* L) {
    constexpr int NL = El<ORDER>::NLOC, NQ = El<ORDER>::NQ, NP = El<ORDER>::NP;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    double v[4][3];
    load_vertices(m, e, v);
    Jac j;
    jacobian(v, j);
    double G[3][3];
    inv_transpose(j, G);
    double K[NP];
    for (int p = 0; p < NP; ++p) K[p] = 0.0;
    for (int q = 0; q < NQ; ++q) {
        double g[NL][3];
        for (int a = 0; a < NL; ++a) {
            double r0 = T_dphi<ORDER>(q, a, 0), r1 = T_dphi<ORDER>(q, a, 1), r2 = T_dphi<ORDER>(q, a, 2);
            for (int d = 0; d < 3; ++d) g[a][d] = G[d][0] * r0 + G[d][1] * r1 + G[d][2] * r2;
        }
        double wq = T_w<ORDER>()[q] * j.det;
        int p = 0;
        for (int a = 0; a < NL; ++a)
            for (int b = a; b < NL; ++b, ++p)
                K[p] += wq * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
    }
    double* out = L + e * NL * NL;
    int p = 0;
    for (int a = 0; a < NL; ++a)
        for (int b = a; b < NL; ++b, ++p) {
            out[a * NL + b] = K[p];
            out[b * NL + a] = K[p];
        }
}

template <int ORDER>
__global__ void __launch_bounds__(128) k_local_mass(Mesh m, const double* Wq, const double* coef, double* L) {
    constexpr int NL = El<ORDER>::NLOC, NQ = El<ORDER>::NQ;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    double c[NQ];
    for (int q = 0; q < NQ; ++q) {
        double w = Wq[e * NQ + q];
        c[q] = coef ? w * coef[e * NQ + q] : w;
    }
    double* out = L + e * NL * NL;
    int p = 0;
    for (int a = 0; a < NL; ++a)
        for (int b = a; b < NL; ++b, ++p) {
            double s = 0.0;
            for (int q = 0; q < NQ; ++q) s += c[q] * T_pp<ORDER>(q, p);
            out[a * NL + b] = s;
            out[b * NL + a] = s;
        }
}

template <int ORDER>
__global__ void k_vext(Mesh m, Nuclei nuc, double* vq) {
    constexpr int NQ = El<ORDER>::NQ;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    double v[4][3];
    load_vertices(m, e, v);
    for (int q = 0; q < NQ; ++q) {
        double x[3];
        for (int d = 0; d < 3; ++d)
            x[d] = T_bary<ORDER>(q, 0) * v[0][d] + T_bary<ORDER>(q, 1) * v[1][d] +
                   T_bary<ORDER>(q, 2) * v[2][d] + T_bary<ORDER>(q, 3) * v[3][d];
        double V = 0.0;
        if (nuc.potential == NAS_POT_HARMONIC) {
            V = 0.5 * nuc.omega * nuc.omega * (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        } else {
            for (int k = 0; k < nuc.count; ++k) {
                double dx = x[0] - nuc.R[3 * k], dy = x[1] - nuc.R[3 * k + 1], dz = x[2] - nuc.R[3 * k + 2];
                double r2 = dx * dx + dy * dy + dz * dz;
                if (nuc.potential == NAS_POT_SMOOTHED) r2 += nuc.smooth_a * nuc.smooth_a;
                V -= nuc.Z[k] / sqrt(r2);
            }
        }
        vq[e * NQ + q] = V;
    }
}

template <int ORDER>
__global__ void k_nodal_to_quad(Mesh m, const double* nodal, double* out) {
    constexpr int NL = El<ORDER>::NLOC, NQ = El<ORDER>::NQ;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    double u[NL];
    for (int a = 0; a < NL; ++a) u[a] = nodal[m.elem[e * NL + a]];
    for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int a = 0; a < NL; ++a) s += T_phi<ORDER>(q, a) * u[a];
        out[e * NQ + q] = s;
    }
}

template <int ORDER>
__global__ void k_nl_coef(Mesh m, const double* VH, const double* rho, int xc, double* coef,
                          double* eps, double* vxc) {
    constexpr int NL = El<ORDER>::NLOC, NQ = El<ORDER>::NQ;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    double u[NL];
    for (int a = 0; a < NL; ++a) u[a] = VH ? VH[m.elem[e * NL + a]] : 0.0;
    for (int q = 0; q < NQ; ++q) {
        double vh = 0.0;
        for (int a = 0; a < NL; ++a) vh += T_phi<ORDER>(q, a) * u[a];
        double ex = 0.0, vx = 0.0;
        if (xc) lda_point(rho[e * NQ + q], ex, vx);
        coef[e * NQ + q] = vh + vx;
        if (eps) eps[e * NQ + q] = ex;
        if (vxc) vxc[e * NQ + q] = vx;
    }
}

__global__ void k_lda(int64_t cnt, const double* rho, double* eps, double* vxc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    double e, v;
    lda_point(rho[i], e, v);
    if (eps) eps[i] = e;
    if (vxc) vxc[i] = v;
}

// rho(q) = sum_{a<=b} (2 - delta_ab) phi_a phi_b D_ab with D_ab = sum_c f_c Psi_a,c Psi_b,c
template <int ORDER>
__global__ void __launch_bounds__(128) k_density(Mesh m, const int32_t* dof_of_node, const double* Psi,
                                                 int N, const double* occ, double* rho) {
    constexpr int NL = El<ORDER>::NLOC, NQ = El<ORDER>::NQ, NP = El<ORDER>::NP;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    int d[NL];
    for (int a = 0; a < NL; ++a) d[a] = dof_of_node[m.elem[e * NL + a]];
    double D[NP];
    for (int p = 0; p < NP; ++p) D[p] = 0.0;
    for (int c = 0; c < N; ++c) {
        double f = occ[c];
        if (f == 0.0) continue;
        double u[NL];
        for (int a = 0; a < NL; ++a) u[a] = d[a] >= 0 ? Psi[(int64_t)d[a] * N + c] : 0.0;
        int p = 0;
        for (int a = 0; a < NL; ++a) {
            double fa = f * u[a];
            for (int b = a; b < NL; ++b, ++p) D[p] += fa * u[b];
        }
    }
    // off-diagonal pairs appear twice in the square
    {
        int p = 0;
        for (int a = 0; a < NL; ++a)
            for (int b = a; b < NL; ++b, ++p)
                if (b != a) D[p] *= 2.0;
    }
    for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int p = 0; p < NP; ++p) s += T_pp<ORDER>(q, p) * D[p];
        rho[e * NQ + q] = s;
    }
}

// ---------------------------------------------------------------- density from pattern pairs
// The same rho(q) as k_density, with the element density matrices assembled
// from one density matrix on the sparsity pattern of the fine space:
// D_p = sum_c f_c Psi_a,c Psi_b,c for every pattern entry p = (a, b), b >= a
// (both interior; Psi vanishes on the boundary), computed once although the
// pair (a, b) belongs to every element around it - about 115M pairs on the
// 32-nucleus mesh against 6M x 55 element pairs.  Then rho(q) of an element
// is sum_p (2 - delta_ab) phi_a(q) phi_b(q) D_slot(e, p), in k_density's order.

// slot[e][p]: the CSR position of the element's local pair p = (a <= b) as
// (min(d_a, d_b), max(d_a, d_b)), or -1 when a node is on the boundary; an
// interior pair missing from the pattern (never expected) sets *err
template <int ORDER>
__global__ void k_pair_slots(Mesh m, const int32_t* dof_of_node, const int32_t* rowptr, const int32_t* col,
                             int32_t* slot, int* err) {
    constexpr int NL = El<ORDER>::NLOC, NP = El<ORDER>::NP;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    int d[NL];
    for (int a = 0; a < NL; ++a) d[a] = dof_of_node[m.elem[e * NL + a]];
    int p = 0;
    for (int a = 0; a < NL; ++a)
        for (int b = a; b < NL; ++b, ++p) {
            int s = -1;
            if (d[a] >= 0 && d[b] >= 0) {
                const int lo = min(d[a], d[b]), hi = max(d[a], d[b]);
                int L = rowptr[lo], R = rowptr[lo + 1] - 1;
                while (L <= R) {
                    const int M = (L + R) >> 1, cm = col[M];
                    if (cm == hi) {
                        s = M;
                        break;
                    }
                    if (cm < hi)
                        L = M + 1;
                    else
                        R = M - 1;
                }
                if (s < 0) atomicExch(err, 1);
            }
            slot[e * NP + p] = s;
        }
}

// D[p] for the entries p = (a, b >= a) of row a: a warp per row, four groups of
// 8 lanes take the row's upper entries in turn; lane k of a group sums the
// orbitals c = k, k + 8, ... (fixed order), then the group adds its 8 lane sums
// by three xor shuffles (fixed order)
__global__ void __launch_bounds__(256) k_pattern_density(int64_t n, const int32_t* rowptr, const int32_t* col,
                                                     const double* Psi, int N, const double* occ, double* D) {
    const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, g = lane >> 3, k = lane & 7;
    if (a >= n) return;
    double u[16];   // f_c Psi_a,c for c = k + 8 j (N <= 128)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int c = k + 8 * j;
        u[j] = c < N ? occ[c] * Psi[a * N + c] : 0.0;
    }
    const int p0 = rowptr[a], p1 = rowptr[a + 1];
    // first upper entry (columns are sorted)
    int lo = p0, hi = p1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (col[mid] < a)
            lo = mid + 1;
        else
            hi = mid;
    }
    for (int pb = lo; pb < p1; pb += 4) {
        const int p = pb + g;
        double s = 0.0;
        if (p < p1) {
            const double* pb_row = Psi + (int64_t)col[p] * N;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = k + 8 * j;
                if (c < N) s = fma(u[j], pb_row[c], s);
            }
        }
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (k == 0 && p < p1) D[p] = s;
    }
}

template <int ORDER>
__global__ void __launch_bounds__(128) k_density_pairs(Mesh m, const int32_t* slot, const double* D, double* rho) {
    constexpr int NL = El<ORDER>::NLOC, NQ = El<ORDER>::NQ, NP = El<ORDER>::NP;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    double Dl[NP];
#pragma unroll
    for (int a = 0, p = 0; a < NL; ++a)
#pragma unroll
        for (int b = a; b < NL; ++b, ++p) {
            const int s = slot[e * NP + p];
            const double v = s >= 0 ? D[s] : 0.0;
            Dl[p] = b != a ? 2.0 * v : v;   // off-diagonal pairs appear twice in the square
        }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double r = 0.0;
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) r += T_pp<ORDER>(q, pp) * Dl[pp];
        rho[e * NQ + q] = r;
    }
}

template <int ORDER>
__global__ void k_local_load(Mesh m, const double* Wq, const double* f, double* Lv) {
    constexpr int NL = El<ORDER>::NLOC, NQ = El<ORDER>::NQ;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    double c[NQ];
    for (int q = 0; q < NQ; ++q) c[q] = Wq[e * NQ + q] * f[e * NQ + q];
    for (int a = 0; a < NL; ++a) {
        double s = 0.0;
        for (int q = 0; q < NQ; ++q) s += c[q] * T_phi<ORDER>(q, a);
        Lv[e * NL + a] = s;
    }
}

__global__ void k_gather(int64_t nslots, const int64_t* ptr, const int32_t* idx, const double* src,
                         double scale, double* out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    double acc = 0.0;
    for (int64_t k = ptr[s]; k < ptr[s + 1]; ++k) acc += src[idx[k]];
    out[s] = scale * acc;
}

// Deterministic block reduction of K values per thread into partial[block][K]
template <int K>
__device__ void block_reduce_store(double (&v)[K], double* partial) {
    __shared__ double sh[K][256];
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off)
            for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < K; ++k) partial[(int64_t)blockIdx.x * K + k] = sh[k][0];
}

template <int K>
__global__ void k_final_reduce(int nblocks, const double* partial, double* out) {
    // one block of 256 threads, fixed order
    __shared__ double sh[256];
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(int64_t)b * K + k];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int off = blockDim.x / 2; off > 0; off >>= 1) {
            if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

static const int kRedBlocks = 1216;  // 8 x 152 SMs

template <int ORDER>
__global__ void __launch_bounds__(256) k_moments(Mesh m, const double* Wq, const double* rho, double* partial) {
    constexpr int NQ = El<ORDER>::NQ;
    double acc[10];
    for (int k = 0; k < 10; ++k) acc[k] = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m.ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        double v[4][3];
        load_vertices(m, e, v);
        for (int q = 0; q < NQ; ++q) {
            double x[3];
            for (int d = 0; d < 3; ++d)
                x[d] = T_bary<ORDER>(q, 0) * v[0][d] + T_bary<ORDER>(q, 1) * v[1][d] +
                       T_bary<ORDER>(q, 2) * v[2][d] + T_bary<ORDER>(q, 3) * v[3][d];
            double wr = Wq[e * NQ + q] * rho[e * NQ + q];
            acc[0] += wr;
            acc[1] += wr * x[0];
            acc[2] += wr * x[1];
            acc[3] += wr * x[2];
            acc[4] += wr * x[0] * x[0];
            acc[5] += wr * x[0] * x[1];
            acc[6] += wr * x[0] * x[2];
            acc[7] += wr * x[1] * x[1];
            acc[8] += wr * x[1] * x[2];
            acc[9] += wr * x[2] * x[2];
        }
    }
    block_reduce_store<10>(acc, partial);
}

__global__ void k_boundary_values(int64_t nb, const int32_t* bnd_node, const double* xyz,
                                  const double* mom, int multipole, double* wB, double* V) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double Q = mom[0];
    double w = 0.0;
    int u = bnd_node[i];
    if (Q != 0.0) {
        double c[3] = {mom[1] / Q, mom[2] / Q, mom[3] / Q};
        double d[3] = {xyz[3 * u] - c[0], xyz[3 * u + 1] - c[1], xyz[3 * u + 2] - c[2]};
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double r = sqrt(r2);
        w = Q / r;
        if (multipole >= 2) {
            // q_ij = int rho (x_i - c_i)(x_j - c_j) = M2_ij - Q c_i c_j
            const int ij[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
            double s = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double qab = mom[ij[a][b]] - Q * c[a] * c[b];
                    s += qab * (3.0 * d[a] * d[b] - (a == b ? r2 : 0.0));
                }
            w += 0.5 * s / (r2 * r2 * r);
        }
    }
    wB[i] = w;
    if (V) V[u] = w;
}

__global__ void k_dof_to_nodal(int64_t n, const int32_t* dof_node, const double* x, double* V) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V[dof_node[i]] = x[i];
}

__global__ void k_nodal_to_dof(int64_t n, const int32_t* dof_node, const double* V, double* x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = V[dof_node[i]];
}

// out[e][q] = sum_c A_c(x_q) U_c(x_q) (both from dof values [n][N]); used by
// the adjoint contraction of the linear problems
template <int ORDER>
__global__ void __launch_bounds__(128) k_pair_density(Mesh m, const int32_t* dof_of_node, const double* A,
                                                      const double* U, int N, double* out) {
    constexpr int NL = El<ORDER>::NLOC, NQ = El<ORDER>::NQ;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    int d[NL];
    for (int a = 0; a < NL; ++a) d[a] = dof_of_node[m.elem[e * NL + a]];
    double prod[NQ];
    for (int q = 0; q < NQ; ++q) prod[q] = 0.0;
    for (int c = 0; c < N; ++c) {
        double av[NL], uv[NL];
        for (int a = 0; a < NL; ++a) {
            av[a] = d[a] >= 0 ? A[(int64_t)d[a] * N + c] : 0.0;
            uv[a] = d[a] >= 0 ? U[(int64_t)d[a] * N + c] : 0.0;
        }
        for (int q = 0; q < NQ; ++q) {
            double aq = 0.0, uq = 0.0;
            for (int a = 0; a < NL; ++a) {
                aq += T_phi<ORDER>(q, a) * av[a];
                uq += T_phi<ORDER>(q, a) * uv[a];
            }
            prod[q] += aq * uq;
        }
    }
    for (int q = 0; q < NQ; ++q) out[e * NQ + q] = prod[q];
}

// partial[block][4*j + c] = sum over the block's quadrature points of
// W_eq w_eq dV_ext/dp_(k0+j, c)(x_q), c = x, y, z, Z, for nuclei k0..k0+7
template <int ORDER>
__global__ void __launch_bounds__(256) k_vext_grad(Mesh m, Nuclei nuc, int k0, const double* Wq, const double* w,
                                                  double* partial) {
    constexpr int NQ = El<ORDER>::NQ;
    const int nk = min(8, nuc.count - k0);
    double acc[32];
    for (int j = 0; j < 32; ++j) acc[j] = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m.ne; e += (int64_t)gridDim.x * blockDim.x) {
        double v[4][3];
        load_vertices(m, e, v);
        for (int q = 0; q < NQ; ++q) {
            const double ww = Wq[e * NQ + q] * w[e * NQ + q];
            if (ww == 0.0) continue;
            double x[3];
            for (int dd = 0; dd < 3; ++dd)
                x[dd] = T_bary<ORDER>(q, 0) * v[0][dd] + T_bary<ORDER>(q, 1) * v[1][dd] +
                        T_bary<ORDER>(q, 2) * v[2][dd] + T_bary<ORDER>(q, 3) * v[3][dd];
            for (int j = 0; j < nk; ++j) {
                const int k = k0 + j;
                const double dx = x[0] - nuc.R[3 * k], dy = x[1] - nuc.R[3 * k + 1], dz = x[2] - nuc.R[3 * k + 2];
                double r2 = dx * dx + dy * dy + dz * dz;
                if (nuc.potential == NAS_POT_SMOOTHED) r2 += nuc.smooth_a * nuc.smooth_a;
                const double inv = 1.0 / sqrt(r2);
                const double zi3 = nuc.Z[k] * inv * inv * inv;
                // V = -Z r2^(-1/2): dV/dR = -Z (x - R) r2^(-3/2), dV/dZ = -r2^(-1/2)
                acc[4 * j + 0] -= ww * zi3 * dx;
                acc[4 * j + 1] -= ww * zi3 * dy;
                acc[4 * j + 2] -= ww * zi3 * dz;
                acc[4 * j + 3] -= ww * inv;
            }
        }
    }
    __shared__ double sh[256];
    for (int j = 0; j < 4 * nk; ++j) {
        sh[threadIdx.x] = acc[j];
        __syncthreads();
        for (int off = blockDim.x / 2; off > 0; off >>= 1) {
            if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * 32 + j] = sh[0];
        __syncthreads();
    }
}

__global__ void k_reduce_grad(int nblocks, int nk4, const double* partial, double* out) {
    int j = threadIdx.x;
    if (j >= nk4) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * 32 + j];
    out[j] = s;
}

// ------------------------------------------------------------------ launchers
#define NAS_DISPATCH(m, KERNEL, ...)                                                 \
    do {                                                                             \
        if ((m).nloc == 4)                                                           \
            KERNEL<1><<<grid_for((m).ne, 128), 128, 0, s>>>(__VA_ARGS__);            \
        else                                                                         \
            KERNEL<2><<<grid_for((m).ne, 128), 128, 0, s>>>(__VA_ARGS__);            \
        NAS_CHECK_LAUNCH();                                                          \
    } while (0)

void launch_geometry(const Mesh& m, double* Wq, int* err, cudaStream_t s) {
    NAS_DISPATCH(m, k_geometry, m, Wq, err);
}
void launch_local_stiffness(const Mesh& m, double* L, cudaStream_t s) {
    NAS_DISPATCH(m, k_local_stiffness, m, L);
}
void launch_local_mass(const Mesh& m, const double* Wq, const double* coef, double* L, cudaStream_t s) {
    NAS_DISPATCH(m, k_local_mass, m, Wq, coef, L);
}
void launch_vext(const Mesh& m, const Nuclei& nuc, double* vq, cudaStream_t s) {
    NAS_DISPATCH(m, k_vext, m, nuc, vq);
}
void launch_nodal_to_quad(const Mesh& m, const double* nodal, double* out, cudaStream_t s) {
    NAS_DISPATCH(m, k_nodal_to_quad, m, nodal, out);
}
void launch_nl_coef(const Mesh& m, const double* VH, const double* rho, int xc, double* coef,
                    double* eps, double* vxc, cudaStream_t s) {
    NAS_DISPATCH(m, k_nl_coef, m, VH, rho, xc, coef, eps, vxc);
}
void launch_lda(int64_t cnt, const double* rho, double* eps, double* vxc, cudaStream_t s) {
    if (cnt <= 0) return;
    k_lda<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, rho, eps, vxc);
    NAS_CHECK_LAUNCH();
}
void launch_density(const Mesh& m, const int32_t* dof_of_node, const double* Psi, int N,
                    const double* occ, double* rho, cudaStream_t s) {
    NAS_DISPATCH(m, k_density, m, dof_of_node, Psi, N, occ, rho);
}
int64_t density_pair_count(const Mesh& m) { return m.ne * (m.nloc == 4 ? 10 : 55); }
bool launch_pair_slots(const Mesh& m, const int32_t* dof_of_node, const int32_t* rowptr, const int32_t* col,
                       int32_t* slot, int* err, cudaStream_t s) {
    NAS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    NAS_DISPATCH(m, k_pair_slots, m, dof_of_node, rowptr, col, slot, err);
    int h = 0;
    NAS_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NAS_CUDA(cudaStreamSynchronize(s));
    return h == 0;
}
void launch_density_pairs(const Mesh& m, int64_t n, const int32_t* rowptr, const int32_t* col, const double* Psi,
                          int N, const double* occ, const int32_t* slot, double* D, double* rho, cudaStream_t s) {
    if (N < 1 || N > 128) fail(NAS_E_INVALID_ARG, "pair density: N out of range");
    if (n > 0) {
        k_pattern_density<<<grid_for(n * 32, 256), 256, 0, s>>>(n, rowptr, col, Psi, N, occ, D);
        NAS_CHECK_LAUNCH();
    }
    NAS_DISPATCH(m, k_density_pairs, m, slot, D, rho);
}
void launch_local_load(const Mesh& m, const double* Wq, const double* f, double* Lv, cudaStream_t s) {
    NAS_DISPATCH(m, k_local_load, m, Wq, f, Lv);
}
void launch_gather(int64_t nslots, const int64_t* ptr, const int32_t* idx, const double* src,
                   double scale, double* out, cudaStream_t s) {
    if (nslots <= 0) return;
    k_gather<<<grid_for(nslots, 256), 256, 0, s>>>(nslots, ptr, idx, src, scale, out);
    NAS_CHECK_LAUNCH();
}
void launch_moments(const Mesh& m, const double* Wq, const double* rho, double* partial,
                    double* out, cudaStream_t s) {
    int nb = (int)std::min<int64_t>(kRedBlocks, (m.ne + 255) / 256);
    if (m.nloc == 4)
        k_moments<1><<<nb, 256, 0, s>>>(m, Wq, rho, partial);
    else
        k_moments<2><<<nb, 256, 0, s>>>(m, Wq, rho, partial);
    NAS_CHECK_LAUNCH();
    k_final_reduce<10><<<1, 256, 0, s>>>(nb, partial, out);
    NAS_CHECK_LAUNCH();
}
void launch_boundary_values(int64_t nb, const int32_t* bnd_node, const double* node_xyz,
                            const double* moments, int multipole, double* wB, double* V_nodal,
                            cudaStream_t s) {
    if (nb <= 0) return;
    k_boundary_values<<<grid_for(nb, 256), 256, 0, s>>>(nb, bnd_node, node_xyz, moments, multipole,
                                                       wB, V_nodal);
    NAS_CHECK_LAUNCH();
}
void launch_pair_density(const Mesh& m, const int32_t* dof_of_node, const double* A, const double* U, int N,
                         double* out, cudaStream_t s) {
    NAS_DISPATCH(m, k_pair_density, m, dof_of_node, A, U, N, out);
}

void launch_vext_grad(const Mesh& m, const Nuclei& nuc, const double* Wq, const double* w, double* partial,
                      double* out, cudaStream_t s) {
    const int nb = (int)std::min<int64_t>(kRedBlocks, (m.ne + 255) / 256);
    for (int k0 = 0; k0 < nuc.count; k0 += 8) {
        if (m.nloc == 4)
            k_vext_grad<1><<<nb, 256, 0, s>>>(m, nuc, k0, Wq, w, partial);
        else
            k_vext_grad<2><<<nb, 256, 0, s>>>(m, nuc, k0, Wq, w, partial);
        NAS_CHECK_LAUNCH();
        const int nk4 = 4 * std::min(8, nuc.count - k0);
        k_reduce_grad<<<1, 32, 0, s>>>(nb, nk4, partial, out + 4 * k0);
        NAS_CHECK_LAUNCH();
    }
}

void launch_nodal_to_dof(int64_t n, const int32_t* dof_node, const double* V, double* x, cudaStream_t s) {
    if (n <= 0) return;
    k_nodal_to_dof<<<grid_for(n, 256), 256, 0, s>>>(n, dof_node, V, x);
    NAS_CHECK_LAUNCH();
}
void launch_dof_to_nodal(int64_t n, const int32_t* dof_node, const double* x, double* V, cudaStream_t s) {
    if (n <= 0) return;
    k_dof_to_nodal<<<grid_for(n, 256), 256, 0, s>>>(n, dof_node, x, V);
    NAS_CHECK_LAUNCH();
}

}  // namespace nas

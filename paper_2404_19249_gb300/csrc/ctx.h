// Solver context: inputs, host topology, device data and state of the
// augmented subspace method.  Internal; the C ABI only sees nas_ctx*.
#pragma once

#include <array>
#include <deque>
#include <string>
#include <vector>

#include "common.h"
#include "kernels.h"
#include "eig_dev.h"
#include "space.h"
#include "transfer_setup.h"

// identity of a captured Poisson PCG graph (its baked-in pointers and parameters)
struct Pcg1Key {
    static const int kPtrs = 12;
    const void* ptr[kPtrs] = {};
    double tol = 0.0;
    int lanes = 0;
    int64_t n = 0;
    bool operator==(const Pcg1Key& o) const {
        for (int i = 0; i < kPtrs; ++i)
            if (ptr[i] != o.ptr[i]) return false;
        return tol == o.tol && lanes == o.lanes && n == o.n;
    }
};

struct nas_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    nas_options opt{};

    // ---- inputs
    bool have_fine = false, have_coarse = false, have_system = false;
    int fine_order = 1;
    std::vector<double> fxyz, cxyz;
    std::vector<int32_t> ftet, ctet;
    int64_t fnv = 0, fne = 0, cnv = 0, cne = 0;
    int n_nuc = 0;
    std::vector<double> R, Z;
    int potential = NAS_POT_COULOMB;
    double smooth_a = 0.0;
    int N = 0;
    std::vector<double> occ;            // occupations given to nas_set_system

    // ---- derived
    bool setup_done = false, initialized = false;
    nas::HostSpace F, C;
    nas::BucketGrid BG;
    nas::GalerkinMaps GM;
    double mu = 0.0, Enn = 0.0;
    int64_t nq = 0;      // quadrature points per element
    int64_t nqt = 0;     // total quadrature points ne*nq
    int64_t nH = 0;      // coarse dofs
    std::vector<int32_t> I_elem, I_col;
    std::vector<double> I_val;
    std::vector<double> BH, AHL;          // coarse Galerkin values [hnnz]
    std::vector<double> BH_chol;          // dense Cholesky factor of B_H [nH][nH]
    nas::DBuf<double> d_BHinv;            // dense B_H^-1 [nH][nH] on the device

    // ---- device: fine mesh
    nas::DBuf<double> d_vxyz, d_node_xyz, d_Wq;
    nas::DBuf<int32_t> d_elem, d_dof_of_node, d_dof_node, d_bnd_node;
    nas::DBuf<int32_t> d_rowptr, d_col, d_contrib, d_browptr, d_bcol, d_bcontrib, d_lcontrib;
    nas::DBuf<int64_t> d_cptr, d_bcptr, d_lptr;
    nas::DBuf<double> d_K, d_M, d_Mvext, d_AL, d_ANL, d_H, d_KIB, d_Hdinv, d_Kdinv;
    nas::DBuf<double> d_L, d_Lv;                       // element matrices / vectors
    nas::DBuf<double> d_coef, d_eps, d_vxc, d_tmpq;    // [nqt]
    nas::DBuf<double> d_rho_in, d_rho_out, d_rho_prev; // [nqt]
    std::vector<nas::DBuf<double>> d_hist_rin, d_hist_F;
    nas::DBuf<double> d_VH, d_wB;                      // [nnode], [nb]
    nas::DBuf<double> d_R, d_Zn;                       // nuclei
    // ---- device: transfer
    nas::DBuf<double> d_cxyz;
    nas::DBuf<int32_t> d_ctet, d_cdof, d_btet, d_Ielem, d_Icol;
    nas::DBuf<int64_t> d_bptr;
    nas::DBuf<double> d_Ival;
    nas::DBuf<int32_t> d_tptr, d_trow, d_wptr, d_wcol, d_wrow, d_w1con, d_hptr, d_hcol, d_h2con;
    nas::DBuf<int64_t> d_w1ptr, d_h2ptr;
    nas::DBuf<double> d_tval, d_W, d_AH;
    nas::DBuf<int32_t> d_tpc_seg, d_h2pc_seg;          // balanced pieces of I^T rows / stage-2 lists
    nas::DBuf<int64_t> d_tpc_start, d_h2pc_start;
    nas::DBuf<double> d_piece_part;                    // piece sums (max of npieces_t * N, npieces_h2)
    nas::DBuf<double> d_cpart;                         // piece sums of I^T r in the Poisson PCG
    nas::DBuf<float> d_cpart32;
    // ---- device: orbitals and solver work
    nas::DBuf<double> d_Psi, d_Uhat, d_occ, d_U;
    nas::DBuf<double> d_X1, d_X2;                      // [n][N] temporaries
    nas::DBuf<double> d_cg_R, d_cg_Z, d_cg_P, d_cg_Q, d_cg_B;
    nas::DBuf<double> d_cg_scal;                       // 8*N scalars
    nas::DBuf<int> d_cg_active, d_flag;
    nas::DBuf<double> d_pv, d_pb;                      // Poisson vectors [n]
    nas::DBuf<double> d_blk_b, d_blk_c;                // [nH][N]
    nas::DBuf<double> d_blk_beta, d_blk_gamma;         // [N][N]
    nas::DBuf<double> d_partial, d_red;                // reduction scratch
    nas::DBuf<double> d_moments;
    nas::DBuf<double> d_pcg1_part, d_pcg1_scal;        // fused Poisson PCG scratch
    nas::DBuf<double> d_khinv, d_khvec;                // two-level preconditioner: K_H^-1, [c ; y]
    nas::DBuf<int64_t> d_sell_ptr;                     // sliced-ELL copy of K (Poisson SpMV)
    nas::DBuf<int32_t> d_sell_col;
    nas::DBuf<double> d_sell_val;
    int64_t sell_slices = 0, sell_entries = 0;
    nas::DBuf<int> d_pcg1_flags;
    nas::DBuf<unsigned> d_pcg1_bar;                   // grid barrier of the persistent PCG
    cudaStream_t cap_stream = nullptr;                 // private stream for graph capture
    cudaGraphExec_t pcg1_exec = nullptr;
    Pcg1Key pcg1_key;
    // timing mode: events around the SpMV of the first two (direct) iterations
    std::vector<cudaEvent_t> pcg1_ev;                  // [4]
    double pcg1_fused_ms = 0.0;                        // event time of the persistent PCG launches
    long long pcg1_fused_iters = 0;
    bool concurrent = false;                           // inside nas_batch_run
    double pcg1_spmv_ms = 0.0;                          // this step: SpMV kernel time
    long long pcg1_spmv_launches = 0;
    // mixed precision: FP32 copies and work arrays of the Poisson solve
    nas::DBuf<float> d_H32, d_Hdinv32, d_bvp32;         // mixed precision: FP32 H~, D^-1 and block PCG vectors
    nas::DBuf<float> d_K32, d_Kdinv32, d_ival32, d_tval32, d_khinv32, d_khvec32, d_f32work, d_f32part;
    cudaGraphExec_t pcg1f_exec = nullptr;
    Pcg1Key pcg1f_key;
    long long pcg1_iters = 0;
    // two-level preconditioner of the N shifted problems: C^-1, C = I^T H~ I
    nas::DBuf<double> d_bvpC, d_bvp_tc, d_bvp_yc;     // [nH][nH], [nH][N], [nH][N]
    nas::DBuf<float> d_bvpC32, d_bvp_part32;
    bool bvp_coarse_ready = false, bvp_coarse_failed = false;

    // ---- state (host)
    int64_t state_id = 0;               // bumped by every call that changes the solver state
    std::vector<double> lam;            // [N]
    std::vector<double> occ_now;        // occupations of the current orbitals [N]
    double e_ts = 0.0;                  // -kT S of occ_now (smearing)
    double inner_tol_now = 0.0;         // stop tolerance of the last inner SCF
    double bvp_tol_now = 0.0;           // tolerance of the last step's linear solves
    bool have_VH = false;
    bool anl_valid = false;             // d_ANL/d_eps/d_vxc match d_rho_in and d_VH
    // density from pattern pairs: element pair -> CSR slot map (built once per
    // mesh), the pattern's pair density, an error flag
    nas::DBuf<int32_t> d_pair_slot;
    nas::DBuf<double> d_pairD;
    nas::DBuf<int> d_pair_err;
    bool pair_ready = false;
    int step_count = 0;
    int last_cg = 0, last_poisson = 0, last_inner = 0, last_inner_conv = 0;
    double last_drho = 0.0, last_inner_res = 0.0;
    std::vector<double> inner_hist;     // density residual of every inner iteration of the last inner SCF
    std::array<double, 6> energy{};
    // host copies of the last small problem
    int last_m = 0;
    std::vector<double> FA, FB;
    // blocks fixed during an inner SCF
    std::vector<double> hb_cH, hb_gamma, hb_bHL, hb_betaL;
    int Na = 0;                         // augmentation columns in use (0 or N)
    std::vector<double> U_warm;         // warm start of the small eigensolver [m][N]
    // device form of the small pencil (arrow structure) for the device LOBPCG
    nas::DBuf<double> d_AHLv, d_BHv;                   // coarse CSR values of A_H^L, B_H
    nas::DBuf<int32_t> d_hdiag;                        // CSR slot of each coarse diagonal entry
    nas::DBuf<double> d_cH, d_gam, d_bL, d_betaL;      // fixed borders/corners of one step
    nas::DBuf<double> d_FAs, d_FAb, d_FAc;             // F_A of the current inner iteration
    nas::DBuf<double> d_Uwarm;                         // warm start [m][N] on the device
    int64_t uwarm_dev_m = 0;                           // m of d_Uwarm's content (0: none)
    bool lob_reuse_ok = false;                         // F_B unchanged since the last device solve
    nas::DevLobpcg lob;
    double eig_tol_hint = 1.0;          // last inner-SCF residual (LOBPCG tolerance)
    double poisson_tol_now = 0.0;       // > 0: tolerance of the next Poisson solve
    int last_lobpcg_iters = 0;
    int last_rr_calls = 0, last_rr_fallbacks = 0;   // device LOBPCG Rayleigh-Ritz steps of the step

    // ---- timing
    double phase_ms[NAS_MAX_PHASES] = {0};
    long long phase_calls[NAS_MAX_PHASES] = {0};
    double spmm_bytes = 0, spmm_flops = 0, spmv_bytes = 0, spmv_flops = 0;
    double spmm32_bytes = 0, spmm32_flops = 0;
    struct EvPair {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<EvPair> ev_pending;
    std::vector<cudaEvent_t> ev_pool;
    long long launches_at_step_start = 0;
};

namespace nas {

// driver entry points (driver.cpp)
void ctx_setup(nas_ctx* c);
void ctx_init(nas_ctx* c, const double* psi0);
int ctx_step(nas_ctx* c, nas_report* rep);
void ctx_fill_report(nas_ctx* c, nas_report* rep);
void ctx_set_state(nas_ctx* c, const double* lam, const double* psi, const double* rho, int on_device);
void ctx_apply(nas_ctx* c, int op, const void* in, int64_t cnt, void* out, int on_device);
void ctx_get(nas_ctx* c, int what, void* dst, size_t bytes, int on_device);
void ctx_update_nuclei(nas_ctx* c);

}  // namespace nas

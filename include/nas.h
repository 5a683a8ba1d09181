/*
 * nas.h - C ABI of the GPU nonnested augmented subspace method for the
 * Kohn-Sham equation (Hu, Xie, Xu, Zhao, arXiv 2404.19249).
 *
 * The library computes, on one GPU, the fine-mesh work of Algorithm 3 (the
 * augmented subspace method, Sec. 3.3): assembly of the finite element
 * Hamiltonian with V_ext, V_Har and LDA V_xc integrated by quadrature, the N
 * shifted linear boundary value problems solved by block preconditioned CG,
 * the nonnested transfer matrix I_H^h built by point location (Algorithm 1),
 * the blocks of the small augmented eigenproblem (F_A, F_B of Sec. 3.3), the density
 * and the Hartree Poisson solve (Sec. 3.1).  The small dense generalized
 * eigenproblem F_A U = lambda F_B U is solved on the host.
 *
 * Conventions for every function below
 *  - Return value: NAS_OK (0) on success, otherwise a negative NAS_E_* code;
 *    nas_last_error() then returns a message for that context.  No function
 *    calls exit() or throws across the ABI.
 *  - Pointers are HOST pointers unless the argument or flag says "device".
 *    The caller owns every buffer it passes; the library copies what it needs
 *    into device memory that it owns and frees in nas_destroy().
 *  - Arrays are C-contiguous (row-major).  "FP64" means IEEE double.
 *  - A context is used by one host thread at a time.  All device work of a
 *    context is ordered on the CUDA stream given to nas_create().
 */
#ifndef NAS_H
#define NAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define NAS_OK                  0
#define NAS_E_INVALID_ARG      -1  /* bad size, NULL pointer, bad enum */
#define NAS_E_MESH             -2  /* inverted/degenerate tetrahedron, bad ids */
#define NAS_E_POINT_NOT_FOUND  -3  /* a fine node lies in no coarse tetrahedron */
#define NAS_E_BREAKDOWN        -4  /* CG p^T A p <= 0 or non-finite values */
#define NAS_E_NOT_CONVERGED    -5  /* an iteration cap was reached */
#define NAS_E_CUDA             -6  /* a CUDA runtime call failed */
#define NAS_E_OOM              -7  /* device or host allocation failed */
#define NAS_E_STATE            -8  /* call made out of order (e.g. step before init) */
#define NAS_E_EIGEN            -9  /* host small eigensolver failed (F_B not SPD ...) */

enum nas_mesh_kind { NAS_FINE = 0, NAS_COARSE = 1 };

/* External potential V_ext (Sec. 2): Coulomb -sum Z_k/|x-R_k|; smoothed
 * Coulomb -sum Z_k/sqrt(|x-R_k|^2 + a^2); harmonic 0.5 omega^2 |x|^2 (a test
 * potential with closed-form levels n + 3/2). */
enum nas_potential { NAS_POT_COULOMB = 0, NAS_POT_SMOOTHED = 1, NAS_POT_HARMONIC = 2 };

/* ------------------------------------------------------------------ options */
typedef struct nas_options {
    double mu;             /* shift of H~ = H + mu (Sec. 3.3); < 0 selects 8 M sum_k Z_k^2
                              (the experiments' choice, Sec. 4)                     */
    double tol_bvp;        /* relative residual of each of the N linear problems     */
    double tol_poisson;    /* relative residual of the Hartree Poisson solve         */
    double tol_scf;        /* ||rho^(l) - rho^(l-1)||_0 stop test of Algorithm 3     */
    double tol_inner;      /* ||rho_out - rho_in||_0 stop test of the inner SCF      */
    int    max_cg;         /* iteration cap of the block PCG                         */
    int    max_poisson;    /* iteration cap of the Poisson PCG                       */
    int    max_inner;      /* inner SCF iterations per step                          */
    int    max_outer;      /* steps of nas_solve                                     */
    int    anderson_depth; /* Anderson history depth, 1..16 (Sec. 4: 5)              */
    double anderson_beta;  /* Anderson damping (Sec. 4: 0.7)                         */
    int    hartree;        /* 1: include V_Har; 0: linear problem                    */
    int    xc;             /* 1: include LDA V_xc                                    */
    int    multipole;      /* Hartree boundary values: 0 monopole, 2 + quadrupole    */
    double omega;          /* harmonic test potential frequency                      */
    int    check_every;    /* CG iterations between host convergence checks (>=1)    */
    int    timing;         /* 1: record per-kernel CUDA-event times (nas_report)     */
    int    eig_dense_max;  /* small problems up to this size use the dense host
                              eigensolver, larger ones warm-started LOBPCG           */
    double eig_tol;        /* LOBPCG relative residual; <= 0: adaptive, eig_adapt x
                              the previous inner-SCF residual clamped to
                              [1e-11, 1e-4]                                        */
    int    spmv_lanes;     /* lanes per row of the Poisson SpMV (1, 2, 4, 8, 16, 32);
                              0 = chosen from the mean row length                    */
    int    poisson_two_level; /* 1: Poisson PCG preconditioner D^-1 + I K_H^-1 I^T with
                              the method's coarse space and transfer (K_H = I^T K I);
                              0: Jacobi only                                        */
    int    precision;      /* 0: FP64 throughout; 1: mixed - the Poisson PCG and the
                              block PCG of the N shifted problems run in FP32
                              (FP32 storage and products) inside FP64 iterative
                              refinement; residual tests, assembly, blocks, the
                              small eigensolve and energies stay FP64.  Poisson
                              solves asked for a relative tolerance below 1e-9
                              run in FP64 (FP32 inner solves leave smooth-mode
                              errors such a residual test does not resolve)    */
    int    eig_device;     /* small problems above eig_dense_max: 1 = LOBPCG with its
                              block vectors, products and Gram matrices on the
                              device (host Rayleigh-Ritz of the 3k x 3k Grams);
                              0 = the host LOBPCG                                  */
    int    eig_precond;    /* LOBPCG preconditioner: 1 = the inverse coarse stiffness
                              (I^T K I)^-1 on the coarse rows (FP32, dense; coarse
                              spaces up to 6000 unknowns; SIMT FP32 product) and the
                              diagonal on the others; 2 = the same with the dense
                              product on the tensor cores (tcgen05, split TF32,
                              FP32-level accuracy); 0 = diag(F_A - sigma F_B)^-1
                              everywhere                                          */
    double eig_adapt;      /* factor of the adaptive LOBPCG tolerance (eig_tol <= 0):
                              eig_adapt x the previous inner-SCF residual, clamped
                              to [1e-11, 1e-4]                                     */
    int    poisson_sell;   /* 1: the FP64 Poisson SpMV reads a sliced-ELL copy of K
                              (32 rows per slice, one thread per row, coalesced
                              value/column loads); 0: the CSR kernel with
                              spmv_lanes lanes per row (the FP32 inner solve of
                              precision = 1 always uses the CSR kernel)            */
    int    poisson_adaptive; /* 1: inside the inner SCF the Poisson tolerance follows
                              the previous density residual res:
                              max(tol_poisson, min(1e-6, 1e-3 res)); 0: always
                              tol_poisson.  The fixed point is unchanged.          */
    int    poisson_fused;  /* 1: the FP64 two-level Poisson PCG with the sliced-ELL
                              matrix runs as one persistent cooperative kernel per
                              16 iterations (grid-wide barriers between the
                              phases, same arithmetic and bit-identical iterates
                              to the per-phase kernels; measured slower on GB300:
                              0.32 against 0.23 ms per iteration); 0: per-phase
                              kernels replayed from a CUDA graph.  Not used inside
                              nas_batch_run; callers that run several contexts'
                              solves at once on one device from their own threads
                              keep 0.                                              */
    double smearing;       /* > 0: Fermi-Dirac occupations at temperature kT = smearing
                              (Ha), f_i = 2 / (1 + exp((lambda_i - eF)/kT)) with eF
                              such that sum f_i = sum of the occupations given to
                              nas_set_system (needs n_orb > n_el / 2), recomputed
                              after every small eigensolve; the energy is then the
                              free energy E - kT S (S = -2 sum g ln g + (1-g)
                              ln(1-g), g = f/2).  0: the given occupations      */
    double inner_adapt;    /* > 0: inexact inner SCF - each step's inner SCF stops at
                              max(tol_inner, inner_adapt x the previous step's
                              ||rho^(l) - rho^(l-1)||_0); the outer fixed point is
                              unchanged (near it the inner SCF again runs to
                              tol_inner).  0: tol_inner in every step           */
    int    bvp_two_level;  /* 1: the block PCG of the N shifted problems in nas_step
                              uses D^-1 + I C^-1 I^T with C = I^T H~ I, the coarse
                              Galerkin matrix of the first step's H~ after
                              nas_init (dense inverse, formed once and kept: a
                              fixed SPD preconditioner); 0: Jacobi only.  The
                              nas_apply BVP ops always use Jacobi.  Measured on
                              the 32-nucleus workload with mu = 36: 168 against
                              152 Jacobi iterations (the shifted operator's bad
                              modes are not the coarse ones), so off by default */
    double bvp_adapt;      /* > 0: inexact linear solves - each step's N shifted
                              problems are solved to max(tol_bvp, min(1e-4,
                              bvp_adapt x the previous step's ||rho^(l) -
                              rho^(l-1)||_0)); the outer fixed point is unchanged
                              (near it the solves again reach tol_bvp).
                              0: tol_bvp in every step                          */
    double anderson_restart; /* > 0: in an inner SCF a density residual above
                              anderson_restart x the smallest one of that inner
                              SCF so far clears the Anderson history (the next
                              mix is the linear one); 0: never                 */
    int    poisson_f32;    /* precision = 1 only.  1: Poisson solves whose tolerance
                              is >= 1e-9 run as FP32 PCG inside FP64 iterative
                              refinement, tighter ones in FP64 to tol_poisson;
                              0: every Poisson solve in FP64 (the block PCG of
                              the shifted problems stays mixed).  Measured on the
                              32-nucleus workload with poisson_adaptive = 1: the
                              FP32 solves to the adaptive tolerance leave smooth
                              V_H errors that a residual test relative to ||b||
                              does not see, and an exact inner SCF then stalls
                              near a density residual of 1e-3                   */
    int    dense_tc;       /* 1: the FP64 dense contractions - the reconstruction
                              Psi = I u_H + U^ alpha and the Gram matrices
                              gamma, beta - run on the tensor cores from
                              error-free integer slices (FP64-level accuracy;
                              see nas_reconstruct_f64) when N <= 64; 0: FP64
                              SIMT kernels                                     */
    int    density_pairs;  /* 1: rho = sum f psi^2 at the quadrature points from the
                              density matrix on the fine sparsity pattern's
                              pairs (each pair once, then each element's pairs;
                              needs N <= 128, about nnz + 55 n_el extra words of
                              device memory); 0: element by element.  Measured
                              on the 32-nucleus workload: 53.4 ms against 51.1
                              ms - 2.3x fewer FP64 operations, but each pattern
                              pair gathers a whole orbital row (59 GB through
                              L2 against 31 GB), so 0 is the default          */
} nas_options;

/* Fill *opt with the defaults: mu = -1 (paper's 8 M sum Z^2), tol_bvp = 1e-12,
 * tol_poisson = 1e-12, tol_scf = tol_inner = 1e-8, max_cg = 2000,
 * max_poisson = 20000, max_inner = 50, max_outer = 100, depth 5, beta 0.7,
 * hartree = xc = 1, multipole = 0, omega = 1, check_every = 1, timing = 0,
 * eig_dense_max = 1200, eig_tol = -1 (adaptive), spmv_lanes = 0 (auto),
 * poisson_two_level = 1, precision = 0, eig_device = 1, eig_precond = 1,
 * eig_adapt = 1e-3, poisson_sell = 1, poisson_adaptive = 0, poisson_fused = 0,
 * smearing = 0, inner_adapt = 0, bvp_two_level = 0, bvp_adapt = 0,
 * anderson_restart = 0, poisson_f32 = 0, dense_tc = 1,
 * density_pairs = 0. */
void nas_default_options(nas_options* opt);

/* ------------------------------------------------------------------ report */
#define NAS_MAX_PHASES 16
enum nas_phase {
    NAS_PH_ASSEMBLY = 0,   /* V_eff at quadrature points + CSR assembly (Sec. 3.3)  */
    NAS_PH_BVP,            /* block PCG for the N linear problems                   */
    NAS_PH_POISSON,        /* Hartree: right-hand side, boundary values, PCG        */
    NAS_PH_BLOCKS,         /* F_A / F_B blocks (Sec. 3.3) incl. I^T A I              */
    NAS_PH_DENSITY,        /* Psi = I u_H + U^ alpha and rho at quadrature points   */
    NAS_PH_MIXING,         /* Anderson inner products and combination               */
    NAS_PH_HOST_EIG,       /* small eigensolve, wall time (host dense / host LOBPCG,
                              or device LOBPCG incl. its host Rayleigh-Ritz)       */
    NAS_PH_TRANSFER,       /* point location + I_H^h                                */
    NAS_PH_SPMM,           /* SpMM launches with N > 1 columns (subset of the above) */
    NAS_PH_SPMV,           /* SpMV launches (N = 1, Poisson and Dirichlet lift)      */
    NAS_PH_EIG_RR,         /* host Rayleigh-Ritz inside the device LOBPCG (subset of
                              NAS_PH_HOST_EIG)                                      */
    NAS_PH_EIG_WAIT,       /* host time blocked in stream synchronisations inside the
                              device LOBPCG (subset of NAS_PH_HOST_EIG)            */
    NAS_PH_SPMV32,         /* timing = 1: the FP32 SpMV of the mixed-precision Poisson
                              PCG, first two iterations of every inner FP32 solve
                              (direct launches with events around the SpMV)        */
    NAS_PH_SPMM32,         /* FP32 SpMM launches of the mixed-precision block PCG     */
    NAS_PH_RECON,          /* the reconstruction Psi = I u_H + U^ alpha (subset of
                              NAS_PH_DENSITY)                                      */
    NAS_PH_DENSK,          /* the density kernel rho = sum f psi^2 (subset of
                              NAS_PH_DENSITY)                                      */
    NAS_PH_COUNT
};

typedef struct nas_report {
    int    n_orb;             /* N                                                  */
    int    step;              /* steps done since nas_init                          */
    int    n_inner;           /* inner SCF iterations of the last step              */
    int    inner_converged;   /* 1 if the last inner SCF met tol_inner              */
    int    cg_iters;          /* block PCG iterations of the last step              */
    int    poisson_iters;     /* Poisson PCG iterations summed over the last step   */
    double drho;              /* ||rho^(l) - rho^(l-1)||_0 of the last step         */
    double inner_res;         /* final ||rho_out - rho_in||_0                        */
    double energy;            /* E of Sec. 3.1 (free energy E - kT S with smearing)  */
    double e_band;            /* sum_i f_i lambda_i                                  */
    double e_hartree;         /* (1/2) int V_H rho                                   */
    double e_xc;              /* int rho eps_xc                                      */
    double e_vxc;             /* int V_xc rho                                        */
    double e_nn;              /* nuclear repulsion                                   */
    double phase_ms[NAS_MAX_PHASES];   /* CUDA-event / host time per nas_phase       */
    long long phase_calls[NAS_MAX_PHASES];
    double spmm_bytes;        /* algorithmic bytes of the SpMM launches (N > 1):
                                 nnz*(8+4) + 4*(n+1) + 2*n*N*8                        */
    double spmm_flops;        /* 2*nnz*N per SpMM launch                             */
    long long kernel_launches;/* kernels this library launched during the step       */
    double spmv_bytes;        /* same for the SpMV launches (N = 1)                  */
    double spmv_flops;
    int    eig_iters;         /* LOBPCG iterations of the last step (0: dense)        */
    double poisson_spmv_ms;   /* timing = 1, poisson_fused = 0: summed CUDA-event time
                                 of the SpMV kernel of the FP64 Poisson PCG, over
                                 the first two iterations of every solve (launched
                                 directly, with events around the SpMV; the rest of
                                 the solve is replayed from the CUDA graph)          */
    long long poisson_spmv_launches; /* SpMV launches counted in poisson_spmv_ms      */
    double poisson_fused_ms;  /* timing = 1, poisson_fused = 1: summed CUDA-event time
                                 of the persistent Poisson PCG launches (every
                                 launch of every FP64 solve)                         */
    long long poisson_fused_iters; /* PCG iterations run inside those launches       */
    double e_ts;              /* -kT S of the smeared occupations (0 without smearing);
                                 `energy` includes it (the free energy)              */
    double inner_tol;         /* stop tolerance the last inner SCF used              */
    double spmm32_bytes;      /* algorithmic bytes of the FP32 SpMM launches (mixed
                                 block PCG): nnz*(4+4) + 4*(n+1) + 2*n*N*4            */
    double spmm32_flops;      /* 2*nnz*N per FP32 SpMM launch                        */
    double bvp_tol;           /* tolerance of the last step's N linear solves        */
    int eig_rr_calls;         /* Rayleigh-Ritz steps of the device LOBPCG in the step */
    int eig_rr_fallbacks;     /* of those, the ones whose basis Gram matrix was too
                                 ill-conditioned for its Cholesky factor (two-pass
                                 eigen-decomposition path)                          */
} nas_report;

/* ------------------------------------------------------------------ context */
typedef struct nas_ctx nas_ctx;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (may be NULL = the legacy default stream; pass PyTorch's current stream to
 * order the library's work with the caller's).  *out receives the context. */
int  nas_create(nas_ctx** out, int device, void* cuda_stream);
void nas_destroy(nas_ctx* ctx);
const char* nas_last_error(const nas_ctx* ctx);
const char* nas_version(void);

/* Tetrahedral mesh (Sec. 2: a shape-regular decomposition T_h of the box).
 *  which  : NAS_FINE or NAS_COARSE (the nonnested coarse mesh T_H, Sec. 3.3)
 *  order  : polynomial order of the Lagrange space on it: 1 or 2 for the fine
 *           mesh, 1 for the coarse mesh (S_H is P1).
 *  xyz    : FP64 [n_vert][3] vertex coordinates.
 *  tet    : int32 [n_tet][4] vertex ids, every tetrahedron positively oriented
 *           (det[v1-v0, v2-v0, v3-v0] > 0), else NAS_E_MESH.
 * P2 nodes are the vertices followed by one node per edge (its midpoint),
 * edges ordered by (smaller, larger) vertex id; element-local order: the 4
 * vertices, then edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3).  Boundary nodes
 * are those on a face of the vertices' bounding box (zero Dirichlet values);
 * the others, in increasing node id, are the unknowns ("dofs"). Both meshes
 * must cover the same box.  Setting a mesh invalidates the solver state. */
int nas_set_mesh(nas_ctx* ctx, int which, int order,
                 int64_t n_vert, const double* xyz,
                 int64_t n_tet, const int32_t* tet);

/* Molecule and orbitals (Sec. 2: M nuclei with charges Z_k at R_k, N orbitals).
 * After nas_init, a call that keeps n_nuc, n_orb, occupations and the
 * potential kind only moves/recharges the nuclei: the mesh structures are
 * kept and the V_ext-dependent matrices are re-assembled (the solver state is
 * kept; call nas_init to restart the SCF from scratch).
 *  R       : FP64 [n_nuc][3];  Z : FP64 [n_nuc]
 *  potential, smooth_a : see enum nas_potential
 *  n_orb   : N >= 1;  occ : FP64 [n_orb] occupations f_i (rho = sum f_i psi_i^2). */
int nas_set_system(nas_ctx* ctx, int n_nuc, const double* R, const double* Z,
                   int potential, double smooth_a, int n_orb, const double* occ);

int nas_set_options(nas_ctx* ctx, const nas_options* opt);

/* Build every mesh-dependent structure (DOF numbering, CSR patterns, the
 * transfer I_H^h by GPU point location, K, M, M_Vext, the fixed Galerkin
 * blocks B_H = I^T M I and A_H^L = I^T A^L I) and the initial state.
 *  psi0 : NULL -> initial guess = the self-consistent solution in the coarse
 *         space S_H alone (carried to the fine mesh by I), starting from
 *         rho = 0; otherwise FP64 [n_dof][n_orb] fine orbitals (host), made
 *         M-orthonormal by the library, with lambda from their Rayleigh
 *         quotients and rho_in = sum f psi^2.
 * Requires both meshes, the system and (optionally) options. */
int nas_init(nas_ctx* ctx, const double* psi0);

/* One augmented-subspace step (Algorithm 3 body): the N shifted linear
 * problems (H~ u^_i, v) = (lambda_i + mu)(psi_i, v), the fixed blocks, and the
 * inner SCF of the small Kohn-Sham problem in S_H + span{u^_i} (Sec. 3.3),
 * then the density update.  Fills *rep (may be NULL).  Returns
 * NAS_E_NOT_CONVERGED if a CG cap was hit (the state is still updated). */
int nas_step(nas_ctx* ctx, nas_report* rep);

/* Steps until ||rho^(l) - rho^(l-1)||_0 < tol_scf or max_outer steps.  Returns
 * NAS_E_NOT_CONVERGED when max_outer steps end above tol_scf, or when the last
 * step hit a CG cap (the state holds the last step either way). */
int nas_solve(nas_ctx* ctx, nas_report* rep);

/* ------------------------------------------------------------------ data out/in */
enum nas_quantity {
    NAS_Q_SIZES = 0,      /* int64[16]: n_dof, nnz, n_coarse_dof, coarse_nnz, n_elem,
                             n_quad_per_elem, n_node, n_orb, n_boundary, nnz_boundary,
                             n_vert, order, n_coarse_elem, sliced-ELL entries of K
                             (padding included), entries of I^T, balanced pieces
                             of the I^T rows                                        */
    NAS_Q_EIGVALS,        /* FP64 [N]                                                */
    NAS_Q_ORBITALS,       /* FP64 [n_dof][N]  Psi (fine interior values)              */
    NAS_Q_RHO_IN,         /* FP64 [n_elem][nq] density defining the potential         */
    NAS_Q_RHO_OUT,        /* FP64 [n_elem][nq] sum f psi^2 of the current orbitals     */
    NAS_Q_VHARTREE,       /* FP64 [n_node] nodal V_Har (boundary values included)     */
    NAS_Q_UHAT,           /* FP64 [n_dof][N] solutions of the last linear problems    */
    NAS_Q_ROWPTR,         /* int32 [n_dof+1] CSR pattern of interior matrices         */
    NAS_Q_COLIDX,         /* int32 [nnz]                                              */
    NAS_Q_K,              /* FP64 [nnz] stiffness  int grad phi_i . grad phi_j         */
    NAS_Q_M,              /* FP64 [nnz] mass                                          */
    NAS_Q_MVEXT,          /* FP64 [nnz] int V_ext phi_i phi_j                         */
    NAS_Q_ANL,            /* FP64 [nnz] A^NL of the current rho_in (Sec. 3.3)           */
    NAS_Q_HTILDE,         /* FP64 [nnz] H~ of the last linear problems                 */
    NAS_Q_TRANSFER_ELEM,  /* int32 [n_dof] coarse element containing each fine dof     */
    NAS_Q_TRANSFER_COL,   /* int32 [n_dof][4] coarse dof per vertex (-1 = boundary)    */
    NAS_Q_TRANSFER_W,     /* FP64 [n_dof][4] barycentric weights                       */
    NAS_Q_FA,             /* FP64 [m][m] last F_A, m = n_coarse_dof + N (dense)        */
    NAS_Q_FB,             /* FP64 [m][m] last F_B                                      */
    NAS_Q_DOF_NODE,       /* int32 [n_dof] node id of each dof                          */
    NAS_Q_ENERGY,         /* FP64 [6]: E, e_band, e_hartree, e_xc, e_vxc, e_nn         */
    NAS_Q_STATE_ID,       /* int64 [1]: counter bumped by every call that changes the
                             solver state (set_mesh/system/options, init, step, solve,
                             set_state); equal values mean an unchanged H~ and density */
    NAS_Q_INNER_HIST,     /* FP64 [max_inner]: ||rho_out - rho_in||_0 of every inner SCF
                             iteration of the last step (or nas_init), 0 after the last */
    NAS_Q_COUNT
};

/* Copy quantity `what` into dst (`bytes` = capacity).  on_device = 1: dst is
 * a device pointer on the context's device.  NAS_E_INVALID_ARG if too small. */
int nas_get(nas_ctx* ctx, int what, void* dst, size_t bytes, int on_device);

/* Replace the solver state (for checkpoint/resume and end-to-end timing).
 *  lam    : FP64 [N];  psi : FP64 [n_dof][N];  rho_in : FP64 [n_elem][nq]
 *  on_device: 1 if the three pointers are device pointers.
 * The Hartree potential of rho_in is recomputed by one Poisson solve. */
int nas_set_state(nas_ctx* ctx, const double* lam, const double* psi,
                  const double* rho_in, int on_device);

/* ------------------------------------------------------------------ single operations
 * Each runs one piece of the path on the context's current mesh and system,
 * with inputs and outputs given by pointer (host, or device if on_device).
 * They expose the kernels for parity tests and benchmarks; the step driver
 * uses the same kernels. */
enum nas_op {
    NAS_OP_LDA = 0,       /* in rho [cnt] -> out [2][cnt]: eps_xc, V_xc (Sec. 3.1)      */
    NAS_OP_HARTREE,       /* in rho at quad points [n_elem][nq] -> out V_H [n_node]     */
    NAS_OP_ASSEMBLE_MASS, /* in coefficient c at quad points [n_elem][nq] ->
                             out [nnz] values of int c phi_i phi_j                       */
    NAS_OP_DENSITY,       /* in Psi [n_dof][N] -> out rho [n_elem][nq] = sum f psi^2    */
    NAS_OP_APPLY_H,       /* in X [n_dof][N] -> out H~ X with the last H~ (SpMM)        */
    NAS_OP_BVP,           /* in R [n_dof][N] -> out solution of H~ U = R (block PCG;
                             FP32 inside FP64 refinement with precision = 1),
                             H~ = A^L + A^NL(rho_in) + mu M of the current state;
                             cnt = 2 n_dof N: `in` is [R ; U0], U0 the initial guess
                             (else U0 = 0).  A zero column of R gives a zero column of
                             U whatever U0                                              */
    NAS_OP_GALERKIN,      /* in fine CSR values [nnz] -> out dense I^T A I [nH][nH]     */
    NAS_OP_ENERGY_GRAD,   /* in rho at quad points [n_elem][nq] -> out [n_nuc][4]:
                             dE/d(R_k x, y, z, Z_k) = int rho dV_ext/dp + dE_nn/dp
                             (Hellmann-Feynman on the fixed mesh)                       */
    NAS_OP_BVP_VJP,       /* in [R ; G] (2 x [n_dof][N]) -> out [U ; A ; dp]: U solves
                             H~ U = R, A = H~^-1 G (adjoint, H~ symmetric) and
                             dp[n_nuc][4] = -sum_q W dV_ext/dp sum_c a_c u_c, the
                             gradient of <G, U> w.r.t. the nuclear parameters at fixed
                             R, mu and density                                           */
    NAS_OP_COUNT
};
int nas_apply(nas_ctx* ctx, int op, const void* in, int64_t cnt, void* out, int on_device);

/* Batched independent instances (one molecule and mesh per context): runs
 * `steps` augmented-subspace steps (nas_step) on each of ctxs[0..count), or
 * nas_solve when steps <= 0, with n_threads host threads taking contexts
 * from a shared queue.  The work of different contexts overlaps on the GPU,
 * which matters for instances too small to fill 152 SMs, and their host-side
 * parts (small dense eigensolves, Anderson, convergence tests) run in
 * parallel.  Every result is the one the context gives on its own: each
 * context is deterministic and shares no device data with the others.
 *  - Every context must be initialised (nas_init), distinct and on one
 *    device (NAS_E_INVALID_ARG otherwise, before any work starts).  During
 *    the call each context runs on a private non-blocking stream of the
 *    library, ordered after the work already queued on the context's own
 *    stream; at return the own stream is made to wait for it, so callers may
 *    keep sharing one stream among contexts.
 *  - status[i] receives the return code of context i's last call (NAS_OK,
 *    NAS_E_NOT_CONVERGED, or an error; an error stops that context only);
 *    reports (may be NULL) receives each context's last nas_report.
 *  - Host OpenMP threads are split evenly among the n_threads workers.
 * Returns NAS_OK when all contexts were run (see status[] for each).
 * Not in the paper (whose experiments are single molecules); it is the
 * batched-instance mode of this library. */
int nas_batch_run(nas_ctx** ctxs, int count, int steps, int n_threads, int* status, nas_report* reports);

/* Stand-alone CSR SpMM with N interleaved right-hand sides, FP64, on device
 * buffers: Y[i][c] = sum_p val[p] X[col[p]][c] for rows i < n_rows.
 *  row_ptr int32 [n_rows+1], col int32 [nnz], val FP64 [nnz], X FP64
 *  [n_cols][N], Y FP64 [n_rows][N], all device pointers; stream: cudaStream_t.
 * This is the kernel that dominates the linear solves (Sec. 3.3, Remark on
 * the cost of A_h^NL and the N boundary value problems). */
int nas_spmm_f64(int64_t n_rows, const int32_t* row_ptr, const int32_t* col,
                 const double* val, int N, const double* X, double* Y, void* stream);

/* The SpMM kernel layouts (N > 1) and their autotuner.  Layout 0 "cols" has
 * one thread per (row, column); layouts "rows<V,R>" put R rows on a warp,
 * 32/R lanes per row, each lane owning V consecutive columns (V-wide vector
 * loads of X), and broadcast the row's indices and values by shuffles.  All
 * layouts add a row's entries in CSR order, so their results are
 * bit-identical.  On the first product with a given (matrix pattern, N,
 * precision) the library times every layout the operands' alignment allows on
 * the caller's own operands and keeps the fastest.
 * nas_spmm_layouts: the number of layouts; nas_spmm_layout_name: the name of
 * layout id (static string, "?" if out of range).
 * nas_spmm_tuning: writes the tuner's record so far (a JSON list: rows, N,
 * precision, chosen layout, the time of every layout tried) into buf
 * (NUL-terminated, truncated to bytes) and returns its full length.
 * nas_spmm_f64_layout / nas_spmm_f32_layout: Y = A X with the given layout
 * (arguments as nas_spmm_f64; FP32 values and blocks for the second).
 * Errors: NAS_E_INVALID_ARG (bad sizes or pointers, unknown layout, or a
 * vector layout whose width does not divide N or whose alignment X/Y lack),
 * NAS_E_CUDA (launch failure). */
/* The dense product of the small eigensolver's preconditioner, W = T R:
 * T FP32 [nH][nH] (the inverse coarse stiffness (I^T K I)^-1 of Algorithm 3's
 * coarse space in the solver), R FP64 [nH][k], W FP64 [nH][k], device
 * pointers, row-major; FP32 products and sums.  tc = 0: SIMT kernel (register
 * tiles); tc = 1: tensor cores (tcgen05.mma kind::tf32 on split-TF32
 * operands, FP32 accumulator in tensor memory, bounded mbarrier waits).
 * Scratch for the split-K partial products (<= 16 nH k floats) is allocated
 * and freed on `stream` (stream-ordered allocator).
 * Errors: NAS_E_INVALID_ARG (nH < 0, k not in 1..256, NULL pointers),
 * NAS_E_CUDA (launch or allocation failure, or a tensor-core wait that
 * exceeded its limit). */
int nas_dense_precond_f32(int tc, int64_t nH, int k, const float* T, const double* R, double* W, void* stream);

/* The reconstruction of Algorithm 3's density update (Sec. 3.3),
 *   Psi[i][j] = sum_{q<4, icol[i][q] >= 0} ival[i][q] U[icol[i][q]][j]
 *             + sum_{c<Na} Uhat[i][c] U[nH + c][j],      i < n, j < N,
 * i.e. Psi = I u_H + U^ alpha with U = [u_H ; alpha] ((nH + Na) x N) and I
 * in the transfer's ELL form (4 coarse columns per fine row, -1 = none).
 * Device pointers, row-major: icol int32 [n][4], ival FP64 [n][4], U FP64
 * [nH + Na][N], Uhat FP64 [n][Na], Psi FP64 [n][N] (written).  tc = 0: FP64
 * SIMT kernel; tc = 1: U^ alpha on the tensor cores (tcgen05.mma kind::f16 on
 * error-free 7-bit integer slices of U^ and alpha, exact FP32 accumulation in
 * tensor memory, one rounding at the end: FP64-level accuracy), I u_H in FP64.
 * Errors: NAS_E_INVALID_ARG (n < 0, N or Na < 1, NULL pointers, or tc = 1
 * with N or Na above 64), NAS_E_CUDA (launch failure or a tensor-core wait
 * that exceeded its limit). */
int nas_reconstruct_f64(int tc, int64_t n, const int32_t* icol, const double* ival, int N, const double* U,
                        int64_t nH, int Na, const double* Uhat, double* Psi, void* stream);

/* A Gram matrix known to be symmetric, G = X^T Y (the blocks gamma = U^T M U^
 * and beta = U^T A U^ of Sec. 3.3): the upper triangle is summed and mirrored,
 * so G is exactly symmetric.  X, Y FP64 [n][N], G FP64 [N][N], device
 * pointers, row-major.  tc = 0: FP64 SIMT; tc = 1: tensor cores, per 64-row
 * chunk from error-free 7-bit integer slices with exact FP32 accumulation in
 * tensor memory, chunks added in FP64 (FP64-level accuracy).  Sums are taken
 * in a fixed order: repeated calls are bit-identical.  Scratch for the
 * partial sums (<= 1216 N^2 doubles) is allocated and freed on `stream`.
 * Errors: NAS_E_INVALID_ARG (n < 0, N < 1, N > 64 with tc = 1 or N > 90
 * without, NULL pointers), NAS_E_CUDA (launch or allocation failure, or a
 * tensor-core wait that exceeded its limit). */
int nas_gram_sym_f64(int tc, int64_t n, int N, const double* X, const double* Y, double* G, void* stream);

int nas_spmm_layouts(void);
const char* nas_spmm_layout_name(int layout);
int nas_spmm_tuning(char* buf, size_t bytes);
int nas_spmm_f64_layout(int layout, int64_t n_rows, const int32_t* row_ptr, const int32_t* col,
                        const double* val, int N, const double* X, double* Y, void* stream);
int nas_spmm_f32_layout(int layout, int64_t n_rows, const int32_t* row_ptr, const int32_t* col,
                        const float* val, int N, const float* X, float* Y, void* stream);

/* Stand-alone weighted column dot products, FP64, on device buffers:
 *   out[c] = sum_i w[i] X[i][c] Y[i][c]   for c < N   (w == NULL: w[i] = 1)
 * X, Y [n][N] row-major, w [n], out [N]: device pointers; stream: cudaStream_t.
 * This is the reduction behind the density stop test ||rho_out - rho_in||_0
 * of Algorithm 3 and the Anderson inner products (Sec. 4), with the
 * quadrature weights as w.  The sum is taken in a fixed order (per-block
 * partial sums, then one ordered pass), so repeated calls are bit-identical.
 * Scratch for the partial sums (<= 1216 * N doubles) is allocated and freed
 * on `stream` by the library (stream-ordered allocator).
 * Errors: NAS_E_INVALID_ARG (n < 0, N not in 1..256, NULL X/Y/out),
 * NAS_E_CUDA (launch or allocation failure). */
int nas_coldot_f64(int64_t n, int N, const double* X, const double* Y, const double* w, double* out,
                   void* stream);

/* Same as nas_coldot_f64, for callers that cannot allocate device memory
 * when they need the reduction (an application whose own pool allocator
 * already owns the device memory, a latency-critical loop where an allocator
 * call may block or synchronise, or code that must not gain a new
 * out-of-memory failure point mid-run).  The paper has no counterpart; this
 * is a property of the library, not of the method.
 * It allocates nothing: its scratch is a fixed array of 64 * 1216 doubles
 * (608 KiB) in device global memory inside the library, held by every GPU
 * that loads the library until the process exits.
 *  - N is limited to 1..64 (NAS_E_INVALID_ARG beyond); other arguments as
 *    for nas_coldot_f64.
 *  - The first call on a device looks up the array's device address on that
 *    device (the calling thread's current device); make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    process: after cudaDeviceReset on a device, do not call this entry point
 *    on that device again (the kept address would be stale).
 *  - All calls share the array: calls that overlap on the GPU (different
 *    streams or host threads) race and may return wrong sums; serialise
 *    them.  Each call writes every scratch entry it reads, so nothing needs
 *    clearing between calls. */
int nas_coldot_f64_noalloc(int64_t n, int N, const double* X, const double* Y, const double* w, double* out,
                           void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NAS_H */

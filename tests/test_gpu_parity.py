"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (FP64 on both sides):
  * integer/index results (CSR pattern, transfer element ids and columns): exact;
  * assembled matrices and quadrature-point quantities: 1e-13 relative to the
    largest entry (different summation order only);
  * transfer weights: 1e-14 absolute (barycentric coordinates are <= 1);
  * quantities behind an iterative solve (V_H, U^, eigenvalues, energies):
    the solves run to relative residuals of 1e-15 (BVP) and 1e-14 (Poisson), so eigenvalues and
    energies must agree to 1e-10 relative (the acceptance bar of the method).
"""
import numpy as np
import pytest

from oracle import lda as olda
from oracle import hartree as ohartree
from oracle.nas import Problem
from workloads import make_instance

pytestmark = pytest.mark.gpu

TOL_MAT = 1e-13
TOL_EIG = 1e-10


@pytest.fixture(scope="module")
def nasmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19249_gb300 import build
    import os
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2404_19249_gb300 import nas
    return nas


def _relmax(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _tight(inst):
    # the paper's mu (8 M sum Z^2) makes u^_i = coarse function + O(1/mu), so
    # the linear solves must be tight for the augmentation directions to be
    # accurate; CG's recursive residual reaches these levels in FP64
    inst.tol_bvp = 1e-15
    inst.tol_poisson = 1e-14
    inst.tol_scf = min(inst.tol_scf, 1e-10)
    return inst


# Lockstep cases need a well-posed SCF: a HOMO-LUMO gap, so that the occupied
# orbitals are well conditioned.  The paper's benzene (Sec. 4.4, 21 orbitals) is
# used for P2; the random 8-nucleus benchmark molecule has a nearly closed gap
# (about 2e-3 Ha), so it is compared over a single step (test below).
CASES = {
    "he_p1_small": dict(name="he_p1", cells=8, coarse_cells=4),
    "c6h6_p2_small": dict(name="paper_molecule", molecule="c6h6", cells=8, coarse_cells=4),
}


@pytest.fixture(scope="module", params=list(CASES))
def pair(request, nasmod):
    kw = dict(CASES[request.param])
    name = kw.pop("name")
    inst = _tight(make_instance(name, **kw))
    oracle = Problem(inst)
    s = nasmod.Solver(inst)
    s.init()
    yield request.param, inst, oracle, s
    s.close()


def test_matrices_match(pair, nasmod):
    _, inst, P, s = pair
    for q, ref in [(nasmod.NAS_Q_K, P.K), (nasmod.NAS_Q_M, P.M), (nasmod.NAS_Q_MVEXT, P.Mvext)]:
        A = s.csr(q).sorted_indices()
        B = ref.tocsr().sorted_indices()   # structural pattern (explicit zeros kept)
        assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
        assert abs(A - B).max() <= TOL_MAT * abs(B).max()


def test_transfer_bit_exact(pair, nasmod):
    _, inst, P, s = pair
    el = s.get(nasmod.NAS_Q_TRANSFER_ELEM)
    assert np.array_equal(el.astype(np.int64), P.I_elem)
    W = s.get(nasmod.NAS_Q_TRANSFER_W)
    assert np.max(np.abs(W - P.I_W)) <= 1e-14
    col = s.get(nasmod.NAS_Q_TRANSFER_COL)
    ocol = P.coarse.dof_of_node[P.I_C]
    assert np.array_equal(col.astype(np.int64), ocol)


def test_lda_kernel(pair, nasmod):
    _, inst, P, s = pair
    rng = np.random.default_rng(7)
    rho = np.concatenate([10 ** rng.uniform(-12, 3, 4000), [0.0, 1e-31, -1e-3, 3 / (4 * np.pi)]])
    out = s.apply(nasmod.NAS_OP_LDA, rho, (2, rho.size))
    e, v = olda.lda(rho)
    assert _relmax(out[0], e) < TOL_MAT and _relmax(out[1], v) < TOL_MAT
    assert np.max(np.abs(out[0] - e) / np.maximum(np.abs(e), 1e-300)) < 1e-13


def test_assembly_with_coefficient(pair, nasmod):
    _, inst, P, s = pair
    rng = np.random.default_rng(3)
    coef = rng.normal(size=P.fine.Wq.shape)
    vals = s.apply(nasmod.NAS_OP_ASSEMBLE_MASS, coef, (s.sizes()["nnz"],))
    sz = s.sizes()
    import scipy.sparse as sp
    A = sp.csr_matrix((vals, s.get(nasmod.NAS_Q_COLIDX), s.get(nasmod.NAS_Q_ROWPTR)), shape=(sz["n"], sz["n"]))
    B = P.fine.interior(P.fine.assemble_full("M", coef=coef))
    assert abs(A - B).max() <= TOL_MAT * abs(B).max()


@pytest.mark.parametrize("pairs", [1, 0])
def test_density_kernel(pair, nasmod, pairs):
    """Both density kernels: element by element (the default) and from the
    sparsity pattern's pair density (density_pairs = 1)."""
    _, inst, P, s = pair
    rng = np.random.default_rng(4)
    Psi = rng.normal(size=(P.fine.n, P.N))
    s.opt.density_pairs = pairs
    nasmod.nas_set_options(s.h, s.opt)
    try:
        rho = s.apply(nasmod.NAS_OP_DENSITY, Psi, P.fine.Wq.shape)
    finally:
        s.opt.density_pairs = 0
        nasmod.nas_set_options(s.h, s.opt)
    ref = P.density(Psi)
    assert _relmax(rho, ref) < TOL_MAT


def test_hartree_kernel(pair, nasmod):
    _, inst, P, s = pair
    c = np.array([0.3, -0.2, 0.1])
    rho = np.exp(-np.sum((P.fine.xq - c) ** 2, axis=-1))
    V = s.apply(nasmod.NAS_OP_HARTREE, rho, (P.fine.nnode,))
    ref = ohartree.hartree(P.fine, P.K, P.K_IB, rho, tol=1e-14)
    assert _relmax(V, ref) < 1e-10


def test_hartree_quadrupole_boundary_values(pair, nasmod):
    # off-centre, anisotropic charge: monopole + quadrupole boundary values
    # (Sec. 3.1's multipole expansion with the textbook 1/2)
    _, inst, P, s = pair
    xq = P.fine.xq
    rho = (np.exp(-2.0 * np.sum((xq - np.array([0.8, 0.3, -0.5])) ** 2, axis=-1))
           + 0.5 * np.exp(-np.sum((xq - np.array([-0.9, -0.4, 0.6])) ** 2, axis=-1)))
    s.opt.multipole = 2
    nasmod.nas_set_options(s.h, s.opt)
    try:
        V2 = s.apply(nasmod.NAS_OP_HARTREE, rho, (P.fine.nnode,))
    finally:
        s.opt.multipole = 0
        nasmod.nas_set_options(s.h, s.opt)
    V0 = s.apply(nasmod.NAS_OP_HARTREE, rho, (P.fine.nnode,))
    ref2 = ohartree.hartree(P.fine, P.K, P.K_IB, rho, tol=1e-14, multipole=2)
    ref0 = ohartree.hartree(P.fine, P.K, P.K_IB, rho, tol=1e-14, multipole=0)
    assert _relmax(V2, ref2) < 1e-10
    # the quadrupole term is really on (the two boundary conditions differ)
    assert _relmax(ref2, ref0) > 1e-4 and _relmax(V2, V0) > 1e-4


def test_hartree_persistent_and_per_phase_pcg(nasmod):
    """The persistent cooperative Poisson PCG (grid-wide barriers between the
    phases) and the per-phase kernels replayed from a CUDA graph solve the
    same two-level preconditioned system with the same grid, rows per thread
    and partial sums: both match the oracle's Hartree potential and each other
    bit for bit."""
    inst = make_instance("mol8_p2", cells=14, coarse_cells=6)
    inst.tol_poisson = 1e-13
    P = Problem(inst, with_transfer=False)
    c = np.array([0.5, -1.0, 0.25])
    rho = np.exp(-0.5 * np.sum((P.fine.xq - c) ** 2, axis=-1)) + 0.3 * np.exp(-np.sum((P.fine.xq + c) ** 2, axis=-1))
    ref = ohartree.hartree(P.fine, P.K, P.K_IB, rho, tol=1e-14)
    out = {}
    for fused in (0, 1):
        s = nasmod.Solver(inst, poisson_fused=fused)
        s.init()
        out[fused] = s.apply(nasmod.NAS_OP_HARTREE, rho, (P.fine.nnode,))
        s.close()
    for fused in (0, 1):
        assert _relmax(out[fused], ref) < 1e-10, fused
    assert np.array_equal(out[1], out[0])


def test_galerkin_kernel(pair, nasmod):
    _, inst, P, s = pair
    sz = s.sizes()
    D = s.apply(nasmod.NAS_OP_GALERKIN, s.get(nasmod.NAS_Q_M), (sz["nH"], sz["nH"]))
    ref = (P.I.T @ P.M @ P.I).toarray()
    assert _relmax(D, ref) < TOL_MAT


def test_lockstep_steps(pair, nasmod):
    """Initial coarse-space SCF and two augmented steps, compared step by step."""
    _, inst, P, s = pair
    st = P.initial_state()
    lam0 = s.get(nasmod.NAS_Q_EIGVALS)
    assert _relmax(lam0, st.lam) < TOL_EIG
    for step in range(2):
        r, rep = s.step()
        assert r == 0
        st = P.step(st)
        lam = s.get(nasmod.NAS_Q_EIGVALS)
        assert _relmax(lam, st.lam) < TOL_EIG, (step, lam, st.lam)
        # a residual sitting on the stopping threshold may take one more or one
        # fewer inner iteration on either side
        assert abs(rep.n_inner - st.n_inner) <= 1
        E = s.get(nasmod.NAS_Q_ENERGY)[0]
        assert abs(E - P.energy(st)) < TOL_EIG * abs(E)
        rho = s.get(nasmod.NAS_Q_RHO_OUT)
        assert _relmax(rho, st.rho_out) < 1e-8
        assert abs(rep.drho - st.info["drho"]) < 1e-8 * max(st.info["drho"], 1e-8)


def test_lockstep_fp64_simt_contractions(nasmod):
    """The lockstep comparison with the FP64 SIMT reconstruction and Gram
    kernels (dense_tc = 0; every other solver test runs the tensor-core
    ones) on the P2 benzene case: initial SCF and two steps at 1e-10."""
    inst = _tight(make_instance("paper_molecule", molecule="c6h6", cells=8, coarse_cells=4))
    P = Problem(inst)
    st = P.initial_state()
    s = nasmod.Solver(inst, dense_tc=0)
    s.init()
    try:
        assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
        for step in range(2):
            r, rep = s.step()
            assert r == 0
            st = P.step(st)
            assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
            assert abs(rep.energy - P.energy(st)) < TOL_EIG * abs(P.energy(st))
    finally:
        s.close()


INEXACT = {
    "exact": {},
    "poisson_adaptive": dict(poisson_adaptive=1),
    # eig_dense_max = 0: the small problem goes to the device LOBPCG, where the tolerance applies
    "eig_adapt_1e-2": dict(eig_adapt=1e-2, eig_dense_max=0),
    "all_inexact": dict(poisson_adaptive=1, eig_adapt=1e-2, inner_adapt=1e-2, bvp_adapt=1e-2, eig_dense_max=0),
}


@pytest.mark.parametrize("opts", list(INEXACT.values()), ids=list(INEXACT))
def test_converged_helium_matches_oracle(nasmod, opts):
    """Converged Algorithm 3 = the oracle's fixed point, also with every
    inexact option the benchmark uses: inner Poisson tolerance tied to the
    density residual, LOBPCG tolerance 1e-2 x the inner residual, inner SCF
    and linear solves stopped at 1e-2 x the previous step's density change
    (near convergence all of them tighten to the exact tolerances)."""
    inst = _tight(make_instance("he_p1", cells=6, coarse_cells=3, tol_scf=1e-12, mu=2.0, max_outer=400))
    P = Problem(inst)
    ref = P.solve(max_outer=400)
    s = nasmod.Solver(inst, **opts)
    s.init()
    r, rep = nasmod.nas_solve(s.h)
    assert rep.drho < 1e-11
    lam = s.get(nasmod.NAS_Q_EIGVALS)
    assert _relmax(lam, ref.lam) < TOL_EIG
    E = s.get(nasmod.NAS_Q_ENERGY)[0]
    assert abs(E - P.energy(ref)) < TOL_EIG * abs(E)
    s.close()


def test_spmm_standalone(nasmod):
    torch = pytest.importorskip("torch")
    inst = make_instance("mol8_p2", cells=6, coarse_cells=4)
    P = Problem(inst, with_transfer=False)
    A = P.K.tocsr().sorted_indices()
    for N in (1, 3, 8, 21):
        X = np.random.default_rng(N).normal(size=(A.shape[0], N))
        dev = torch.device("cuda:0")
        rp = torch.tensor(A.indptr, dtype=torch.int32, device=dev)
        ci = torch.tensor(A.indices, dtype=torch.int32, device=dev)
        va = torch.tensor(A.data, dtype=torch.float64, device=dev)
        Xd = torch.tensor(X, dtype=torch.float64, device=dev)
        Yd = torch.zeros((A.shape[0], N), dtype=torch.float64, device=dev)
        nasmod.nas_spmm_f64(A.shape[0], rp.data_ptr(), ci.data_ptr(), va.data_ptr(), N, Xd.data_ptr(),
                            Yd.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        ref = A @ X
        assert _relmax(Yd.cpu().numpy(), ref) < 1e-14


def test_benchmark_molecule_first_step(nasmod):
    """One augmented step of the 8-nucleus benchmark molecule on a reduced mesh,
    with the paper's mu = 8 M sum Z^2.  (The workload's own mu = max Z^2 makes
    the shifted operator ~250x worse conditioned on this 6^3 mesh; one step
    from the coarse-space start, far from self-consistency, then depends to
    first order on the FP64 CG solves, whose attainable accuracy is ~eps
    cond(H~): GPU and the oracle's exact solves differ by 1.8e-9.)"""
    inst = _tight(make_instance("mol8_p2", cells=6, coarse_cells=4, mu=None))
    P = Problem(inst)
    s = nasmod.Solver(inst)
    s.init()
    st = P.initial_state()
    assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
    r, rep = s.step()
    st = P.step(st)
    assert r == 0 and abs(rep.n_inner - st.n_inner) <= 1
    assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
    assert abs(s.get(nasmod.NAS_Q_ENERGY)[0] - P.energy(st)) < TOL_EIG * abs(P.energy(st))
    s.close()


@pytest.mark.parametrize("eig_device,eig_precond", [(0, 0), (1, 0), (1, 1)],
                         ids=["host_lobpcg", "device_lobpcg_diag", "device_lobpcg_coarse_stiffness"])
def test_lobpcg_path_matches_oracle(nasmod, eig_device, eig_precond):
    """The warm-started LOBPCG eigensolvers used for large coarse spaces (host
    block vectors, or device block vectors with a host Rayleigh-Ritz) give the
    same steps as the oracle's dense generalized eigensolver."""
    inst = _tight(make_instance("paper_molecule", molecule="c6h6", cells=8, coarse_cells=4))
    P = Problem(inst)
    s = nasmod.Solver(inst, eig_dense_max=0, eig_tol=1e-12, eig_device=eig_device, eig_precond=eig_precond)
    s.init()
    st = P.initial_state()
    assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
    for _ in range(2):
        r, rep = s.step()
        st = P.step(st)
        assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
    s.close()


def test_coldot_standalone(nasmod):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(11)
    for n, N in ((1, 1), (1000, 1), (123457, 21), (5000, 64)):
        X = rng.normal(size=(n, N))
        Y = rng.normal(size=(n, N))
        w = rng.uniform(0.1, 2.0, size=n)
        Xd, Yd, wd = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (X, Y, w))
        out = torch.zeros(N, dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream().cuda_stream
        nasmod.nas_coldot_f64(n, N, Xd.data_ptr(), Yd.data_ptr(), wd.data_ptr(), out.data_ptr(), st)
        torch.cuda.synchronize()
        ref = np.einsum("i,ic,ic->c", w, X, Y)
        scale = np.einsum("i,ic,ic->c", w, np.abs(X), np.abs(Y))
        assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-13 * scale)
        out2 = torch.zeros_like(out)
        nasmod.nas_coldot_f64(n, N, Xd.data_ptr(), Yd.data_ptr(), wd.data_ptr(), out2.data_ptr(), st)
        torch.cuda.synchronize()
        assert torch.equal(out, out2)   # fixed summation order: bit-identical repeats


@pytest.mark.parametrize("poisson_f32", [0, 1])
def test_mixed_precision_poisson_matches_fp64(nasmod, poisson_f32):
    """Mixed precision (FP32 block PCG of the N shifted problems and, with
    poisson_f32, FP32 Poisson PCG, each inside FP64 iterative refinement)
    reproduces the FP64 steps: eigenvalues within 1e-8 Ha and the oracle
    within 1e-10."""
    inst = _tight(make_instance("paper_molecule", molecule="c6h6", cells=8, coarse_cells=4))
    P = Problem(inst)
    res = {}
    for prec in (0, 1):
        # adaptive inner Poisson tolerance: the early inner iterations ask for
        # loose tolerances, which the mixed form solves with FP32 inner PCG
        s = nasmod.Solver(inst, precision=prec, poisson_adaptive=1, poisson_f32=poisson_f32, timing=1)
        s.init()
        for _ in range(2):
            r, rep = s.step()
            assert r == 0
            spmv32 = rep.phase_calls[nasmod.PHASES.index("spmv32")]
            assert (spmv32 > 0) == (prec == 1 and poisson_f32 == 1)
            assert (rep.phase_calls[nasmod.PHASES.index("spmm32")] > 0) == (prec == 1)
        res[prec] = (s.get(nasmod.NAS_Q_EIGVALS), s.get(nasmod.NAS_Q_ENERGY)[0])
        s.close()
    assert np.max(np.abs(res[1][0] - res[0][0])) < 1e-8
    assert abs(res[1][1] - res[0][1]) < 1e-8
    st = P.initial_state()
    for _ in range(2):
        st = P.step(st)
    assert _relmax(res[1][0], st.lam) < TOL_EIG


def test_smeared_occupations_lockstep(nasmod):
    """Fermi-Dirac occupations (option smearing): a Be-like atom whose 2s and
    2p levels share two electrons; initial SCF and three steps against the
    oracle, eigenvalues, occupations and free energies at 1e-10."""
    inst = _tight(make_instance("he_p1", cells=6, coarse_cells=3, mu=6.0))
    inst.Z = np.array([4.0])
    inst.occ = np.array([2.0, 2.0, 0.0, 0.0])
    inst.smearing = 0.05
    P = Problem(inst)
    st = P.initial_state()
    s = nasmod.Solver(inst)
    s.init()
    try:
        assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
        for step in range(3):
            r, rep = s.step()
            assert r == 0
            st = P.step(st)
            assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
            E = P.energy(st)
            assert abs(rep.energy - E) < TOL_EIG * abs(E)
            assert abs(rep.e_ts - st.minus_TS) < TOL_EIG * abs(E)
            assert rep.e_ts < 0.0 and 0.0 < st.occ[2] < 2.0
            rho = s.get(nasmod.NAS_Q_RHO_OUT)
            assert _relmax(rho, st.rho_out) < 1e-8
    finally:
        s.close()


@pytest.mark.parametrize("restart", [0.0, 1.5])
def test_deep_anderson_history_lockstep(nasmod, restart):
    """Anderson mixing with a 6-entry history (beta 0.15): LiH's inner SCF
    takes 20-30 iterations, so the history wraps around several times;
    initial SCF and two steps against the oracle's mixing with the same depth,
    eigenvalues and energies at 1e-10.  With restart 1.5 the history is
    cleared at the residual jumps of 1.70x, 2.29x (initial SCF) and 1.52x
    (first step) over the best residual, the same iterations on both sides."""
    inst = _tight(make_instance("paper_molecule", molecule="lih", cells=8, coarse_cells=4))
    inst.anderson_depth = 6
    inst.anderson_beta = 0.15
    inst.anderson_restart = restart
    P = Problem(inst)
    st = P.initial_state()
    assert st.inner_converged and st.n_inner > 12
    s = nasmod.Solver(inst)
    s.init()
    try:
        assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
        for step in range(2):
            r, rep = s.step()
            assert r == 0
            st = P.step(st)
            assert st.inner_converged and rep.inner_converged
            assert _relmax(s.get(nasmod.NAS_Q_EIGVALS), st.lam) < TOL_EIG
            assert abs(rep.n_inner - st.n_inner) <= 1
            assert abs(rep.energy - P.energy(st)) < TOL_EIG * abs(P.energy(st))
    finally:
        s.close()

"""The benchmark workload at full size (8-nucleus P2 molecule, 970,299
unknowns), run with bench.py's solver settings: outputs the oracle can
compute one by one on samples, and properties that hold at any size."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem
from oracle.transfer import build_transfer
from workloads import make_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19249_gb300 import nas
    inst = make_instance("mol8_p2")
    s = nas.Solver(inst, tol_poisson=1e-10, tol_bvp=1e-10, check_every=4, poisson_adaptive=1, eig_adapt=1e-2)
    s.init()
    r, rep = s.step()
    F = fem.Space(inst.fine_xyz, inst.fine_tet, inst.order)
    yield nas, inst, s, r, rep, F
    s.close()


def test_step_status_and_sizes(full):
    nas, inst, s, r, rep, F = full
    sz = s.sizes()
    assert r == 0 and rep.inner_converged == 1
    assert sz["n"] == F.n == 970299 and sz["N"] == len(inst.occ)
    lam = s.get(nas.NAS_Q_EIGVALS)
    assert np.all(np.diff(lam) >= 0) and np.all(np.isfinite(lam))
    assert np.isfinite(rep.energy)


def test_transfer_sampled_bit_exact(full):
    """Coarse element ids (canonical smallest id), columns and weights of
    I_H^h at 1500 sampled fine unknowns against the oracle's Algorithm 1."""
    nas, inst, s, r, rep, F = full
    C = fem.Space(inst.coarse_xyz, inst.coarse_tet, 1)
    rows = np.sort(np.random.default_rng(21).choice(F.n, 1500, replace=False))
    _, elem, W, Cn = build_transfer(F, C, rows)
    assert np.array_equal(s.get(nas.NAS_Q_TRANSFER_ELEM)[rows].astype(np.int64), elem)
    assert np.array_equal(s.get(nas.NAS_Q_TRANSFER_COL)[rows].astype(np.int64), C.dof_of_node[Cn])
    assert np.max(np.abs(s.get(nas.NAS_Q_TRANSFER_W)[rows] - W)) <= 1e-14


def test_density_sampled_elements(full):
    """rho = sum_i f_i psi_i^2 at the quadrature points of 600 sampled elements,
    from the library's orbitals, against the oracle's basis tables."""
    nas, inst, s, r, rep, F = full
    psi = s.get(nas.NAS_Q_ORBITALS)
    nodal = F.to_nodes(psi)
    es = np.sort(np.random.default_rng(22).choice(F.ne, 600, replace=False))
    pq = np.einsum("qa,eac->eqc", F.phi, nodal[F.elem[es]])
    ref = np.einsum("eqc,c->eq", pq * pq, np.asarray(inst.occ))
    got = s.get(nas.NAS_Q_RHO_OUT)[es]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_orbitals_mass_orthonormal(full):
    """The Rayleigh-Ritz vectors of the augmented space are M-orthonormal in the
    fine space (F_B is their exact Gram matrix): Psi^T M Psi = I."""
    nas, inst, s, r, rep, F = full
    rp, ci, mv = (s.get(q) for q in (nas.NAS_Q_ROWPTR, nas.NAS_Q_COLIDX, nas.NAS_Q_M))
    M = sp.csr_matrix((mv, ci, rp), shape=(F.n, F.n))
    psi = s.get(nas.NAS_Q_ORBITALS)
    G = psi.T @ (M @ psi)
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-9

"""Degenerate sizes and error behaviour through the C ABI: empty inputs,
empty CSR rows, ragged column counts, and the documented error codes for
inconsistent inputs (no fault is provoked: every case is rejected by the
host-side checks or handled as an empty launch)."""
import numpy as np
import pytest
import scipy.sparse as sp

from workloads import make_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19249_gb300 import nas
    return nas, torch


def test_empty_and_ragged_spmm(env):
    nas, torch = env
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream().cuda_stream
    # empty matrix: nothing launched, Y untouched
    rp = torch.zeros(1, dtype=torch.int32, device=dev)
    col = torch.zeros(1, dtype=torch.int32, device=dev)
    val = torch.zeros(1, dtype=torch.float64, device=dev)
    X = torch.ones(4, dtype=torch.float64, device=dev)
    Y = torch.full((4,), 7.0, dtype=torch.float64, device=dev)
    assert nas.nas_spmm_f64(0, rp.data_ptr(), col.data_ptr(), val.data_ptr(), 1, X.data_ptr(), Y.data_ptr(), st) == 0
    torch.cuda.synchronize()
    assert torch.all(Y == 7.0)
    # rows without entries, ragged row lengths, 1 and 3 columns
    rng = np.random.default_rng(4)
    A = sp.random(257, 300, density=0.03, format="csr", random_state=5)
    A = A.tolil()
    A[10, :] = 0
    A[100:140, :] = 0
    A = A.tocsr()
    A.sort_indices()
    for N in (1, 3):
        Xh = rng.normal(size=(300, N))
        ref = A @ Xh
        d = [torch.tensor(a, device=dev) for a in (A.indptr.astype(np.int32), A.indices.astype(np.int32),
                                                   A.data.astype(np.float64), Xh)]
        Yd = torch.full((257, N), np.nan, dtype=torch.float64, device=dev)
        assert nas.nas_spmm_f64(257, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), N, d[3].data_ptr(),
                                Yd.data_ptr(), st) == 0
        torch.cuda.synchronize()
        got = Yd.cpu().numpy()
        assert np.all(got[10] == 0.0) and np.all(got[100:140] == 0.0)
        assert np.max(np.abs(got - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_empty_coldot(env):
    nas, torch = env
    dev = torch.device("cuda:0")
    X = torch.zeros(1, dtype=torch.float64, device=dev)
    out = torch.full((3,), 5.0, dtype=torch.float64, device=dev)
    assert nas.nas_coldot_f64(0, 3, X.data_ptr(), X.data_ptr(), 0, out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert torch.all(out == 0.0)


def test_error_codes(env):
    nas, torch = env
    # more orbitals than coarse unknowns: the coarse-space initial guess is impossible
    inst = make_instance("harmonic", cells=4, coarse_cells=2, n_orb=3)
    s = nas.Solver(inst)
    with pytest.raises(nas.NasError) as e:
        s.init()
    assert e.value.code == -1
    s.close()
    # fine and coarse meshes covering different boxes
    inst = make_instance("he_p1", cells=6, coarse_cells=3)
    inst.coarse_xyz = inst.coarse_xyz * 0.9
    s = nas.Solver(inst)
    with pytest.raises(nas.NasError) as e:
        s.init()
    assert e.value.code == -2
    s.close()
    # an unknown operation
    inst = make_instance("he_p1", cells=6, coarse_cells=3)
    s = nas.Solver(inst)
    s.init()
    with pytest.raises(nas.NasError):
        nas.nas_apply(s.h, 99, np.zeros(4), np.zeros(4))
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_bvp_zero_rhs_column_with_nonzero_guess(env, precision):
    """A zero right-hand side has the zero solution whatever the initial guess:
    the block PCG (FP64, and FP32 inside FP64 refinement) returns an exactly
    zero column for it and solves the other columns as from a zero guess."""
    nas, torch = env
    inst = make_instance("harmonic", cells=8, coarse_cells=4, n_orb=3)
    inst.tol_bvp = 1e-12
    s = nas.Solver(inst, precision=precision)
    s.init()
    n, N = s.sizes()["n"], s.sizes()["N"]
    rng = np.random.default_rng(11)
    R = rng.normal(size=(n, N))
    R[:, 1] = 0.0
    U0 = rng.normal(size=(n, N))
    U_guess = s.apply(nas.NAS_OP_BVP, np.concatenate([R.ravel(), U0.ravel()]), (n, N), cnt=2 * n * N)
    U_zero = s.apply(nas.NAS_OP_BVP, R, (n, N))
    s.close()
    assert np.all(U_guess[:, 1] == 0.0) and np.all(U_zero[:, 1] == 0.0)
    for j in (0, 2):
        assert np.max(np.abs(U_guess[:, j] - U_zero[:, j])) < 1e-9 * np.max(np.abs(U_zero[:, j]))

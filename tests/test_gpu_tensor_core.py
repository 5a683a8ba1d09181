"""The tensor-core product of the small eigensolver's preconditioner
(tcgen05.mma kind::tf32 on split-TF32 operands, FP32 accumulator in tensor
memory), through the C ABI: against an FP64 NumPy product and the FP32 SIMT
kernel, for ragged sizes (nH not a multiple of the 128-row tile or of the
32-element K tile, k not a multiple of 16), and inside the device LOBPCG
against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19249_gb300 import nas
    return nas, torch


@pytest.mark.parametrize("nH,k", [(1, 1), (37, 5), (200, 16), (1000, 80), (3375, 80), (513, 256)])
def test_tensor_core_product_matches_fp64(env, nH, k):
    nas, torch = env
    rng = np.random.default_rng(nH + k)
    A = rng.standard_normal((nH, nH))
    T = (A @ A.T / nH + np.eye(nH)).astype(np.float32)     # SPD, like an inverse stiffness
    R = rng.standard_normal((nH, k))
    ref = T.astype(np.float64) @ R
    dev = torch.device("cuda:0")
    Td = torch.tensor(T, device=dev)
    Rd = torch.tensor(R, device=dev)
    out = {}
    for tc in (0, 1):
        W = torch.full((nH, k), 7.0, dtype=torch.float64, device=dev)
        nas.nas_dense_precond_f32(tc, nH, k, Td.data_ptr(), Rd.data_ptr(), W.data_ptr())
        torch.cuda.synchronize()
        out[tc] = W.cpu().numpy()
    scale = np.max(np.abs(ref))
    # FP32 operands (T exactly, R rounded once) and FP32 accumulation: ~1e-6
    assert np.max(np.abs(out[0] - ref)) < 2e-5 * scale
    assert np.max(np.abs(out[1] - ref)) < 2e-5 * scale
    assert np.max(np.abs(out[1] - out[0])) < 2e-5 * scale


def test_tensor_core_preconditioner_in_lobpcg_matches_oracle(env):
    nas, torch = env
    from oracle.nas import Problem
    from workloads import make_instance
    inst = make_instance("paper_molecule", molecule="c6h6", cells=8, coarse_cells=4)
    inst.tol_bvp, inst.tol_poisson, inst.tol_scf = 1e-15, 1e-14, 1e-10
    P = Problem(inst)
    st = P.step(P.initial_state())
    s = nas.Solver(inst, eig_dense_max=0, eig_tol=1e-12, eig_device=1, eig_precond=2)
    s.init()
    s.step()
    lam = s.get(nas.NAS_Q_EIGVALS)
    s.close()
    assert np.max(np.abs(lam - st.lam)) < 1e-10 * np.max(np.abs(st.lam))

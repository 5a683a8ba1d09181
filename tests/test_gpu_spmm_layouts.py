"""The SpMM kernel layouts and their autotuner, through the C ABI.

Every layout adds a row's entries in CSR order, so all layouts must give
bit-identical results, in FP64 and in FP32, for ragged rows (empty rows, rows
longer than one 32-entry chunk of a warp) and for column counts that no vector
width divides; FP64 must also match SciPy.  Operands whose alignment a vector
layout cannot use are rejected by the host-side check (no launch).  After a
solver step the autotuner has recorded a choice for the block of N columns.
"""
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


def _ragged(n_rows=1003, n_cols=1201, seed=3):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 24, size=n_rows)
    lens[::97] = 0                      # empty rows
    lens[5::101] = 70                   # rows spanning three 32-entry chunks
    rows, cols = [], []
    for r, k in enumerate(lens):
        c = np.sort(rng.choice(n_cols, size=min(int(k), n_cols), replace=False))
        rows += [r] * len(c)
        cols += list(c)
    vals = rng.standard_normal(len(rows))
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_rows, n_cols))


@pytest.mark.parametrize("N", [1, 2, 3, 21, 64, 66])
@pytest.mark.parametrize("fp32", [False, True])
def test_layouts_bit_identical(env, N, fp32):
    nas, torch = env
    A = _ragged()
    dt = torch.float32 if fp32 else torch.float64
    dev = torch.device("cuda:0")
    rp = torch.tensor(A.indptr, dtype=torch.int32, device=dev)
    ci = torch.tensor(A.indices, dtype=torch.int32, device=dev)
    va = torch.tensor(A.data, dtype=dt, device=dev)
    Xh = np.random.default_rng(N).standard_normal((A.shape[1], N))
    X = torch.tensor(Xh, dtype=dt, device=dev)
    names = nas.nas_spmm_layouts()
    ref = None
    st = torch.cuda.current_stream().cuda_stream
    for lid, name in enumerate(names):
        vec = 1 if name == "cols" else int(name[5])
        if N % vec or (not fp32 and vec > 2):
            continue
        Y = torch.full((A.shape[0], N), 7.0, dtype=dt, device=dev)
        nas.nas_spmm_layout(lid, A.shape[0], rp.data_ptr(), ci.data_ptr(), va.data_ptr(), N, X.data_ptr(),
                            Y.data_ptr(), fp32=fp32, stream=st)
        torch.cuda.synchronize()
        y = Y.cpu().numpy()
        if ref is None:
            ref = y
            if not fp32:
                exact = A @ Xh
                assert np.max(np.abs(y - exact)) <= 1e-13 * max(1.0, np.max(np.abs(exact)))
        else:
            assert np.array_equal(y, ref), (name, N, fp32)


def test_misaligned_vector_layout_is_rejected(env):
    nas, torch = env
    A = _ragged(64, 64)
    dev = torch.device("cuda:0")
    rp = torch.tensor(A.indptr, dtype=torch.int32, device=dev)
    ci = torch.tensor(A.indices, dtype=torch.int32, device=dev)
    va = torch.tensor(A.data, dtype=torch.float32, device=dev)
    X = torch.zeros(64 * 64 + 1, dtype=torch.float32, device=dev)
    Y = torch.zeros(64 * 64, dtype=torch.float32, device=dev)
    lid = nas.nas_spmm_layouts().index("rows<4,1>")
    with pytest.raises(nas.NasError):   # X + 1 float is not 16-byte aligned: refused before any launch
        nas.nas_spmm_layout(lid, 64, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 64, X.data_ptr() + 4,
                            Y.data_ptr(), fp32=True)
    with pytest.raises(nas.NasError):   # 4 does not divide N = 66
        nas.nas_spmm_layout(lid, 64, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 66, X.data_ptr(),
                            Y.data_ptr(), fp32=True)


def test_autotuner_records_a_choice(env):
    nas, torch = env
    inst = make_instance("paper_molecule", molecule="c6h6", cells=6, coarse_cells=4)
    s = nas.Solver(inst)
    s.init()
    s.step()
    n, N = s.sizes()["n"], s.sizes()["N"]
    s.close()
    rec = [r for r in nas.nas_spmm_tuning() if r["rows"] == n and r["N"] == N and r["type"] == "f64"]
    assert rec and rec[0]["layout"] in nas.nas_spmm_layouts()
    # N = 21: no vector width divides it, so "cols" and the three scalar row layouts are tried
    assert all(t > 0 for t in rec[0]["ms"].values()) and len(rec[0]["ms"]) == 4

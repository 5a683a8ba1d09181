"""The oracle's OpenMP CSR SpMM (oracle/spmm_omp.c, the CPU baseline's
SpMM) against SciPy's product, on the CPU, for one and several threads and
for N = 1 and N interleaved right-hand sides."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import build_c


@pytest.fixture(scope="module")
def lib():
    try:
        return build_c.load()
    except RuntimeError as e:
        pytest.skip(str(e))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@pytest.mark.parametrize("N,threads", [(1, 1), (21, 1), (21, 4), (8, 3)])
def test_spmm_equals_scipy(lib, N, threads):
    rng = np.random.default_rng(N + threads)
    n = 1537
    A = sp.random(n, n, density=0.01, format="csr", random_state=rng) + sp.eye(n, format="csr")
    A.sort_indices()
    rowptr = A.indptr.astype(np.int32)
    col = A.indices.astype(np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    X = rng.standard_normal((n, N))
    Y = np.full((n, N), np.nan)
    lib.oracle_spmm(n, _p(rowptr), _p(col), _p(val), N, _p(X), _p(Y), threads)
    np.testing.assert_allclose(Y, A @ X, rtol=1e-13, atol=1e-13)
    t = lib.oracle_spmm_seconds(n, _p(rowptr), _p(col), _p(val), N, _p(X), _p(Y), threads, 2)
    assert t > 0.0
    np.testing.assert_allclose(Y, A @ X, rtol=1e-13, atol=1e-13)


def test_empty_rows(lib):
    n, N = 5, 3
    rowptr = np.array([0, 0, 2, 2, 3, 3], dtype=np.int32)
    col = np.array([1, 4, 0], dtype=np.int32)
    val = np.array([2.0, -1.0, 0.5])
    X = np.arange(n * N, dtype=np.float64).reshape(n, N)
    Y = np.full((n, N), np.nan)
    lib.oracle_spmm(n, _p(rowptr), _p(col), _p(val), N, _p(X), _p(Y), 2)
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    np.testing.assert_array_equal(Y, A @ X)

"""The symmetric Gram matrices G = X^T Y of Sec. 3.3 (gamma = U^T M U^,
beta = U^T A U^) on the tensor cores (per 64-row chunk from error-free 7-bit
integer slices, exact FP32 accumulation in tensor memory, chunks added in
FP64), through the C ABI.

* Against NumPy FP64 for row counts that leave ragged chunks, N from 1 to 64,
  rows of very different magnitudes (orbitals decaying over the mesh), zero
  rows and subnormal entries: every upper-triangle entry within the scheme's
  per-chunk bound 2^-38 sum_chunks max|X_ca| max|Y_cb| (a factor 4 above its
  derivation) plus FP64 rounding relative to |X|^T |Y|.
* G exactly symmetric, repeated calls bit-identical.
* Integer inputs whose FP64 sums are exact: the tensor-core G equals the exact
  result bit for bit.
* Against the FP64 SIMT kernel, and the argument checks.
"""
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


def _inputs(n, N, seed, integer=False):
    rng = np.random.default_rng(seed)
    if integer:
        return (rng.integers(-1000, 1001, size=(n, N)).astype(np.float64),
                rng.integers(-1000, 1001, size=(n, N)).astype(np.float64))
    decay = 10.0 ** rng.uniform(-10, 1, size=(n, 1))        # row magnitudes over the mesh
    X = rng.standard_normal((n, N)) * decay
    Y = rng.standard_normal((n, N)) * decay * 10.0 ** rng.uniform(-2, 2, size=(1, N))
    X[::31] = 0.0
    Y[3::37, 0] = 1e-310
    return X, Y


def _gram(nas, torch, tc, X, Y):
    dev = torch.device("cuda:0")
    n, N = X.shape
    Xd = torch.tensor(X, device=dev)
    Yd = torch.tensor(Y, device=dev)
    G = torch.full((N, N), 7.0, dtype=torch.float64, device=dev)
    nas.nas_gram_sym_f64(tc, n, N, Xd.data_ptr(), Yd.data_ptr(), G.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return G.cpu().numpy()


def _bound(X, Y):
    n, N = X.shape
    nch = (n + 63) // 64
    pad = nch * 64 - n
    Xm = np.max(np.abs(np.vstack([X, np.zeros((pad, N))])).reshape(nch, 64, N), axis=1)
    Ym = np.max(np.abs(np.vstack([Y, np.zeros((pad, N))])).reshape(nch, 64, N), axis=1)
    return 2.0 ** -38 * (Xm.T @ Ym) + 1e-14 * (np.abs(X).T @ np.abs(Y)) + 1e-300


@pytest.mark.parametrize("n,N", [(1, 1), (63, 7), (64, 16), (65, 21), (1000, 48), (100003, 64), (4097, 64)])
def test_tensor_core_gram_within_bound(env, n, N):
    nas, torch = env
    X, Y = _inputs(n, N, seed=n + N)
    ref = X.T @ Y
    G = _gram(nas, torch, 1, X, Y)
    assert np.array_equal(G, G.T)
    iu = np.triu_indices(N)
    b = _bound(X, Y)
    err = np.abs(G - ref)
    assert np.all(err[iu] <= b[iu]), (np.max(err[iu] / b[iu]), n, N)
    assert np.array_equal(_gram(nas, torch, 1, X, Y), G)        # fixed summation order
    S = _gram(nas, torch, 0, X, Y)
    assert np.all(np.abs(G - S)[iu] <= 2 * b[iu])


@pytest.mark.parametrize("n,N", [(500, 64), (70, 5)])
def test_tensor_core_gram_exact_on_integers(env, n, N):
    nas, torch = env
    X, Y = _inputs(n, N, seed=11, integer=True)
    exact = X.T @ Y          # every product and partial sum is an integer below 2^53
    iu = np.triu_indices(N)
    G = _gram(nas, torch, 1, X, Y)
    assert np.array_equal(G[iu], exact[iu]) and np.array_equal(G, G.T)


def test_tensor_core_gram_edges(env):
    nas, torch = env
    dev = torch.device("cuda:0")
    X = torch.zeros((4, 65), dtype=torch.float64, device=dev)
    G = torch.zeros((65, 65), dtype=torch.float64, device=dev)
    with pytest.raises(nas.NasError):       # N > 64: refused on the host, nothing launched
        nas.nas_gram_sym_f64(1, 4, 65, X.data_ptr(), X.data_ptr(), G.data_ptr())
    nas.nas_gram_sym_f64(0, 4, 65, X.data_ptr(), X.data_ptr(), G.data_ptr())
    # no rows: G = 0
    G2 = torch.full((8, 8), 3.0, dtype=torch.float64, device=dev)
    nas.nas_gram_sym_f64(1, 0, 8, X.data_ptr(), X.data_ptr(), G2.data_ptr())
    torch.cuda.synchronize()
    assert not G2.any()

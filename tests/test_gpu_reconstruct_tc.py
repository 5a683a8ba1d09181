"""The reconstruction Psi = I u_H + U^ alpha of Algorithm 3 with its dense
part on the tensor cores (error-free 7-bit integer slices, exact FP32
accumulation in tensor memory), through the C ABI.

* Against NumPy FP64 for ragged row counts (tile tails), N and Na from 1 to
  64, rows and columns of very different magnitudes, zero rows and columns,
  subnormal entries and missing transfer columns: every entry within the
  scheme's bound, 2^-38 max_c |U^_ic| max_c |alpha_cj| (a factor 4 above its
  derivation), plus FP64 rounding relative to the sums of absolute terms
  (sum_q |w_iq| |u_H| + sum_c |U^_ic| |alpha_cj|): both sums cancel.
* Integer inputs whose products and sums FP64 represents exactly: the
  tensor-core result equals the exact result bit for bit (a truncated slice or
  an inexact accumulator would show here first).
* Against the FP64 SIMT kernel on the same inputs, and the argument checks.
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


def _inputs(n, N, Na, nH, seed, integer=False):
    rng = np.random.default_rng(seed)
    icol = rng.integers(-1, nH, size=(n, 4)).astype(np.int32)
    if integer:
        ival = rng.integers(-8, 9, size=(n, 4)).astype(np.float64)
        uH = rng.integers(-1000, 1001, size=(nH, N)).astype(np.float64)
        uhat = rng.integers(-1000, 1001, size=(n, Na)).astype(np.float64)
        alpha = rng.integers(-1000, 1001, size=(Na, N)).astype(np.float64)
    else:
        ival = rng.uniform(0.0, 1.0, size=(n, 4))
        uH = rng.standard_normal((nH, N))
        uhat = rng.standard_normal((n, Na)) * 10.0 ** rng.uniform(-9, 3, size=(n, 1))
        uhat[::17] = 0.0                                   # zero rows
        uhat[5::23, 0] = 1e-310                            # subnormal entries
        uhat[7::29] *= 10.0 ** rng.uniform(-12, 0, size=Na)  # wide range inside a row
        alpha = rng.standard_normal((Na, N)) * 10.0 ** rng.uniform(-6, 2, size=(1, N))
        if N > 2:
            alpha[:, 1] = 0.0                              # a zero column
    return icol, ival, np.vstack([uH, alpha]), uhat


def _reference(icol, ival, U, uhat, nH, absolute=False):
    n = icol.shape[0]
    if absolute:
        icol, ival, U, uhat = icol, np.abs(ival), np.abs(U), np.abs(uhat)
    iu = np.zeros((n, U.shape[1]))
    for q in range(4):
        a = icol[:, q]
        m = a >= 0
        iu[m] += ival[m, q:q + 1] * U[a[m]]
    return iu, uhat @ U[nH:]


def _run(nas, torch, tc, icol, ival, U, uhat, nH):
    dev = torch.device("cuda:0")
    n, Na = uhat.shape
    N = U.shape[1]
    t = [torch.tensor(a, device=dev) for a in (icol, ival, U, uhat)]
    psi = torch.full((n, N), 7.0, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream().cuda_stream
    nas.nas_reconstruct_f64(tc, n, t[0].data_ptr(), t[1].data_ptr(), N, t[2].data_ptr(), nH, Na, t[3].data_ptr(),
                            psi.data_ptr(), st)
    torch.cuda.synchronize()
    return psi.cpu().numpy()


@pytest.mark.parametrize("n,N,Na", [(1, 1, 1), (127, 5, 7), (128, 16, 16), (129, 21, 21), (1000, 33, 64),
                                    (5003, 64, 64), (2049, 48, 13), (640, 64, 1)])
def test_tensor_core_reconstruction_within_bound(env, n, N, Na):
    nas, torch = env
    nH = 97
    icol, ival, U, uhat = _inputs(n, N, Na, nH, seed=n + N + Na)
    iu, dense = _reference(icol, ival, U, uhat, nH)
    psi = _run(nas, torch, 1, icol, ival, U, uhat, nH)
    rowmax = np.max(np.abs(uhat), axis=1, keepdims=True)
    colmax = np.max(np.abs(U[nH:]), axis=0, keepdims=True)
    abs_iu, abs_dense = _reference(icol, ival, U, uhat, nH, absolute=True)
    bound = 2.0 ** -38 * rowmax * colmax + 1e-15 * (abs_iu + abs_dense) + 1e-300
    err = np.abs(psi - (iu + dense))
    assert np.all(err <= bound), (np.max(err / bound), n, N, Na)
    # zero rows of U^ (subnormals count as zero) leave the I u_H part alone
    assert np.all(np.abs(psi[::17] - iu[::17]) <= 1e-15 * abs_iu[::17] + 1e-300)
    simt = _run(nas, torch, 0, icol, ival, U, uhat, nH)
    assert np.all(np.abs(psi - simt) <= 2 * bound)


@pytest.mark.parametrize("n,N,Na", [(300, 64, 64), (77, 10, 3)])
def test_tensor_core_reconstruction_exact_on_integers(env, n, N, Na):
    nas, torch = env
    nH = 50
    icol, ival, U, uhat = _inputs(n, N, Na, nH, seed=7, integer=True)
    iu, dense = _reference(icol, ival, U, uhat, nH)
    exact = iu + dense      # every product and partial sum is an integer below 2^53
    assert np.array_equal(_run(nas, torch, 1, icol, ival, U, uhat, nH), exact)
    assert np.array_equal(_run(nas, torch, 0, icol, ival, U, uhat, nH), exact)


def test_tensor_core_reconstruction_rejects_wide_blocks(env):
    nas, torch = env
    dev = torch.device("cuda:0")
    n, nH = 8, 4
    icol = torch.zeros((n, 4), dtype=torch.int32, device=dev)
    ival = torch.zeros((n, 4), dtype=torch.float64, device=dev)
    for N, Na in ((65, 4), (4, 65)):
        U = torch.zeros((nH + Na, N), dtype=torch.float64, device=dev)
        uhat = torch.zeros((n, Na), dtype=torch.float64, device=dev)
        psi = torch.zeros((n, N), dtype=torch.float64, device=dev)
        with pytest.raises(nas.NasError):   # refused on the host, nothing launched
            nas.nas_reconstruct_f64(1, n, icol.data_ptr(), ival.data_ptr(), N, U.data_ptr(), nH, Na,
                                    uhat.data_ptr(), psi.data_ptr())
        nas.nas_reconstruct_f64(0, n, icol.data_ptr(), ival.data_ptr(), N, U.data_ptr(), nH, Na,
                                uhat.data_ptr(), psi.data_ptr())

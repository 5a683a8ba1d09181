"""Host eigensolver of the small augmented problem (csrc/small_eig.cpp) on
the CPU: the dense generalized solver, the Rayleigh-Ritz step of LOBPCG
(Cholesky fast path and the fallback that drops near-dependent directions),
the host LOBPCG on an arrow-structured pencil, the Cholesky inverse and the
small Anderson solve, against scipy.linalg on random and degenerate inputs.
The sources are compiled with g++ into a temporary shared library through a
small extern "C" shim (tests/host_eig_shim.cpp)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2404_19249_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("hosteig") / "libhosteig.so")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-fopenmp", "-I", CSRC,
                           os.path.join(HERE, "host_eig_shim.cpp"), os.path.join(CSRC, "small_eig.cpp"),
                           "-o", out])
    return C.CDLL(out)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def dense_gen_eig(lib, A, B, k):
    m = A.shape[0]
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lam = np.zeros(k)
    U = np.zeros((m, k))
    r = lib.shim_dense_gen_eig(C.c_int(m), _p(A), _p(B), C.c_int(k), _p(lam), _p(U))
    return r, lam, U


def _spd(rng, m, cond=10.0):
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    return (Q * np.geomspace(1.0, cond, m)) @ Q.T


def _check_pairs(A, B, lam, U, lam_ref, tol):
    scale = max(1.0, np.max(np.abs(lam_ref)))
    assert np.max(np.abs(lam - lam_ref)) < tol * scale
    k = U.shape[1]
    assert np.max(np.abs(U.T @ B @ U - np.eye(k))) < 1e-10
    assert np.max(np.abs(A @ U - (B @ U) * lam)) < 1e-9 * scale


@pytest.mark.parametrize("m,k", [(1, 1), (2, 1), (3, 2), (17, 5), (60, 20), (78, 26)])
def test_dense_generalized_random(lib, m, k):
    rng = np.random.default_rng(m)
    S = rng.standard_normal((m, m))
    A = S + S.T
    B = _spd(rng, m, 50.0)
    r, lam, U = dense_gen_eig(lib, A, B, k)
    assert r == 0
    _check_pairs(A, B, lam, U, sla.eigh(A, B, eigvals_only=True)[:k], 1e-12)


def test_dense_generalized_degenerate_clusters(lib):
    # eigenvalues with multiplicities 3, 2, 4 (as the degenerate orbitals of a
    # symmetric molecule): values, B-orthonormality and residuals
    rng = np.random.default_rng(7)
    m = 40
    w = np.concatenate([[-2.0] * 3, [-1.25] * 2, [-0.5] * 4, np.linspace(0.0, 5.0, m - 9)])
    B = _spd(rng, m, 20.0)
    L = np.linalg.cholesky(B)
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    A = L @ (Q * w) @ Q.T @ L.T
    A = 0.5 * (A + A.T)
    r, lam, U = dense_gen_eig(lib, A, B, 9)
    assert r == 0
    _check_pairs(A, B, lam, U, w[:9], 1e-12)


def test_dense_generalized_rejects_indefinite_B(lib):
    A = np.eye(3)
    B = np.diag([1.0, -1.0, 1.0])
    r, _, _ = dense_gen_eig(lib, A, B, 1)
    assert r != 0


def _rr(lib, G, H, k):
    ns = G.shape[0]
    G = np.ascontiguousarray(G)
    H = np.ascontiguousarray(H)
    Y = np.zeros((ns, k))
    th = np.zeros(k)
    r = lib.shim_rayleigh_ritz(C.c_int(ns), _p(G), _p(H), C.c_int(k), _p(Y), _p(th))
    return r, th, Y


@pytest.mark.parametrize("dependent", [False, True], ids=["cholesky_path", "dropping_path"])
def test_rayleigh_ritz_of_gram_matrices(lib, dependent):
    rng = np.random.default_rng(11)
    m, ns, k = 120, 30, 8
    A = rng.standard_normal((m, m))
    A = A + A.T
    B = _spd(rng, m, 10.0)
    S = rng.standard_normal((m, ns))
    if dependent:
        # two columns repeat others up to 1e-13: the basis Gram matrix is
        # numerically singular and the fallback must drop those directions
        S[:, 5] = S[:, 2] + 1e-13 * rng.standard_normal(m)
        S[:, 9] = 2.0 * S[:, 4]
    G, H = S.T @ B @ S, S.T @ A @ S
    r, th, Y = _rr(lib, G, H, k)
    assert r == 0
    # reference: Ritz values of the pencil on an orthonormal basis of span(S)
    Uo, sv, _ = np.linalg.svd(S, full_matrices=False)
    V = Uo[:, sv > 1e-8 * sv[0]]
    ref = sla.eigh(V.T @ A @ V, V.T @ B @ V, eigvals_only=True)[:k]
    assert np.max(np.abs(th - ref)) < 1e-8 * np.max(np.abs(ref))
    X = S @ Y
    assert np.max(np.abs(X.T @ B @ X - np.eye(k))) < 1e-8


def test_rayleigh_ritz_too_few_directions(lib):
    rng = np.random.default_rng(3)
    S = rng.standard_normal((20, 6))
    S[:, 3:] = S[:, :3]                    # rank 3
    G = S.T @ S
    r, _, _ = _rr(lib, G, G.copy(), 4)
    assert r != 0


def _arrow(rng, nH, Na, shift):
    # coarse block: a 1D Laplacian-like SPD band plus a random diagonal; dense border and corner
    main = 2.0 + rng.uniform(0.0, 1.0, nH)
    Ks = sp.diags([-np.ones(nH - 1), main, -np.ones(nH - 1)], [-1, 0, 1]).tocsr()
    Ms = sp.diags([0.1 * np.ones(nH - 1), np.ones(nH), 0.1 * np.ones(nH - 1)], [-1, 0, 1]).tocsr()
    Ks.sort_indices()
    Ms = sp.csr_matrix((Ms[Ks.nonzero()].A1, Ks.indices, Ks.indptr), shape=Ks.shape)
    bA = 0.05 * rng.standard_normal((nH, Na))
    cA = rng.standard_normal((Na, Na))
    cA = cA + cA.T + shift * np.eye(Na)
    bB = 0.01 * rng.standard_normal((nH, Na))
    cB = np.eye(Na) + 0.01 * np.ones((Na, Na))
    FA = np.block([[Ks.toarray(), bA], [bA.T, cA]])
    FB = np.block([[Ms.toarray(), bB], [bB.T, cB]])
    return Ks, Ms, bA, cA, bB, cB, FA, FB


def test_host_lobpcg_on_arrow_pencil(lib):
    rng = np.random.default_rng(5)
    nH, Na, nev = 400, 6, 6
    Ks, Ms, bA, cA, bB, cB, FA, FB = _arrow(rng, nH, Na, 4.0)
    ref = sla.eigh(FA, FB, eigvals_only=True)[:nev]
    lam = np.zeros(nev)
    U = np.zeros((nH + Na, nev))
    arr = [np.ascontiguousarray(x) for x in (Ks.indptr.astype(np.int32), Ks.indices.astype(np.int32), Ks.data,
                                            bA, cA, Ms.data, bB, cB)]
    it = lib.shim_lobpcg_arrow(C.c_int64(nH), C.c_int(Na), *[_p(a) for a in arr], C.c_int(nev), C.c_int(4),
                               _p(lam), _p(U), C.c_int(0), C.c_double(1e-10), C.c_int(2000))
    assert it > 0
    assert np.max(np.abs(lam - ref)) < 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(U.T @ FB @ U - np.eye(nev))) < 1e-9
    # warm restart from the solution converges at once
    it2 = lib.shim_lobpcg_arrow(C.c_int64(nH), C.c_int(Na), *[_p(a) for a in arr], C.c_int(nev), C.c_int(4),
                                _p(lam), _p(U), C.c_int(1), C.c_double(1e-9), C.c_int(2000))
    assert 0 <= it2 <= 2


def test_cholesky_inverse(lib):
    rng = np.random.default_rng(2)
    m = 150
    A = _spd(rng, m, 1e4)
    F = np.ascontiguousarray(A.copy())
    Inv = np.zeros((m, m))
    assert lib.shim_chol_inverse(C.c_int(m), _p(F), _p(Inv)) == 0
    assert np.max(np.abs(Inv @ A - np.eye(m))) < 1e-8
    bad = np.ascontiguousarray(-np.eye(4))
    assert lib.shim_chol_inverse(C.c_int(4), _p(bad), _p(np.zeros((4, 4)))) != 0


def test_small_solve(lib):
    rng = np.random.default_rng(9)
    for n in range(1, 9):
        A = rng.standard_normal((n, n)) + n * np.eye(n)
        b = rng.standard_normal(n)
        x = np.zeros(n)
        assert lib.shim_small_solve(C.c_int(n), _p(np.ascontiguousarray(A)), _p(b), _p(x)) == 0
        np.testing.assert_allclose(A @ x, b, atol=1e-12)
    sing = np.zeros((3, 3))
    assert lib.shim_small_solve(C.c_int(3), _p(sing), _p(np.ones(3)), _p(np.zeros(3))) != 0

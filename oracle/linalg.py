"""Linear-algebra helpers of the oracle (test infrastructure).

solve_spd solves a sparse symmetric positive definite system exactly by a
sparse LU factorisation when it is small enough, and otherwise by Jacobi
preconditioned CG to a relative residual `tol` (the definition being the
exact solution, CG is only used where a factorisation does not fit).
"""
import numpy as np
import scipy.sparse.linalg as spla

DIRECT_MAX = 60000


def solve_spd(A, B, tol=1e-13, x0=None, direct_max=DIRECT_MAX):
    B = np.asarray(B, dtype=np.float64)
    one = B.ndim == 1
    Bm = B[:, None] if one else B
    n = A.shape[0]
    if n <= direct_max:
        lu = spla.splu(A.tocsc())
        X = lu.solve(Bm)
    else:
        d = A.diagonal()
        Pre = spla.LinearOperator(A.shape, matvec=lambda v: v / d)
        X = np.empty_like(Bm)
        for c in range(Bm.shape[1]):
            g = None if x0 is None else (x0 if one else x0[:, c])
            x, info = spla.cg(A, Bm[:, c], x0=g, rtol=tol, atol=0.0, M=Pre, maxiter=100000)
            if info != 0:
                raise RuntimeError("CG did not converge")
            X[:, c] = x
    return X[:, 0] if one else X

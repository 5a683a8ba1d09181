"""Anderson density mixing (oracle; test infrastructure).

Sec. 4 of the paper (Anderson mixing).  With F^(j) = rho_out^(j) - rho_in^(j)
and the history j = m0..m (depth = m - m0 + 1):
  rho~_in(out) = rho_in(out)^(m) + sum_{j<m} alpha_j (rho_in(out)^(j) - rho_in(out)^(m))
  sum_k (F^m - F^j, F^m - F^k) alpha_k = (F^m - F^j, F^m),  j = m0..m-1
  rho_in^(m+1) = beta rho~_out + (1 - beta) rho~_in.
Defaults depth = 5, beta = 0.7 (as in the experiments).

Readings: the inner product is the quadrature-weighted L2 product (the same
one as the ||.||_0 stopping test); with no history the step is linear mixing
rho_in + beta F; when the (depth-1)^2 system has condition number above 1e12
the oldest entry is dropped until it is not.
"""
import numpy as np


class Anderson:
    def __init__(self, weights, depth=5, beta=0.7, cond_max=1e12):
        self.w = np.asarray(weights).ravel()
        self.depth = depth
        self.beta = beta
        self.cond_max = cond_max
        self.hist = []  # list of (rho_in, F)

    def dot(self, f, g):
        return float(np.sum(self.w * f.ravel() * g.ravel()))

    def mix(self, rho_in, rho_out):
        F = rho_out - rho_in
        self.hist.append((rho_in.copy(), F.copy()))
        if len(self.hist) > self.depth:
            self.hist.pop(0)
        while True:
            prev = self.hist[:-1]
            if not prev:
                return rho_in + self.beta * F
            Fm = F
            dF = [Fm - Fj for (_, Fj) in prev]
            k = len(prev)
            Amat = np.empty((k, k))
            rhs = np.empty(k)
            for a in range(k):
                rhs[a] = self.dot(dF[a], Fm)
                for b in range(k):
                    Amat[a, b] = self.dot(dF[a], dF[b])
            if np.linalg.cond(Amat) > self.cond_max:
                self.hist.pop(0)
                continue
            alpha = np.linalg.solve(Amat, rhs)
            rin_t = rho_in.copy()
            F_t = F.copy()
            for a, (rj, Fj) in enumerate(prev):
                rin_t = rin_t + alpha[a] * (rj - rho_in)
                F_t = F_t + alpha[a] * (Fj - Fm)
            return rin_t + self.beta * F_t

"""Quadrature rules on the reference tetrahedron (oracle; test infrastructure).

The paper (Sec. 2, finite element discretisation) does not fix a rule; these
are the readings used on both sides:
  P1 fine space : symmetric 4-point rule, exact for degree 2 (mass matrix exact)
  P2 fine space : symmetric 14-point rule, exact for degree 5 (mass matrix,
                  degree 4, exact; stiffness, degree 2, exact).

Points are given in barycentric coordinates (L0, L1, L2, L3) of the reference
tetrahedron with vertices (0,0,0), (1,0,0), (0,1,0), (0,0,1) (volume 1/6), and
the weights sum to 1/6.

The 14-point rule has three orbits: (a,a,a,1-3a) x4, (b,b,b,1-3b) x4 and
(c,c,1/2-c,1/2-c) x6.  Its six parameters are obtained here by Newton's method
on the moment equations (exact integrals of all monomials of degree <= 5,
int x^i y^j z^k = i! j! k! / (i+j+k+3)!), so the rule follows from its
definition rather than from a table.
"""
import itertools
from math import factorial, sqrt

import numpy as np


def exact_monomial(i, j, k):
    """Exact integral of x^i y^j z^k over the reference tetrahedron."""
    return factorial(i) * factorial(j) * factorial(k) / factorial(i + j + k + 3)


def _orbit_points(a, b, c):
    pts = []
    for t in (a, b):
        for k in range(4):
            l = [t] * 4
            l[k] = 1.0 - 3.0 * t
            pts.append(l)
    for (i, j) in itertools.combinations(range(4), 2):
        l = [0.5 - c] * 4
        l[i] = c
        l[j] = c
        pts.append(l)
    return np.array(pts)


def _monomials(deg):
    return [(i, j, k) for i in range(deg + 1) for j in range(deg + 1) for k in range(deg + 1)
            if i + j + k <= deg]


def _residual(v, mons):
    a, b, c, w1, w2, w3 = v
    P = _orbit_points(a, b, c)
    W = np.array([w1] * 4 + [w2] * 4 + [w3] * 6)
    return np.array([np.sum(W * P[:, 1] ** i * P[:, 2] ** j * P[:, 3] ** k) - exact_monomial(i, j, k)
                     for (i, j, k) in mons])


def _solve_rule14():
    mons = _monomials(5)
    v = np.array([0.09, 0.31, 0.045, 0.012, 0.019, 0.007])
    for _ in range(50):
        r = _residual(v, mons)
        J = np.empty((len(mons), 6))
        for p in range(6):
            h = 1e-7 * max(1.0, abs(v[p]))
            vp = v.copy()
            vp[p] += h
            vm = v.copy()
            vm[p] -= h
            J[:, p] = (_residual(vp, mons) - _residual(vm, mons)) / (2 * h)
        dv = np.linalg.lstsq(J, -r, rcond=None)[0]
        v = v + dv
        if np.max(np.abs(dv)) < 1e-17:
            break
    if np.max(np.abs(_residual(v, mons))) > 1e-15:
        raise RuntimeError("14-point rule did not converge")
    return v


def rule(order):
    """Return (bary [nq, 4], weights [nq]) for the given fine-space order."""
    if order == 1:
        a = (5.0 + 3.0 * sqrt(5.0)) / 20.0
        b = (5.0 - sqrt(5.0)) / 20.0
        bary = np.full((4, 4), b)
        for k in range(4):
            bary[k, k] = a
        return bary, np.full(4, 1.0 / 24.0)
    if order == 2:
        a, b, c, w1, w2, w3 = _RULE14
        bary = _orbit_points(a, b, c)
        return bary, np.array([w1] * 4 + [w2] * 4 + [w3] * 6)
    raise ValueError("order must be 1 or 2")


_RULE14 = _solve_rule14()

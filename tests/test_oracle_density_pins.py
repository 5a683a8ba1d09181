"""Pins of the oracle's density and of its quadrupole boundary values.

The density rho = sum_i f_i psi_i^2 (Algorithm 3's density update, with the
square and the occupations of Sec. 4's closed-shell runs) is checked against

  * the electron count: for M-orthonormal orbitals int rho = sum_i f_i
    exactly, because the quadrature integrates products of two basis
    functions exactly (degree 2 for P1, 4 for P2);
  * a closed form: nodal interpolants of the hydrogen 1s function
    e^(-r)/sqrt(pi) about two centres, with unequal occupations, converge to
    sum_i f_i e^(-2 r_i)/pi under refinement.  A dropped square, a dropped or
    permuted occupation fails one of the two.

The optional quadrupole term of the Hartree boundary values (Sec. 3.1,
the multipole expansion about the charge centre, with the textbook
factor 1/2) is checked against a pair of off-centre Gaussian charges, whose
moments and exterior potential sum_k q_k erf(sqrt(a_k) r_k)/r_k are known in
closed form.
"""
from math import erf, pi, sqrt

import numpy as np
import pytest

from oracle import fem, hartree
from oracle.nas import Problem
from workloads import make_instance


def _m_orthonormal(P, X):
    G = X.T @ (P.M @ X)
    L = np.linalg.cholesky(0.5 * (G + G.T))
    return np.linalg.solve(L, X.T).T


@pytest.mark.parametrize("order", [1, 2])
def test_density_integrates_to_occupation_sum(order):
    inst = make_instance("he_p1", cells=6, coarse_cells=3)
    inst.order = order
    inst.occ = np.array([2.0, 2.0, 1.0, 0.5])
    P = Problem(inst, with_transfer=False)
    X = np.random.default_rng(7).standard_normal((P.fine.n, 4))
    Psi = _m_orthonormal(P, X)
    rho = P.density(Psi)
    assert np.all(rho >= 0.0)
    assert abs(P.fine.integrate(rho) - 5.5) < 1e-12
    # each orbital alone carries its own occupation
    for i, f in enumerate(inst.occ):
        sub = Problem.__new__(Problem)
        sub.fine, sub.occ = P.fine, np.eye(4)[i] * f
        assert abs(P.fine.integrate(sub.density(Psi)) - f) < 1e-12


@pytest.mark.parametrize("kw,n_el", [
    (dict(name="he_p1", cells=6, coarse_cells=3), 2.0),
    (dict(name="paper_molecule", molecule="c6h6", cells=6, coarse_cells=4), 42.0),
])
def test_density_of_oracle_states_counts_electrons(kw, n_el):
    kw = dict(kw)
    inst = make_instance(kw.pop("name"), **kw)
    inst.tol_bvp = inst.tol_poisson = 1e-12
    inst.max_inner = 30
    P = Problem(inst)
    st0 = P.initial_state()
    st1 = P.step(st0)
    # Ritz vectors of the small pencil of Sec. 3.3 are F_B-orthonormal, i.e. M-orthonormal in S_h
    for st in (st0, st1):
        assert abs(P.fine.integrate(st.rho_out) - n_el) < 1e-10 * n_el
        G = st.Psi.T @ (P.M @ st.Psi)
        assert np.max(np.abs(G - np.eye(P.N))) < 1e-10


def _hydrogenic_error(cells):
    inst = make_instance("hydrogen", cells=cells, order=2, half=10.0, power=2.0)
    inst.occ = np.array([2.0, 1.0])
    P = Problem(inst, with_transfer=False)
    f = P.fine
    a = np.array([1.0, 0.5, -0.5])
    x = f.node_xyz[f.interior_nodes]
    Psi = np.stack([np.exp(-np.linalg.norm(x, axis=1)),
                    np.exp(-np.linalg.norm(x - a, axis=1))], axis=1) / sqrt(pi)
    rho = P.density(Psi)
    exact = (2.0 * np.exp(-2.0 * np.linalg.norm(f.xq, axis=-1))
             + np.exp(-2.0 * np.linalg.norm(f.xq - a, axis=-1))) / pi
    return float(np.sqrt(f.integrate((rho - exact) ** 2))), f.integrate(rho)


def test_density_hydrogenic_closed_form():
    e8, _ = _hydrogenic_error(8)
    e16, total = _hydrogenic_error(16)
    # P2 interpolation of the cusped 1s functions: L2 error falls ~6x per halving
    assert e16 < 0.25 * e8 and e16 < 1e-2
    # int (2 e^(-2r)/pi + e^(-2r')/pi) over R^3 = 3 (box truncation < 1e-6)
    assert abs(total - 3.0) < 5e-3


def _gaussian_pair():
    qs = [1.0, 0.5]
    cs = [np.array([0.6, 0.3, -0.4]), np.array([-0.9, -0.2, 0.5])]
    al = [3.0, 2.0]
    return qs, cs, al


def test_quadrupole_boundary_values_closed_form():
    inst = make_instance("he_p1", cells=16, coarse_cells=2)
    s = fem.Space(inst.fine_xyz, inst.fine_tet, 2)
    qs, cs, al = _gaussian_pair()
    rho = sum(q * (a / pi) ** 1.5 * np.exp(-a * np.sum((s.xq - c) ** 2, axis=-1))
              for q, c, a in zip(qs, cs, al))
    w0, Q0, c0 = hartree.boundary_values(s, rho, 0)
    w2, Q, ctr = hartree.boundary_values(s, rho, 2)
    # exact moments of the pair: charge, centre, second moments about the centre
    Qa = sum(qs)
    xa = sum(q * c for q, c in zip(qs, cs)) / Qa
    qa = sum(q * (np.outer(c - xa, c - xa) + np.eye(3) / (2.0 * a)) for q, c, a in zip(qs, cs, al))
    assert abs(Q - Qa) < 1e-4 and np.max(np.abs(ctr - xa)) < 1e-4
    assert Q0 == Q and np.array_equal(c0, ctr)
    xb = s.node_xyz[s.boundary_nodes]
    d = xb - xa
    r = np.linalg.norm(d, axis=1)
    # monopole + quadrupole with exact moments: Q/r + (1/2) q_ij (3 d_i d_j - delta_ij r^2)/r^5
    textbook = Qa / r + 0.5 * (3.0 * np.einsum("ij,bi,bj->b", qa, d, d) - np.trace(qa) * r * r) / r ** 5
    assert np.max(np.abs(w2 - textbook)) < 1e-5
    # against the exact exterior potential: the quadrupole removes >90 % of the
    # monopole truncation error (what is left is the octupole, O(a^3/r^4))
    V = np.zeros(len(xb))
    for q, c, a in zip(qs, cs, al):
        rk = np.linalg.norm(xb - c, axis=1)
        V += q * np.array([erf(sqrt(a) * x) for x in rk]) / rk
    e0 = np.max(np.abs(w0 - V))
    e2 = np.max(np.abs(w2 - V))
    assert e0 > 5e-4
    assert e2 < 0.1 * e0

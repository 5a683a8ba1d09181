"""Hartree potential by a Poisson solve with multipole boundary values (oracle).

Sec. 3.1 of the paper:  -Laplace V_Har = 4 pi rho in Omega,  V_Har = w_D on the
boundary, with w_D from a multipole expansion about the charge centre
x'' = int x rho / int rho.  Readings:
  * monopole (default): w_D(x) = Q / |x - x''|, Q = int rho.  The dipole term
    vanishes identically because x'' is the charge centre.
  * multipole=2 adds the quadrupole term with the textbook factor 1/2,
    (1/2) sum_ij q_ij (3 d_i d_j - delta_ij |d|^2) / |d|^5, d = x - x''
    (the printed formula lacks the 1/2).
  * rho is known at quadrature points; the weak form is
    int grad V . grad phi_i = 4 pi int rho phi_i for every interior node i,
    with the boundary nodes fixed to w_D (V_Har is a function of the fine
    space, boundary included).
"""
import numpy as np

from .linalg import solve_spd


def boundary_values(space, rho_q, multipole=0):
    """Return (w_B at boundary nodes, Q, x'')."""
    Q = space.integrate(rho_q)
    xb = space.node_xyz[space.boundary_nodes]
    if Q == 0.0:
        return np.zeros(len(xb)), 0.0, np.zeros(3)
    centre = np.array([space.integrate(rho_q * space.xq[:, :, d]) for d in range(3)]) / Q
    dvec = xb - centre
    r = np.linalg.norm(dvec, axis=1)
    w = Q / r
    if multipole >= 2:
        q = np.empty((3, 3))
        for i in range(3):
            for j in range(3):
                q[i, j] = space.integrate(rho_q * (space.xq[:, :, i] - centre[i])
                                          * (space.xq[:, :, j] - centre[j]))
        quad = np.zeros(len(xb))
        for i in range(3):
            for j in range(3):
                quad += q[i, j] * (3.0 * dvec[:, i] * dvec[:, j] - (i == j) * r ** 2)
        w = w + 0.5 * quad / r ** 5
    return w, Q, centre


def hartree(space, K_II, K_IB, rho_q, tol=1e-13, multipole=0, x0=None):
    """Nodal V_Har over all fine nodes (boundary values included)."""
    wB, Q, centre = boundary_values(space, rho_q, multipole)
    b = 4.0 * np.pi * space.load_vector(rho_q)[space.interior_nodes] - K_IB @ wB
    vI = solve_spd(K_II, b, tol=tol, x0=x0)
    V = np.zeros(space.nnode)
    V[space.interior_nodes] = vI
    V[space.boundary_nodes] = wB
    return V

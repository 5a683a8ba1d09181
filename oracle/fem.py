"""P1/P2 Lagrange finite elements on tetrahedra (oracle; test infrastructure).

Follows the discretisation of the paper's Sec. 2 (a conforming space S_h of
continuous piecewise polynomials on a tetrahedral mesh, zero Dirichlet values
on the boundary of the box) and the matrices of Sec. 3.3:
  K_ij   = int grad(phi_i) . grad(phi_j)          (kinetic part of A_h^L is K/2)
  M_ij   = int phi_i phi_j                        (mass)
  M_V,ij = int V phi_i phi_j                      (potential parts of A_h^L, A_h^NL)
all integrated element by element with the rule of `oracle.quadrature`.

Node numbering of the fine space:
  P1: the mesh vertices.
  P2: the vertices, then one node per edge at its midpoint, edges ordered by
      their (smaller, larger) vertex id.  Local element nodes are the 4
      vertices followed by the edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3).
A node is a boundary node if it lies on a face of the bounding box of the
vertices (exact comparison); the remaining nodes, in increasing node id,
are the degrees of freedom 0..n-1.
"""
import numpy as np
import scipy.sparse as sp

from . import quadrature

LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]

# gradient of the barycentric coordinates L0..L3 with respect to the reference
# coordinates (xi, eta, zeta); L0 = 1 - xi - eta - zeta, Lk = k-th coordinate.
_DL = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def basis_values(order, bary):
    """phi_a at barycentric points: [nq, nloc]."""
    L = np.asarray(bary)
    if order == 1:
        return L.copy()
    vals = [L[:, i] * (2.0 * L[:, i] - 1.0) for i in range(4)]
    vals += [4.0 * L[:, i] * L[:, j] for (i, j) in LOCAL_EDGES]
    return np.stack(vals, axis=1)


def basis_ref_gradients(order, bary):
    """d phi_a / d(xi, eta, zeta) at barycentric points: [nq, nloc, 3]."""
    L = np.asarray(bary)
    nq = L.shape[0]
    if order == 1:
        return np.broadcast_to(_DL, (nq, 4, 3)).copy()
    g = [(4.0 * L[:, i] - 1.0)[:, None] * _DL[i][None, :] for i in range(4)]
    g += [4.0 * (L[:, j][:, None] * _DL[i][None, :] + L[:, i][:, None] * _DL[j][None, :])
          for (i, j) in LOCAL_EDGES]
    return np.stack(g, axis=1)


class Space:
    """A Lagrange space of order 1 or 2 on a tetrahedral mesh."""

    def __init__(self, xyz, tet, order):
        self.order = int(order)
        self.vxyz = np.asarray(xyz, dtype=np.float64)
        self.tet = np.asarray(tet, dtype=np.int64)
        self.nv = self.vxyz.shape[0]
        self.ne = self.tet.shape[0]
        if self.order == 1:
            self.elem = self.tet.copy()
            self.node_xyz = self.vxyz.copy()
        elif self.order == 2:
            pairs = np.stack([np.sort(self.tet[:, [i, j]], axis=1) for (i, j) in LOCAL_EDGES], axis=1)
            keys = pairs[:, :, 0] * self.nv + pairs[:, :, 1]
            ukeys, inv = np.unique(keys.ravel(), return_inverse=True)
            self.edges = np.stack([ukeys // self.nv, ukeys % self.nv], axis=1)
            self.elem = np.concatenate([self.tet, self.nv + inv.reshape(self.ne, 6)], axis=1)
            mid = 0.5 * (self.vxyz[self.edges[:, 0]] + self.vxyz[self.edges[:, 1]])
            self.node_xyz = np.concatenate([self.vxyz, mid], axis=0)
        else:
            raise ValueError("order must be 1 or 2")
        self.nnode = self.node_xyz.shape[0]
        self.nloc = self.elem.shape[1]
        lo = self.vxyz.min(axis=0)
        hi = self.vxyz.max(axis=0)
        self.box_lo, self.box_hi = lo, hi
        on_b = np.any((self.node_xyz == lo) | (self.node_xyz == hi), axis=1)
        self.boundary = on_b
        self.interior_nodes = np.nonzero(~on_b)[0]
        self.boundary_nodes = np.nonzero(on_b)[0]
        self.n = self.interior_nodes.size
        self.dof_of_node = np.full(self.nnode, -1, dtype=np.int64)
        self.dof_of_node[self.interior_nodes] = np.arange(self.n)

        # geometry: x = v0 + J xi, J columns v1-v0, v2-v0, v3-v0
        v = self.vxyz[self.tet]
        self.J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
        self.detJ = np.linalg.det(self.J)
        if np.any(self.detJ <= 0):
            raise ValueError("mesh has non-positively oriented tetrahedra")
        self.JinvT = np.transpose(np.linalg.inv(self.J), (0, 2, 1))

        self.qbary, self.qw = quadrature.rule(self.order)
        self.nq = self.qw.size
        self.phi = basis_values(self.order, self.qbary)              # [nq, nloc]
        self.dphi_ref = basis_ref_gradients(self.order, self.qbary)  # [nq, nloc, 3]
        # physical quadrature points and weights
        self.xq = np.einsum("qk,ekd->eqd", self.qbary, v)              # [ne, nq, 3]
        self.Wq = self.qw[None, :] * self.detJ[:, None]                # [ne, nq]

    # ---------------------------------------------------------------- element matrices
    def grad_phi(self, elems=None):
        """Physical basis gradients [ne, nq, nloc, 3]."""
        JinvT = self.JinvT if elems is None else self.JinvT[elems]
        return np.einsum("eij,qaj->eqai", JinvT, self.dphi_ref)

    def local_stiffness(self, elems=None):
        G = self.grad_phi(elems)
        W = self.Wq if elems is None else self.Wq[elems]
        return np.einsum("eq,eqai,eqbi->eab", W, G, G)

    def local_mass(self, coef=None, elems=None):
        """sum_q W_eq c_eq phi_a(q) phi_b(q); coef [ne, nq] or None for c = 1."""
        W = self.Wq if elems is None else self.Wq[elems]
        c = W if coef is None else W * coef
        return np.einsum("eq,qa,qb->eab", c, self.phi, self.phi)

    # ---------------------------------------------------------------- global assembly
    def _global(self, local, elems=None):
        el = self.elem if elems is None else self.elem[elems]
        rows = np.repeat(el[:, :, None], self.nloc, axis=2).ravel()
        cols = np.repeat(el[:, None, :], self.nloc, axis=1).ravel()
        return sp.csr_matrix((local.ravel(), (rows, cols)), shape=(self.nnode, self.nnode))

    def assemble_full(self, kind, coef=None, elems=None):
        """Matrix over all nodes (boundary included): kind 'K' or 'M'."""
        if kind == "K":
            loc = self.local_stiffness(elems)
        elif kind == "M":
            loc = self.local_mass(coef, elems)
        else:
            raise ValueError(kind)
        return self._global(loc, elems)

    def interior(self, A_full):
        """Restriction to interior rows and columns (the Dirichlet space S_h)."""
        I = self.interior_nodes
        return A_full[I][:, I].tocsr()

    def interior_boundary(self, A_full):
        return A_full[self.interior_nodes][:, self.boundary_nodes].tocsr()

    # ---------------------------------------------------------------- functions
    def to_nodes(self, u_dof):
        """Interior DOF vector(s) [n] or [n, N] -> nodal values with zero boundary."""
        u = np.asarray(u_dof)
        out = np.zeros((self.nnode,) + u.shape[1:])
        out[self.interior_nodes] = u
        return out

    def at_quad(self, u_nodal):
        """Nodal values [nnode] or [nnode, N] -> values at quadrature points [ne, nq(, N)]."""
        u = np.asarray(u_nodal)
        ue = u[self.elem]  # [ne, nloc(, N)]
        if u.ndim == 1:
            return np.einsum("qa,ea->eq", self.phi, ue)
        return np.einsum("qa,ean->eqn", self.phi, ue)

    def integrate(self, f_q):
        """int f for f given at quadrature points [ne, nq]."""
        return float(np.sum(self.Wq * f_q))

    def load_vector(self, f_q):
        """b_i = int f phi_i over all nodes, f at quadrature points."""
        loc = np.einsum("eq,qa->ea", self.Wq * f_q, self.phi)
        return np.bincount(self.elem.ravel(), weights=loc.ravel(), minlength=self.nnode)

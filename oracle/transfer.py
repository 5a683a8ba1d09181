"""Nonnested transfer I_H^h (oracle; test infrastructure).

Follows the paper's Sec. 3.2, Algorithm 1 (fast interpolation between two
nonnested meshes): an octree over the coarse vertices (at most 2^d = 8 per
leaf), the nearest coarse vertex to the fine point inside its leaf, a coarse
tetrahedron having that vertex, then a walk through face neighbours until all
barycentric coordinates of the point are non-negative; the fine value is the
barycentric combination of the coarse vertex values.  I_H^h is that linear map
written as a matrix (I_H^h of Sec. 3.3): row = interior fine node, columns = interior
coarse nodes (the coarse space S_H vanishes on the boundary), weights = the
barycentric coordinates.

Readings where Algorithm 1 is silent or garbled (it says "quadtree" and
"triangle" in 3-D, breaks ties at random, and loops on strictly positive
coordinates, which never ends for points on faces):
  * the walk leaves through the face with the most negative coordinate
    (lowest local index on ties);
  * "inside" means inside the closed tetrahedron: all four orientation signs
    >= 0, decided exactly (floating filter, then exact rational arithmetic);
  * the result is canonical: the smallest element id among ALL closed coarse
    tetrahedra containing the point (the walk's answer, then every
    tetrahedron of its vertex stars is tested);
  * a barycentric weight whose exact sign is 0 is stored as exactly 0;
    the other weights are D_k / D in floating point, with D_k the
    orientation determinant of the tetrahedron with vertex k replaced by
    the point and D that of the tetrahedron.
"""
from fractions import Fraction

import numpy as np
import scipy.sparse as sp

_EPS = np.finfo(np.float64).eps / 2.0  # unit roundoff 2^-53
_ERRBOUND = 16.0 * _EPS


def orient_float(a, b, c, d):
    """det[b-a, c-a, d-a] in floating point plus an error bound (vectorised)."""
    ba = b - a
    ca = c - a
    da = d - a
    m1 = ca[..., 1] * da[..., 2] - ca[..., 2] * da[..., 1]
    m2 = ca[..., 0] * da[..., 2] - ca[..., 2] * da[..., 0]
    m3 = ca[..., 0] * da[..., 1] - ca[..., 1] * da[..., 0]
    det = ba[..., 0] * m1 - ba[..., 1] * m2 + ba[..., 2] * m3
    aba = np.abs(ba)
    aca = np.abs(ca)
    ada = np.abs(da)
    perm = (aba[..., 0] * (aca[..., 1] * ada[..., 2] + aca[..., 2] * ada[..., 1])
            + aba[..., 1] * (aca[..., 0] * ada[..., 2] + aca[..., 2] * ada[..., 0])
            + aba[..., 2] * (aca[..., 0] * ada[..., 1] + aca[..., 1] * ada[..., 0]))
    return det, _ERRBOUND * perm


def orient_exact_sign(a, b, c, d):
    """Exact sign of det[b-a, c-a, d-a] for double inputs (rational arithmetic)."""
    A = [Fraction(float(x)) for x in a]
    Bv = [Fraction(float(x)) - A[i] for i, x in enumerate(b)]
    Cv = [Fraction(float(x)) - A[i] for i, x in enumerate(c)]
    Dv = [Fraction(float(x)) - A[i] for i, x in enumerate(d)]
    det = (Bv[0] * (Cv[1] * Dv[2] - Cv[2] * Dv[1])
           - Bv[1] * (Cv[0] * Dv[2] - Cv[2] * Dv[0])
           + Bv[2] * (Cv[0] * Dv[1] - Cv[1] * Dv[0]))
    return (det > 0) - (det < 0)


def orient_sign(a, b, c, d):
    det, err = orient_float(np.asarray(a), np.asarray(b), np.asarray(c), np.asarray(d))
    if det > err:
        return 1
    if det < -err:
        return -1
    return orient_exact_sign(a, b, c, d)


def bary_signs(p, V):
    """Exact signs and float values of D_k (vertex k of tet V [4,3] replaced by p)."""
    W = np.repeat(np.asarray(V, dtype=np.float64)[None], 4, axis=0)
    W[np.arange(4), np.arange(4)] = p
    det, err = orient_float(W[:, 0], W[:, 1], W[:, 2], W[:, 3])
    signs = np.where(det > err, 1, np.where(det < -err, -1, 0))
    for k in np.nonzero(signs == 0)[0]:
        signs[k] = orient_exact_sign(W[k, 0], W[k, 1], W[k, 2], W[k, 3])
    vals = np.where(signs == 0, 0.0, det)
    return signs, vals


def contains(p, V):
    s, _ = bary_signs(p, V)
    return bool(np.all(s >= 0))


class Octree:
    """Octree over points, at most `leaf` points per terminal cell (Algorithm 1 data)."""

    def __init__(self, pts, leaf=8):
        self.pts = np.asarray(pts)
        self.leaf = leaf
        lo = self.pts.min(axis=0)
        hi = self.pts.max(axis=0)
        self.root = self._build(np.arange(len(self.pts)), lo, hi, 0)

    def _build(self, idx, lo, hi, depth):
        node = {"lo": lo, "hi": hi, "idx": idx, "kids": None}
        if len(idx) <= self.leaf or depth > 40:
            return node
        mid = 0.5 * (lo + hi)
        P = self.pts[idx]
        kids = []
        for o in range(8):
            bits = [(o >> d) & 1 for d in range(3)]
            sel = np.ones(len(idx), dtype=bool)
            clo = lo.copy()
            chi = hi.copy()
            for d in range(3):
                if bits[d]:
                    sel &= P[:, d] >= mid[d]
                    clo[d] = mid[d]
                else:
                    sel &= P[:, d] < mid[d]
                    chi[d] = mid[d]
            kids.append(self._build(idx[sel], clo, chi, depth + 1))
        node["kids"] = kids
        return node

    def nearest_in_leaf(self, q):
        """Nearest point to q among the points of the terminal cell containing q
        (the parent cell when that cell is empty)."""
        path = [self.root]
        node = self.root
        while node["kids"] is not None:
            mid = 0.5 * (node["lo"] + node["hi"])
            o = sum((1 << d) for d in range(3) if q[d] >= mid[d])
            node = node["kids"][o]
            path.append(node)
        for node in reversed(path):
            if len(node["idx"]) > 0:
                P = self.pts[node["idx"]]
                dist = np.sum((P - q) ** 2, axis=1)
                return int(node["idx"][np.argmin(dist)])
        raise RuntimeError("empty octree")


class CoarseMesh:
    """Coarse mesh adjacency used by the walk."""

    def __init__(self, xyz, tet):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tet = np.asarray(tet, dtype=np.int64)
        nv = self.xyz.shape[0]
        # vertex -> incident tets (sorted ids)
        order = np.argsort(self.tet.ravel(), kind="stable")
        verts = self.tet.ravel()[order]
        self.vstar_ptr = np.searchsorted(verts, np.arange(nv + 1))
        self.vstar = order // 4
        # face -> tets
        self.face_nbr = -np.ones((len(self.tet), 4), dtype=np.int64)
        faces = {}
        for t, T in enumerate(self.tet):
            for k in range(4):
                key = tuple(sorted(int(T[j]) for j in range(4) if j != k))
                faces.setdefault(key, []).append((t, k))
        for lst in faces.values():
            if len(lst) == 2:
                (t0, k0), (t1, k1) = lst
                self.face_nbr[t0, k0] = t1
                self.face_nbr[t1, k1] = t0
        self.octree = Octree(self.xyz)

    def star(self, v):
        return self.vstar[self.vstar_ptr[v]:self.vstar_ptr[v + 1]]

    def brute_force(self, p):
        """Smallest id of a closed tetrahedron containing p (all tets tested).

        Tetrahedra that a certain (filtered) negative sign excludes are
        skipped; every other one is decided exactly, in ascending id order.
        """
        V = self.xyz[self.tet]                       # [nt, 4, 3]
        maybe = np.ones(len(self.tet), dtype=bool)
        for k in range(4):
            W = V.copy()
            W[:, k] = p
            det, err = orient_float(W[:, 0], W[:, 1], W[:, 2], W[:, 3])
            maybe &= ~(det < -err)
        for t in np.nonzero(maybe)[0]:
            if contains(p, V[t]):
                return int(t)
        return -1

    def locate(self, p, max_steps=100000):
        """Algorithm 1 walk followed by the canonical smallest-id rule."""
        v = self.octree.nearest_in_leaf(p)
        t = int(self.star(v).min())
        found = -1
        for _ in range(max_steps):
            s, vals = bary_signs(p, self.xyz[self.tet[t]])
            if np.all(s >= 0):
                found = t
                break
            neg = np.nonzero(s < 0)[0]
            k = int(neg[np.argmin(vals[neg])])
            nt = self.face_nbr[t, k]
            if nt < 0:
                break
            t = int(nt)
        if found < 0:
            return self.brute_force(p)
        if np.all(s > 0):   # strictly inside: no other tetrahedron contains p
            return found
        cand = np.unique(np.concatenate([self.star(int(u)) for u in self.tet[found]]))
        for c in cand:  # ascending ids
            if contains(p, self.xyz[self.tet[c]]):
                return int(c)
        return found


def weights(p, V):
    """Barycentric weights of p in tet V with exact zeros (see module doc)."""
    s, vals = bary_signs(p, V)
    D, _ = orient_float(V[0], V[1], V[2], V[3])
    w = np.where(s == 0, 0.0, vals / D)
    return w


def build_transfer(fine_space, coarse_space, points=None):
    """I_H^h as CSR [n_fine_interior, n_coarse_interior] plus the element ids.

    `points`: optional subset of fine interior DOF indices (rows returned in
    that order); default all interior fine nodes.
    Returns (I csr, elem_ids int64 [rows], W [rows,4] weights, C [rows,4]
    coarse node ids of the containing tet).
    """
    cm = CoarseMesh(coarse_space.vxyz, coarse_space.tet)
    rows = np.arange(fine_space.n) if points is None else np.asarray(points)
    P = fine_space.node_xyz[fine_space.interior_nodes[rows]]
    elem = np.empty(len(rows), dtype=np.int64)
    W = np.empty((len(rows), 4))
    for r, p in enumerate(P):
        t = cm.locate(p)
        if t < 0:
            raise RuntimeError("fine node outside the coarse mesh")
        elem[r] = t
        W[r] = weights(p, cm.xyz[cm.tet[t]])
    C = cm.tet[elem]
    cdof = coarse_space.dof_of_node[C]
    keep = cdof >= 0
    ri = np.repeat(np.arange(len(rows)), 4)[keep.ravel()]
    I = sp.csr_matrix((W.ravel()[keep.ravel()], (ri, cdof.ravel()[keep.ravel()])),
                      shape=(len(rows), coarse_space.n))
    return I, elem, W, C

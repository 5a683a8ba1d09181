"""Tensor-grid tetrahedral meshes for the synthetic workloads.

A mesh is a tensor grid of hexahedra whose node coordinates along each axis
are given as a strictly increasing 1-D array.  Every hexahedron is split into
the 6 Kuhn (Freudenthal) tetrahedra that share its main diagonal; neighbouring
hexahedra then match face to face, so the result is a conforming mesh.

Output format (the one the library and the oracle both read):
  xyz : float64 [n_vert, 3]
  tet : int32   [n_tet, 4], every tetrahedron positively oriented
        (det[v1-v0, v2-v0, v3-v0] > 0).
Orientation follows from the combinatorics of the split (the parity of the
axis permutation), not from a floating-point determinant.
"""
import itertools

import numpy as np

# The 6 axis permutations; a Kuhn tet walks from corner (0,0,0) to (1,1,1)
# adding one unit step per axis in the permutation's order.
_PERMS = list(itertools.permutations(range(3)))


def _parity(p):
    inv = sum(1 for i in range(3) for j in range(i + 1, 3) if p[i] > p[j])
    return inv % 2


def uniform_axis(lo, hi, n):
    """n cells of equal width on [lo, hi] (n+1 nodes, end points exact)."""
    x = np.linspace(lo, hi, n + 1)
    x[0], x[-1] = lo, hi
    return x


def graded_axis_power(half_width, n, power):
    """Nodes x = L*sign(s)*|s|**power for s uniform on [-1, 1] (n cells).

    With power > 1 the nodes cluster around 0.  Used for the helium workload
    (L = 10, power = 1.5, 20 cells).
    """
    s = np.linspace(-1.0, 1.0, n + 1)
    x = half_width * np.sign(s) * np.abs(s) ** power
    x[0], x[-1] = -half_width, half_width
    if n % 2 == 0:
        x[n // 2] = 0.0
    return x


def graded_axis_lorentz(lo, hi, n, centres, amplitude=8.0, width=0.5):
    """Nodes equidistributing the density g(x) = 1 + sum_k A/(1+((x-c_k)/w)^2).

    The node x_i solves G(x_i) = (i/n) G(hi) with G the primitive of g from
    lo; G is strictly increasing, so plain bisection (60 halvings) gives the
    nodes to full double precision.  Used for the molecule workloads, with
    c_k the nuclear coordinates along the axis.
    """
    c = np.asarray(centres, dtype=np.float64).reshape(-1)

    def G(x):
        x = np.asarray(x, dtype=np.float64)
        v = x - lo
        for ck in c:
            v = v + amplitude * width * (np.arctan((x - ck) / width) - np.arctan((lo - ck) / width))
        return v

    total = G(np.array(hi))
    targets = total * np.arange(n + 1) / n
    a = np.full(n + 1, lo, dtype=np.float64)
    b = np.full(n + 1, hi, dtype=np.float64)
    for _ in range(80):
        m = 0.5 * (a + b)
        left = G(m) < targets
        a = np.where(left, m, a)
        b = np.where(left, b, m)
    x = 0.5 * (a + b)
    x[0], x[-1] = lo, hi
    if np.any(np.diff(x) <= 0):
        raise ValueError("graded axis is not strictly increasing")
    return x


def kuhn_mesh(xs, ys, zs):
    """Kuhn-split tensor mesh on the grid xs x ys x zs.

    Vertex (i, j, k) has id i + nx1*(j + ny1*k) with nx1 = len(xs) etc.
    Returns (xyz float64 [nv,3], tet int32 [6*nx*ny*nz, 4]).
    """
    xs = np.asarray(xs, dtype=np.float64)
    ys = np.asarray(ys, dtype=np.float64)
    zs = np.asarray(zs, dtype=np.float64)
    nx1, ny1, nz1 = len(xs), len(ys), len(zs)
    nx, ny, nz = nx1 - 1, ny1 - 1, nz1 - 1
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    # id = i + nx1*(j + ny1*k) -> Fortran order over (i, j, k)
    xyz = np.stack([X.ravel(order="F"), Y.ravel(order="F"), Z.ravel(order="F")], axis=1)

    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    I, J, K = I.ravel(order="F"), J.ravel(order="F"), K.ravel(order="F")

    def vid(di, dj, dk):
        return (I + di) + nx1 * ((J + dj) + ny1 * (K + dk))

    tets = []
    for p in _PERMS:
        step = [0, 0, 0]
        verts = [vid(0, 0, 0)]
        for ax in p:
            step[ax] += 1
            verts.append(vid(*step))
        v = np.stack(verts, axis=1)
        if _parity(p) == 1:  # odd permutation: swap the last two to make it positive
            v = v[:, [0, 1, 3, 2]]
        tets.append(v)
    # interleave so that the 6 tets of one hexahedron are consecutive
    tet = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return xyz, tet

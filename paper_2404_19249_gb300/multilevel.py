"""Moving-mesh multilevel loop (Algorithm 2) on tensor-product meshes.

Algorithm 2 solves the Kohn-Sham problem on a sequence of meshes: after each
solve the mesh is moved toward the features of sqrt(rho), the orbitals are
interpolated onto the new mesh, and the next level starts from them, until
the relative energy change falls below a tolerance or the level cap is hit.
The paper moves unstructured meshes with a Hessian metric (remeshing tools
outside this library); here the meshes are Kuhn-split tensor grids and the
move is an r-adaptation per axis: the nodes of each axis are redistributed so
that they equidistribute the monitor

    g(x) = 1 + alpha * F(x) / max F,   F(x_i) = sum over the other two axes of
                                       sqrt(rho) at the vertices of the plane x = x_i,

which keeps the number of cells and the box and concentrates nodes where the
density (and so the orbitals' curvature) is large.  Every level is solved
with Algorithm 3 (nas_solve) from the interpolated orbitals (the paper's
first K_asm levels use a plain SCF instead; Algorithm 3 reaches the same
discrete ground state and needs no separate solver).

The interpolation between two non-nested meshes evaluates the old P1/P2
finite element functions at the new nodes: a point of a tensor cell with
local coordinates t lies in the Kuhn tetrahedron of the permutation that
sorts t decreasingly, with barycentric coordinates 1 - t_p0, t_p0 - t_p1,
t_p1 - t_p2, t_p2.

Host-side orchestration only: the solves run in libnas.so.
"""
import dataclasses

import numpy as np

from . import nas

# local vertex pairs of the 6 edges of a tetrahedron
_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def tensor_axes(xyz):
    """The three coordinate axes of a tensor-grid vertex set (sorted unique values)."""
    axes = [np.unique(xyz[:, d]) for d in range(3)]
    if np.prod([len(a) for a in axes]) != len(xyz):
        raise ValueError("the fine mesh is not a tensor grid")
    return axes


def fe_nodes(xyz, tet, order):
    """Node coordinates of the library's P1/P2 space (vertices, then the unique
    edges sorted by (min, max) vertex id, at their midpoints), the edge keys
    (min * n_vert + max, sorted) and the dof list (nodes off the bounding box,
    increasing node id)."""
    nv = len(xyz)
    if order == 2:
        t = tet.astype(np.int64)
        pairs = np.concatenate([np.sort(t[:, [i, j]], axis=1) for i, j in _EDGES])
        keys = np.unique(pairs[:, 0] * nv + pairs[:, 1])
        a, b = keys // nv, keys % nv
        nodes = np.concatenate([xyz, 0.5 * (xyz[a] + xyz[b])])
    else:
        keys = np.zeros(0, dtype=np.int64)
        nodes = xyz
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    on_b = np.any((nodes == lo) | (nodes == hi), axis=1)
    return nodes, keys, np.nonzero(~on_b)[0]


def interpolate(axes, order, nodal, edge_keys, pts):
    """Values at pts [n, 3] of the finite element function with node values
    `nodal` [n_node, ...] on the Kuhn mesh of `axes` (vertex id i + nx1 (j +
    ny1 k)); points outside the box are clamped onto it."""
    xs, ys, zs = axes
    nx1, ny1 = len(xs), len(ys)
    nv = nx1 * ny1 * len(zs)
    cell, loc = [], []
    for d, ax in enumerate(axes):
        p = np.clip(pts[:, d], ax[0], ax[-1])
        c = np.clip(np.searchsorted(ax, p, side="right") - 1, 0, len(ax) - 2)
        cell.append(c)
        loc.append(np.clip((p - ax[c]) / (ax[c + 1] - ax[c]), 0.0, 1.0))
    t = np.stack(loc, axis=1)                          # [n, 3]
    perm = np.argsort(-t, axis=1, kind="stable")       # axes by decreasing local coordinate
    ts = np.take_along_axis(t, perm, axis=1)
    lam = np.stack([1.0 - ts[:, 0], ts[:, 0] - ts[:, 1], ts[:, 1] - ts[:, 2], ts[:, 2]], axis=1)
    # vertices of the Kuhn tetrahedron: corner, then one unit step per axis in perm order
    step = np.zeros((len(pts), 3), dtype=np.int64)
    verts = []
    base = np.stack(cell, axis=1).astype(np.int64)
    for q in range(4):
        if q > 0:
            np.put_along_axis(step, perm[:, q - 1:q], 1, axis=1)
        ijk = base + step
        verts.append(ijk[:, 0] + nx1 * (ijk[:, 1] + ny1 * ijk[:, 2]))
    verts = np.stack(verts, axis=1)                    # [n, 4]
    extra = (1,) * (nodal.ndim - 1)
    if order == 1:
        return sum(lam[:, q].reshape(-1, *extra) * nodal[verts[:, q]] for q in range(4))
    out = sum((lam[:, q] * (2.0 * lam[:, q] - 1.0)).reshape(-1, *extra) * nodal[verts[:, q]] for q in range(4))
    for a, b in _EDGES:
        va, vb = verts[:, a], verts[:, b]
        key = np.minimum(va, vb) * nv + np.maximum(va, vb)
        e = nv + np.searchsorted(edge_keys, key)
        out = out + (4.0 * lam[:, a] * lam[:, b]).reshape(-1, *extra) * nodal[e]
    return out


def adapt_axes(axes, rho_vertex, alpha=8.0):
    """New axes (same cell counts, same end points) equidistributing the
    monitor 1 + alpha F / max F per axis, F the sum of sqrt(rho) over the
    orthogonal vertex planes.  rho_vertex: [nx1, ny1, nz1]."""
    root = np.sqrt(np.maximum(rho_vertex, 0.0))
    new = []
    for d, ax in enumerate(axes):
        F = root.sum(axis=tuple(k for k in range(3) if k != d))
        g = 1.0 + alpha * F / max(F.max(), 1e-300)
        G = np.concatenate([[0.0], np.cumsum(0.5 * (g[1:] + g[:-1]) * np.diff(ax))])
        targets = G[-1] * np.arange(len(ax)) / (len(ax) - 1)
        x = np.interp(targets, G, ax)
        x[0], x[-1] = ax[0], ax[-1]
        if np.any(np.diff(x) <= 0):
            raise ValueError("adapted axis is not strictly increasing")
        new.append(x)
    return new


def moving_mesh_solve(inst, levels=4, tol_energy=1e-6, alpha=8.0, make_mesh=None, **options):
    """Algorithm 2 on tensor meshes: returns (history, solver of the last level).

    inst: an instance whose fine mesh is a Kuhn tensor grid (its coarse mesh
    and system are kept on every level); make_mesh(xs, ys, zs) -> (xyz, tet)
    builds a fine mesh from axes (default: the Kuhn split of workloads.mesh);
    options: nas_options fields for every level's solver.
    """
    if make_mesh is None:
        from workloads.mesh import kuhn_mesh as make_mesh
    axes = tensor_axes(inst.fine_xyz)
    occ = np.asarray(inst.occ, dtype=np.float64)
    history, psi0, solver = [], None, None
    for level in range(levels):
        xyz, tet = (inst.fine_xyz, inst.fine_tet) if level == 0 else make_mesh(*axes)
        lv = dataclasses.replace(inst, fine_xyz=xyz, fine_tet=tet)
        if solver is not None:
            solver.close()
        solver = nas.Solver(lv, **options)
        solver.init(psi0)
        r, rep = nas.nas_solve(solver.h)
        E = float(solver.get(nas.NAS_Q_ENERGY)[0])
        history.append({"level": level, "energy": E, "steps": int(rep.step), "drho": float(rep.drho),
                        "status": int(r), "unknowns": int(solver.sizes()["n"]),
                        "min_cell": float(min(np.diff(a).min() for a in axes)),
                        "axes": [a.copy() for a in axes]})
        if level > 0 and abs(E - history[-2]["energy"]) <= tol_energy * abs(E):
            break
        if level == levels - 1:
            break
        # orbitals at every node (zero on the boundary), density at the vertices
        nodes, keys, dofs = fe_nodes(xyz, tet, inst.order)
        psi = solver.get(nas.NAS_Q_ORBITALS)
        nodal = np.zeros((len(nodes), psi.shape[1]))
        nodal[dofs] = psi
        nv = len(xyz)
        rho_v = (nodal[:nv] ** 2 @ occ).reshape(len(axes[2]), len(axes[1]), len(axes[0])).transpose(2, 1, 0)
        new_axes = adapt_axes(axes, rho_v, alpha)
        nxyz, ntet = make_mesh(*new_axes)
        nnodes, _, ndofs = fe_nodes(nxyz, ntet, inst.order)
        psi0 = np.ascontiguousarray(interpolate(axes, inst.order, nodal, keys, nnodes[ndofs]))
        axes = new_axes
    return history, solver

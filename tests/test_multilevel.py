"""Moving-mesh multilevel loop (Algorithm 2) on tensor meshes: the host-side
interpolation between non-nested meshes and the axis r-adaptation (CPU), and
a short multilevel solve through the library (GPU)."""
import numpy as np
import pytest

from paper_2404_19249_gb300.multilevel import adapt_axes, fe_nodes, interpolate, moving_mesh_solve, tensor_axes
from workloads.mesh import graded_axis_lorentz, kuhn_mesh, uniform_axis


def _mesh():
    xs = graded_axis_lorentz(-3.0, 3.0, 5, [0.4])
    ys = uniform_axis(-2.0, 2.0, 4)
    zs = graded_axis_lorentz(-1.0, 2.0, 3, [0.1, 1.0])
    return [xs, ys, zs], kuhn_mesh(xs, ys, zs)


@pytest.mark.parametrize("order", [1, 2])
def test_interpolation_reproduces_polynomials(order):
    """P1 interpolation is exact for affine functions and P2 for quadratics,
    at arbitrary points of a graded tensor mesh (cells located through the
    Kuhn split by sorting the local coordinates)."""
    axes, (xyz, tet) = _mesh()
    assert all(np.array_equal(a, b) for a, b in zip(tensor_axes(xyz), axes))
    nodes, keys, _ = fe_nodes(xyz, tet, order)
    rng = np.random.default_rng(5)
    pts = np.stack([rng.uniform(a[0], a[-1], 400) for a in axes], axis=1)
    pts[:20] = xyz[rng.integers(0, len(xyz), 20)]          # exactly on vertices
    if order == 1:
        f = lambda p: 1.5 - 2.0 * p[:, 0] + 0.25 * p[:, 1] + 3.0 * p[:, 2]
    else:
        f = lambda p: (0.3 + p[:, 0] * p[:, 1] - 2.0 * p[:, 2] ** 2 + 0.5 * p[:, 0] ** 2
                       + p[:, 1] * p[:, 2] - p[:, 0])
    vals = np.stack([f(nodes), 2.0 * f(nodes)], axis=1)
    out = interpolate(axes, order, vals, keys, pts)
    ref = np.stack([f(pts), 2.0 * f(pts)], axis=1)
    assert np.max(np.abs(out - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_fe_nodes_dof_order():
    """Dofs are the nodes off the bounding box, in increasing node id; P2 edge
    nodes are the midpoints of the unique edges sorted by (min, max) vertex."""
    axes, (xyz, tet) = _mesh()
    nodes, keys, dofs = fe_nodes(xyz, tet, 2)
    nv = len(xyz)
    assert np.all(np.diff(keys) > 0) and len(nodes) == nv + len(keys)
    a, b = keys // nv, keys % nv
    assert np.allclose(nodes[nv:], 0.5 * (xyz[a] + xyz[b]))
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    inside = ~np.any((nodes == lo) | (nodes == hi), axis=1)
    assert np.array_equal(dofs, np.nonzero(inside)[0])


def test_axis_adaptation_equidistributes_the_monitor():
    ax = uniform_axis(-5.0, 5.0, 20)
    axes = [ax, ax, ax]
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    rho = np.exp(-2.0 * np.sqrt((X - 1.5) ** 2 + Y ** 2 + (Z + 2.0) ** 2)) / np.pi
    new = adapt_axes(axes, rho, alpha=8.0)
    for d, centre in enumerate((1.5, 0.0, -2.0)):
        x = new[d]
        assert x[0] == -5.0 and x[-1] == 5.0 and np.all(np.diff(x) > 0) and len(x) == len(ax)
        widths = np.diff(x)
        mids = 0.5 * (x[1:] + x[:-1])
        assert abs(mids[np.argmin(widths)] - centre) < 1.0       # finest cells at the density peak
        assert widths.max() / widths.min() > 2.0


@pytest.mark.gpu
def test_moving_mesh_levels_through_the_library():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19249_gb300 import nas
    from workloads import make_instance
    inst = make_instance("he_p1", cells=8, coarse_cells=3, tol_scf=1e-9, mu=2.0, max_outer=400)
    hist, solver = moving_mesh_solve(inst, levels=3, tol_energy=0.0, alpha=8.0, tol_bvp=1e-12, tol_poisson=1e-12)
    assert len(hist) == 3
    for h in hist:
        assert h["status"] == 0 and np.isfinite(h["energy"]) and h["drho"] < 1e-9
    # the library numbers the dofs of the last mesh as fe_nodes does
    xyz, tet = kuhn_mesh(*hist[-1]["axes"])
    _, _, dofs = fe_nodes(xyz, tet, inst.order)
    assert np.array_equal(solver.get(nas.NAS_Q_DOF_NODE), dofs)
    # levels after the first start from interpolated orbitals
    assert hist[1]["steps"] <= hist[0]["steps"] and hist[2]["steps"] <= hist[0]["steps"]
    # the adapted meshes refine around the nucleus
    assert hist[2]["min_cell"] < hist[0]["min_cell"]
    solver.close()


@pytest.mark.gpu
def test_moving_mesh_levels_match_oracle_direct_scf():
    """Every level of the moving-mesh loop converges to the discrete ground
    state of that level's mesh: the oracle's direct SCF on the whole fine
    space (the plain definition) on the same adapted axes gives the same
    eigenvalue and energy, at 1e-10 relative."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import dataclasses
    from oracle.nas import Problem
    from paper_2404_19249_gb300 import nas
    from workloads import make_instance
    inst = make_instance("he_p1", cells=8, coarse_cells=3, tol_scf=1e-12, mu=2.0, max_outer=600)
    hist, solver = moving_mesh_solve(inst, levels=3, tol_energy=0.0, alpha=8.0, tol_bvp=1e-14, tol_poisson=1e-14)
    solver.close()
    assert len(hist) == 3
    for h in hist:
        assert h["status"] == 0 and h["drho"] < 1e-11
        xyz, tet = kuhn_mesh(*h["axes"])
        lv = dataclasses.replace(inst, fine_xyz=xyz, fine_tet=tet, tol_bvp=1e-14, tol_poisson=1e-14)
        P = Problem(lv, with_transfer=False)
        d = P.direct_scf(tol=1e-12)
        assert d.inner_converged
        E = P.energy(d)
        assert abs(h["energy"] - E) < 1e-10 * abs(E), (h["level"], h["energy"], E)

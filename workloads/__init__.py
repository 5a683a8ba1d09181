"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only *generates inputs*: tensor-grid tetrahedral meshes (graded
node placement, Kuhn 6-tet split of every hexahedron), seeded random
molecules, and the workload recipes built from them.  It holds none of the
method's arithmetic (no finite elements, no quadrature, no potentials, no
solvers), so both the CPU oracle and the GPU library can consume what it
produces without sharing any computation.
"""
from .mesh import kuhn_mesh, graded_axis_power, graded_axis_lorentz, uniform_axis
from .molecules import random_molecule
from .configs import Instance, make_instance, WORKLOADS

__all__ = [
    "kuhn_mesh", "graded_axis_power", "graded_axis_lorentz", "uniform_axis",
    "random_molecule", "Instance", "make_instance", "WORKLOADS",
]

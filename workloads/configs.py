"""Workload recipes: meshes + molecules + run parameters, all seeded.

Every recipe returns an :class:`Instance`.  Sizes follow the workloads the
method is measured on:

  he_p1            helium atom, Z=2 at the origin, one doubly occupied orbital,
                   P1 on a 20^3 hexahedral grid of [-10,10]^3 split 6 tets/hex,
                   nodes graded toward the nucleus by x = 10 sign(s)|s|^1.5,
                   nonnested coarse mesh 8^3 uniform.  (9261 vertices.)
  mol8_p2          8 nuclei, Z uniform in {1..8}, R uniform in [-4,4]^3 with
                   >= 1.2 bohr separation (seed 1), N = ceil(sum Z / 2) closed
                   shell orbitals, P2 on a 50^3 grid of [-16,16]^3 graded toward
                   the nuclei, coarse 16^3 P1.  (~1.03M P2 nodes.)
  mol32_p2         32 nuclei, Z in {1..6}, R in [-8,8]^3 (seed 2), N = 64, P2 on
                   100^3 (~8.1M nodes), coarse 16^3; Fermi-Dirac occupations at
                   kT = 0.01 Ha (the random system has a dense spectrum at the
                   Fermi level, where integer occupations make the SCF swap
                   orbitals from one iteration to the next) and Anderson mixing
                   with a 16-entry history and beta = 0.5 (with the paper's
                   depth 5 and beta 0.7 the density residual of this 32-atom
                   system stalls at ~1e-3: long-wavelength charge oscillations;
                   measured on a 75^3 mesh, inner iterations to 1e-8: 50+ at
                   depth 5 / beta 0.1, 36 at depth 16 / beta 0.5).
  The two random molecules use mu = max_k Z_k^2: twice the magnitude of the
  hydrogen-like bound -Z^2/2 on the lowest level, so H + mu is coercive with
  margin.  (The paper's 8 M sum Z^2, 1.7e4 and 2.5e4 here, makes each step's
  correction O(1/mu) and the outer iteration crawl: measured on mol8_p2, the
  energy still falls by ~1 Ha per step after 30 steps, against convergence
  toward -290 Ha with mu = 50.)
  smooth4_p1       4 nuclei, Z in {1..3}, R in [-3,3]^3 (seed 3), smoothed
                   Coulomb -Z/sqrt(r^2+0.1^2), P1 on 62^3 (250,047 vertices).
  harmonic / hydrogen
                   linear test problems (no Hartree, no exchange-correlation).

The `cells` / `coarse_cells` overrides shrink a workload while keeping its
molecule, grading and parameters; the parity tests use such reduced copies.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .mesh import kuhn_mesh, graded_axis_power, graded_axis_lorentz, uniform_axis
from .molecules import random_molecule

POT_COULOMB = 0
POT_SMOOTHED = 1
POT_HARMONIC = 2


@dataclass
class Instance:
    name: str
    order: int                    # fine-space polynomial order (1 or 2)
    fine_xyz: np.ndarray          # float64 [nv, 3]
    fine_tet: np.ndarray          # int32 [ne, 4]
    coarse_xyz: np.ndarray
    coarse_tet: np.ndarray
    R: np.ndarray                 # float64 [M, 3] nuclear positions
    Z: np.ndarray                 # float64 [M] nuclear charges
    occ: np.ndarray               # float64 [N] occupation numbers
    potential: int = POT_COULOMB
    smooth_a: float = 0.0         # smoothing length of the smoothed Coulomb potential
    omega: float = 1.0            # harmonic test potential 0.5*omega^2*|x|^2
    hartree: bool = True          # include the Hartree potential
    xc: bool = True               # include LDA exchange-correlation
    mu: Optional[float] = None    # None -> the paper's 8*M*sum(Z^2)
    tol_scf: float = 1e-8
    tol_bvp: float = 1e-12
    tol_poisson: float = 1e-12
    max_outer: int = 100
    max_inner: int = 50
    smearing: float = 0.0         # Fermi-Dirac kT (Ha); 0: the occupations in `occ`
    anderson_depth: int = 5       # Anderson mixing history (Sec. 4: 5)
    anderson_beta: float = 0.7    # Anderson damping (Sec. 4: 0.7)
    anderson_restart: float = 0.0 # > 0: clear the history when the residual exceeds this x the best
    extra: dict = field(default_factory=dict)

    @property
    def n_orb(self):
        return len(self.occ)


def closed_shell_occupations(n_electrons, n_orb=None):
    """2 electrons per orbital, the last one singly occupied for an odd count.

    With n_orb larger than needed, the extra orbitals get occupation 0.
    """
    n_el = int(round(n_electrons))
    n_need = (n_el + 1) // 2
    n_orb = n_need if n_orb is None else n_orb
    if n_orb < n_need:
        raise ValueError("too few orbitals for the electron count")
    occ = np.zeros(n_orb)
    occ[: n_el // 2] = 2.0
    if n_el % 2:
        occ[n_el // 2] = 1.0
    return occ


def _he_p1(cells=20, coarse_cells=8, **kw):
    ax = graded_axis_power(10.0, cells, 1.5)
    fxyz, ftet = kuhn_mesh(ax, ax, ax)
    cax = uniform_axis(-10.0, 10.0, coarse_cells)
    cxyz, ctet = kuhn_mesh(cax, cax, cax)
    inst = Instance("he_p1", 1, fxyz, ftet, cxyz, ctet,
                    R=np.zeros((1, 3)), Z=np.array([2.0]), occ=np.array([2.0]),
                    tol_scf=1e-8)
    return inst


def _molecule_instance(name, seed, n_nuc, z_max, box_half, half, cells, coarse_cells,
                       order, n_orb=None, potential=POT_COULOMB, smooth_a=0.0):
    rng = np.random.default_rng(seed)
    while True:
        R, Z = random_molecule(rng, n_nuc, z_max, box_half)
        n_el = int(Z.sum())
        if n_orb is None or (n_el + 1) // 2 <= n_orb:
            break
    occ = closed_shell_occupations(n_el, n_orb)
    axes = [graded_axis_lorentz(-half, half, cells, R[:, d]) for d in range(3)]
    fxyz, ftet = kuhn_mesh(*axes)
    cax = uniform_axis(-half, half, coarse_cells)
    cxyz, ctet = kuhn_mesh(cax, cax, cax)
    return Instance(name, order, fxyz, ftet, cxyz, ctet, R=R, Z=Z, occ=occ,
                    potential=potential, smooth_a=smooth_a)


def _mol8_p2(cells=50, coarse_cells=16, order=2, seed=1, **kw):
    inst = _molecule_instance("mol8_p2", seed, 8, 8, 4.0, 16.0, cells, coarse_cells, order)
    inst.mu = float(np.max(inst.Z)) ** 2
    return inst


def _mol32_p2(cells=100, coarse_cells=16, order=2, **kw):
    inst = _molecule_instance("mol32_p2", 2, 32, 6, 8.0, 16.0, cells, coarse_cells, order,
                              n_orb=64)
    inst.mu = float(np.max(inst.Z)) ** 2
    inst.smearing = 0.01
    inst.anderson_beta = 0.5
    inst.anderson_depth = 16
    return inst


def _smooth4_p1(cells=62, coarse_cells=8, order=1, **kw):
    return _molecule_instance("smooth4_p1", 3, 4, 3, 3.0, 10.0, cells, coarse_cells, order,
                              potential=POT_SMOOTHED, smooth_a=0.1)


def _harmonic(cells=8, coarse_cells=4, order=1, half=6.0, n_orb=1, omega=1.0, **kw):
    ax = uniform_axis(-half, half, cells)
    fxyz, ftet = kuhn_mesh(ax, ax, ax)
    cax = uniform_axis(-half, half, coarse_cells)
    cxyz, ctet = kuhn_mesh(cax, cax, cax)
    return Instance("harmonic", order, fxyz, ftet, cxyz, ctet,
                    R=np.zeros((0, 3)), Z=np.zeros(0), occ=np.full(n_orb, 2.0),
                    potential=POT_HARMONIC, omega=omega, hartree=False, xc=False, mu=10.0)


def _hydrogen(cells=16, coarse_cells=4, order=1, half=12.0, power=2.0, **kw):
    ax = graded_axis_power(half, cells, power)
    fxyz, ftet = kuhn_mesh(ax, ax, ax)
    cax = uniform_axis(-half, half, coarse_cells)
    cxyz, ctet = kuhn_mesh(cax, cax, cax)
    return Instance("hydrogen", order, fxyz, ftet, cxyz, ctet,
                    R=np.zeros((1, 3)), Z=np.array([1.0]), occ=np.array([1.0]),
                    hartree=False, xc=False)


# Molecules of the paper's experiments (Sec. 4.2-4.4), coordinates as printed.  The
# LiH and CH4 tables are in bohr (Li-H 3.015, C-H 2.268); the benzene table is
# in angstrom (C-C 1.397, C-H 1.084) and is converted to bohr.
ANGSTROM = 1.0 / 0.529177210903
PAPER_MOLECULES = {
    "lih": ([[-1.0075, 0.0, 0.0], [2.0075, 0.0, 0.0]], [3.0, 1.0], 1.0),
    "ch4": ([[0.0, 0.0, 0.0], [1.3092, 1.3092, 1.3092], [-1.3092, -1.3092, 1.3092],
             [1.3092, -1.3092, -1.3092], [-1.3092, 1.3092, -1.3092]], [6.0, 1.0, 1.0, 1.0, 1.0], 1.0),
    "c6h6": ([[0.0, 1.3970, 0.0], [1.2098, 0.6985, 0.0], [1.2098, -0.6985, 0.0], [0.0, -1.3970, 0.0],
              [-1.2098, -0.6985, 0.0], [-1.2098, 0.6985, 0.0], [0.0, 2.4810, 0.0], [2.1486, 1.2405, 0.0],
              [2.1486, -1.2405, 0.0], [0.0, -2.4810, 0.0], [-2.1486, -1.2405, 0.0], [-2.1486, 1.2405, 0.0]],
             [6.0] * 6 + [1.0] * 6, ANGSTROM),
}


def _paper_molecule(molecule="ch4", cells=24, coarse_cells=8, order=2, **kw):
    R, Z, unit = PAPER_MOLECULES[molecule]
    R = np.asarray(R, dtype=np.float64) * unit
    Z = np.asarray(Z, dtype=np.float64)
    axes = [graded_axis_lorentz(-10.0, 10.0, cells, R[:, d]) for d in range(3)]
    fxyz, ftet = kuhn_mesh(*axes)
    cax = uniform_axis(-10.0, 10.0, coarse_cells)
    cxyz, ctet = kuhn_mesh(cax, cax, cax)
    return Instance("paper_" + molecule, order, fxyz, ftet, cxyz, ctet, R=R, Z=Z,
                    occ=closed_shell_occupations(Z.sum()))


def batch_instances(count=64, seed=4, dof_lo=1e4, dof_hi=4e5, max_orb=8):
    """The batched workload: `count` independent small molecules.

    Each instance: 1-6 nuclei with Z uniform in {1..4} and positions uniform in
    [-3,3]^3 (>= 1.2 bohr apart), redrawn until N = ceil(sum Z / 2) <= max_orb;
    fine order P1 or P2 by a fair coin; the number of fine unknowns log-uniform
    in [dof_lo, dof_hi] (rounded to a whole number of cells per axis);
    Omega = [-10,10]^3 with a mild grading toward the nuclei (amplitude 2,
    width 1 bohr) and a uniform coarse mesh of about a quarter (P1) or half
    (P2) the cells per axis, at least 3.  mu is the paper's 8 M sum Z^2.
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        while True:
            n_nuc = int(rng.integers(1, 7))
            R, Z = random_molecule(rng, n_nuc, 4, 3.0)
            if (int(Z.sum()) + 1) // 2 <= max_orb:
                break
        order = int(rng.integers(1, 3))
        side = float(np.exp(rng.uniform(np.log(dof_lo), np.log(dof_hi)))) ** (1.0 / 3.0)
        if order == 1:
            cells = max(6, int(round(side + 1.0)))
            coarse = max(3, cells // 4)
        else:
            cells = max(4, int(round((side + 1.0) / 2.0)))
            coarse = max(3, cells // 2)
        axes = [graded_axis_lorentz(-10.0, 10.0, cells, R[:, d], amplitude=2.0, width=1.0) for d in range(3)]
        fxyz, ftet = kuhn_mesh(*axes)
        cax = uniform_axis(-10.0, 10.0, coarse)
        cxyz, ctet = kuhn_mesh(cax, cax, cax)
        out.append(Instance("batch%d" % b, order, fxyz, ftet, cxyz, ctet, R=R, Z=Z,
                            occ=closed_shell_occupations(Z.sum())))
    return out


WORKLOADS = {
    "paper_molecule": _paper_molecule,
    "he_p1": _he_p1,
    "mol8_p2": _mol8_p2,
    "mol32_p2": _mol32_p2,
    "smooth4_p1": _smooth4_p1,
    "harmonic": _harmonic,
    "hydrogen": _hydrogen,
}


def make_instance(name, **overrides):
    """Build a workload by name; keyword overrides change sizes or run parameters.

    Size keywords (cells, coarse_cells, order, ...) go to the recipe; any
    keyword that names an Instance field (tol_scf, mu, max_inner, ...) is set
    on the result afterwards.
    """
    recipe = WORKLOADS[name]
    fields = set(Instance.__dataclass_fields__)
    size_kw = {k: v for k, v in overrides.items() if k not in fields}
    inst = recipe(**size_kw)
    for k, v in overrides.items():
        if k in fields:
            setattr(inst, k, v)
    return inst

"""Seeded random molecules (nuclear charges and positions)."""
import numpy as np


def random_molecule(rng, n_nuc, z_max, box_half, min_sep=1.2, z_min=1, max_tries=100000):
    """Charges uniform in {z_min..z_max}, positions uniform in [-box_half, box_half]^3.

    Positions are drawn one at a time and rejected until every pair is at
    least `min_sep` bohr apart.  Returns (R float64 [M,3], Z float64 [M]).
    """
    Z = rng.integers(z_min, z_max + 1, size=n_nuc).astype(np.float64)
    R = np.zeros((n_nuc, 3))
    placed = 0
    tries = 0
    while placed < n_nuc:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place nuclei with the requested separation")
        p = rng.uniform(-box_half, box_half, size=3)
        if placed == 0 or np.min(np.linalg.norm(R[:placed] - p, axis=1)) >= min_sep:
            R[placed] = p
            placed += 1
    return R, Z

"""Pins of the oracle's Fermi-Dirac occupations (option `smearing`).

For independent spin-degenerate levels lambda_i at temperature kT and Fermi
level eF, the grand potential is Omega = -2 kT sum_i ln(1 + exp(-(lambda_i - eF)/kT)).
Statistical mechanics fixes, independently of the oracle's formulas:
  * f_i = dOmega/dlambda_i (at fixed eF, kT)      - the occupations;
  * S = -dOmega/dT                                  - the entropy;
  * sum_i f_i lambda_i - kT S = Omega + eF n_el     - the free energy;
  * kT -> 0 with a gap at the Fermi level gives the Aufbau occupations.
A wrong sign, a dropped spin factor 2 or a mis-scaled entropy fails one of
these.  Algorithm 3 with smearing converges to the direct fine-space SCF with
the same smearing (the plain definition).
"""
import numpy as np
import pytest

from oracle.nas import Problem, fermi_dirac
from workloads import make_instance


def _omega(lam, eF, kT):
    return -2.0 * kT * float(np.sum(np.log1p(np.exp(-(lam - eF) / kT))))


def _fermi_level(lam, f, kT):
    i = int(np.argmin(np.abs(f - 1.0)))          # a level with 0 < f < 2
    return lam[i] - kT * np.log(2.0 / f[i] - 1.0)


LAM = np.array([-1.3, -0.71, -0.42, -0.40, -0.385, -0.37, -0.2, -0.05])


@pytest.mark.parametrize("n_el,kT", [(7.0, 0.01), (6.0, 0.03), (9.0, 0.005)])
def test_fermi_dirac_thermodynamic_identities(n_el, kT):
    f, mts = fermi_dirac(LAM, n_el, kT)
    assert abs(np.sum(f) - n_el) < 1e-12
    assert np.all(f >= 0.0) and np.all(f <= 2.0) and np.all(np.diff(f) <= 0.0)
    eF = _fermi_level(LAM, f, kT)
    h = 1e-6
    for i in range(len(LAM)):
        dl = np.zeros_like(LAM)
        dl[i] = h
        d = (_omega(LAM + dl, eF, kT) - _omega(LAM - dl, eF, kT)) / (2 * h)
        assert abs(d - f[i]) < 1e-7
    dT = 1e-7
    S = -(_omega(LAM, eF, kT + dT) - _omega(LAM, eF, kT - dT)) / (2 * dT)
    assert abs(mts - (-kT * S)) < 1e-8
    assert abs(float(np.dot(f, LAM)) + mts - (_omega(LAM, eF, kT) + eF * n_el)) < 1e-11


def test_fermi_dirac_zero_temperature_limit():
    lam = np.array([-2.0, -1.0, -0.5, 0.3, 0.9])
    f, mts = fermi_dirac(lam, 6.0, 1e-3)     # gap 0.8 at the Fermi level
    assert np.max(np.abs(f - [2, 2, 2, 0, 0])) < 1e-12 and abs(mts) < 1e-12
    f, mts = fermi_dirac(lam, 5.0, 1e-3)     # odd count: the HOMO half filled
    assert np.max(np.abs(f - [2, 2, 1, 0, 0])) < 1e-12
    with pytest.raises(ValueError):
        fermi_dirac(lam, 10.0, 1e-3)


def test_augmented_method_with_smearing_equals_direct_scf():
    # Be-like: 4 electrons in 4 orbitals, smeared (kT = 0.05): the 2s and the
    # 2p levels share 2 electrons (mu = 6 keeps H + mu coercive, lambda_1 ~ -1.75)
    inst = make_instance("he_p1", cells=6, coarse_cells=3, tol_scf=1e-12, mu=6.0)
    inst.Z = np.array([4.0])
    inst.occ = np.array([2.0, 2.0, 0.0, 0.0])
    inst.smearing = 0.05
    P = Problem(inst)
    st = P.solve(max_outer=500)
    assert st.info["drho"] < 1e-12
    assert abs(np.sum(st.occ) - 4.0) < 1e-12 and 0.0 < st.occ[1] < 2.0 and st.occ[2] > 1e-6
    d = P.direct_scf(tol=1e-12)
    assert np.max(np.abs(st.lam - d.lam)) < 1e-10 * np.max(np.abs(d.lam))
    assert abs(P.energy(st) - P.energy(d)) < 1e-10 * abs(P.energy(d))

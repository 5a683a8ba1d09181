"""The helium workload at its full size (Z = 2, P1 on the 20^3 graded mesh,
coarse 8^3, mu = 32) against the CPU oracle's Algorithm 3 trajectory stored
in tests/golden/he_p1_trajectory.json (written by
tests/golden/make_he_p1_trajectory.py, which calls only the oracle): the GPU
runs the same 200 steps from the same coarse-space initial guess and its
eigenvalue and energy match the oracle's at 1e-10 relative along the way."""
import json
import os

import numpy as np
import pytest

from workloads import make_instance

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "he_p1_trajectory.json")


def test_full_size_helium_trajectory_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19249_gb300 import nas
    ref = json.load(open(GOLDEN))
    traj = ref["trajectory"]
    inst = make_instance("he_p1", **ref["settings"])
    s = nas.Solver(inst)
    s.init()
    assert s.sizes()["n"] == ref["unknowns"]
    lam = s.get(nas.NAS_Q_EIGVALS)
    assert abs(lam[0] - traj[0]["lam"][0]) < 1e-10 * abs(traj[0]["lam"][0])
    checks = {1, 2, 5, 10, 25, 50, 100, 150, len(traj) - 1}
    for k in range(1, len(traj)):
        r, rep = s.step()
        assert r == 0
        if k in checks:
            t = traj[k]
            lam = s.get(nas.NAS_Q_EIGVALS)
            assert abs(lam[0] - t["lam"][0]) < 1e-10 * abs(t["lam"][0]), (k, lam[0], t["lam"][0])
            assert abs(rep.energy - t["energy"]) < 1e-10 * abs(t["energy"]), (k, rep.energy, t["energy"])
            assert abs(rep.drho - t["drho"]) < 1e-6 * t["drho"] + 1e-12, (k, rep.drho, t["drho"])
    s.close()

"""Writes he_p1_trajectory.json: the CPU oracle's Algorithm 3 trajectory for
the helium workload at its full size (Z = 2, one doubly occupied orbital, P1
on the 20^3 graded mesh of [-10,10]^3, coarse 8^3, mu = 8 M sum Z^2 = 32), from
the coarse-space initial guess until ||rho^(l) - rho^(l-1)||_0 < 1e-8 (the
workload's SCF tolerance): per step the eigenvalue, the energy of Sec. 3.1,
the density change and the inner-iteration count.

Calls only the oracle (oracle/) and the input recipe (workloads/).  Run from
the repository root:  python tests/golden/make_he_p1_trajectory.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.nas import Problem          # noqa: E402
from workloads import make_instance     # noqa: E402

SETTINGS = dict(tol_bvp=1e-13, tol_poisson=1e-13, tol_scf=1e-8, max_outer=200)


def main():
    inst = make_instance("he_p1", **SETTINGS)
    P = Problem(inst)
    st = P.initial_state()
    traj = [{"step": 0, "lam": [float(x) for x in st.lam], "energy": P.energy(st), "drho": None,
             "n_inner": int(st.n_inner)}]
    for step in range(1, SETTINGS["max_outer"] + 1):
        st = P.step(st)
        traj.append({"step": step, "lam": [float(x) for x in st.lam], "energy": P.energy(st),
                     "drho": float(st.info["drho"]), "n_inner": int(st.n_inner)})
        print(step, traj[-1]["lam"][0], traj[-1]["energy"], traj[-1]["drho"], flush=True)
        if st.info["drho"] < inst.tol_scf:
            break
    out = {"workload": "he_p1 (20^3 P1 graded, coarse 8^3, mu = %g)" % P.mu, "settings": SETTINGS,
           "unknowns": int(P.fine.n), "coarse_unknowns": int(P.coarse.n), "trajectory": traj}
    with open(os.path.join(HERE, "he_p1_trajectory.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

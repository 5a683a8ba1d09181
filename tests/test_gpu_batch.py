"""Batched independent instances (nas_batch_run): concurrent contexts on their
own streams give bit-identical results to the same contexts run one after
another, and the batched workload generator is seeded."""
import numpy as np
import pytest

from workloads.configs import batch_instances


def test_batch_workload_recipe():
    a = batch_instances(count=8)
    b = batch_instances(count=8)
    for x, y in zip(a, b):
        assert x.order == y.order and np.array_equal(x.fine_xyz, y.fine_xyz) and np.array_equal(x.R, y.R)
    full = batch_instances()
    assert len(full) == 64
    orders = {i.order for i in full}
    assert orders == {1, 2}
    for i in full:
        assert 1 <= len(i.Z) <= 6 and len(i.occ) <= 8 and set(i.Z) <= {1.0, 2.0, 3.0, 4.0}


@pytest.mark.gpu
def test_batch_run_matches_sequential():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19249_gb300 import nas
    insts = [i for i in batch_instances(count=64, dof_hi=3e4)][:6]
    streams = [torch.cuda.Stream() for _ in range(2 * len(insts))]

    def make(k, inst):
        s = nas.Solver(inst, stream=streams[k].cuda_stream, tol_poisson=1e-10, tol_bvp=1e-10)
        s.init()
        return s

    seq = [make(k, inst) for k, inst in enumerate(insts)]
    for s in seq:
        for _ in range(2):
            s.step()
    bat = [make(len(insts) + k, inst) for k, inst in enumerate(insts)]
    status, reps = nas.nas_batch_run([s.h for s in bat], 2, 4)
    assert all(st in (0, -5) for st in status)
    for a, b, rep in zip(seq, bat, reps):
        assert np.array_equal(a.get(nas.NAS_Q_EIGVALS), b.get(nas.NAS_Q_EIGVALS))
        assert np.array_equal(a.get(nas.NAS_Q_ENERGY), b.get(nas.NAS_Q_ENERGY))
        assert np.array_equal(a.get(nas.NAS_Q_RHO_OUT), b.get(nas.NAS_Q_RHO_OUT))
        assert rep.step == 2
    with pytest.raises(nas.NasError):
        nas.nas_batch_run([bat[0].h, bat[0].h], 1, 2)   # the same context twice
    for s in seq + bat:
        s.close()


@pytest.mark.gpu
def test_batch_run_matches_oracle():
    """Eight instances of the batched workload run concurrently through
    nas_batch_run, each compared with the CPU oracle run on its own (initial
    coarse-space SCF and one augmented step): eigenvalues and energies within
    1e-10 relative wherever every inner SCF met its tolerance.  Closed-shell
    instances only: with an odd electron count the half-filled highest level
    lies close to the next one on these coarse spaces (a lithium atom on 3^3
    coarse cells: -0.053 and -0.043 Ha), the coarse-space initial SCF stops at
    its iteration cap, and an unconverged start is an iterate that rounding
    decides, with nothing well defined to compare."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.nas import Problem
    from paper_2404_19249_gb300 import nas
    # the batched workload's recipe at 2-4k unknowns per instance (the oracle
    # takes 100-330 s per instance at the 1e4-3e4 unknowns of the full recipe)
    insts = [i for i in batch_instances(count=64, dof_lo=2e3, dof_hi=4e3) if int(i.Z.sum()) % 2 == 0][:8]
    for inst in insts:
        inst.tol_bvp = 1e-15
        inst.tol_poisson = 1e-14
        inst.tol_scf = 1e-10
    solvers = []
    for inst in insts:
        s = nas.Solver(inst)
        s.init()
        solvers.append(s)
    status, reps = nas.nas_batch_run([s.h for s in solvers], 1, 4)
    compared = 0
    for inst, s, st_gpu, rep in zip(insts, solvers, status, reps):
        P = Problem(inst)
        st0 = P.initial_state()
        st = P.step(st0)
        if not (st0.inner_converged and st.inner_converged and rep.inner_converged):
            continue
        assert st_gpu == 0
        lam = s.get(nas.NAS_Q_EIGVALS)
        assert np.max(np.abs(lam - st.lam)) < 1e-10 * np.max(np.abs(st.lam))
        E = P.energy(st)
        assert abs(rep.energy - E) < 1e-10 * abs(E)
        compared += 1
    assert compared >= 5     # the oracle's inner SCFs converge for 6 of the 8
    for s in solvers:
        s.close()

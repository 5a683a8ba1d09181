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

"""bench.py host logic on the CPU: the batched-workload report (with a fake
library, so that no GPU is needed) and the per-kernel source hash that keys
the recorded DRAM traffic."""
import importlib.util
import os
import types

import numpy as np
import pytest

ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..")


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _fake_library(n_inst, unconverged=()):
    """A stand-in for the library: every instance reports energy -2 and
    eigenvalues (-1, -0.5) in FP64; the mixed-precision run shifts them by
    1e-11, except that instances listed in `unconverged` stop their inner SCF
    at its cap and move by 0.05."""
    state = {"precision": 0}

    class Opt:
        precision = 0

    class Solver:
        count = 0

        def __init__(self, inst, **kw):
            self.opt = Opt()
            self.h = Solver.count
            Solver.count += 1

        def sizes(self):
            return {"n": 100}

        def init(self):
            pass

        def get(self, q):
            shift = 0.0
            if self.opt.precision:
                shift = 0.05 if self.h in unconverged else 1e-11
            return np.array([-1.0 + shift, -0.5])

        def close(self):
            pass

    class Rep:
        def __init__(self, h, precision):
            bad = h in unconverged
            self.energy = -2.0 + ((0.05 if bad else 1e-11) if precision else 0.0)
            self.inner_converged = 0 if bad else 1

    solvers = {}

    def make(inst, **kw):
        s = Solver(inst, **kw)
        solvers[s.h] = s
        return s

    def batch_run(hs, steps, threads):
        return [0] * len(hs), [Rep(h, solvers[h].opt.precision) for h in hs]

    return types.SimpleNamespace(Solver=make, NAS_Q_EIGVALS=1, nas_set_options=lambda h, o: None,
                                 nas_batch_run=batch_run), state


def _torch():
    cuda = types.SimpleNamespace(current_stream=lambda d: types.SimpleNamespace(cuda_stream=0),
                                 synchronize=lambda d: None)
    return types.SimpleNamespace(cuda=cuda)


def test_batch_report_separates_unconverged_instances(bench, monkeypatch):
    import workloads.configs as wc
    monkeypatch.setattr(wc, "batch_instances", lambda count: [None] * count)
    nas, _ = _fake_library(6, unconverged=(3,))
    args = types.SimpleNamespace(batch=6, tol_poisson=1e-10, tol_bvp=1e-10, poisson_adaptive=1, batch_steps=1,
                                 batch_threads=2, batch_mixed=1)
    out = bench.run_batch(args, nas, _torch(), 0)
    assert out["identical_results"] is True
    bm = out["batched_mixed"]
    assert bm["precision"] == "mixed" and out["batched"]["precision"] == "fp64"
    assert bm["inner_scf_not_converged"] == 1 and out["sequential"]["inner_scf_not_converged"] == 1
    assert bm["converged_instances"] == 5
    assert abs(bm["max_energy_diff_ha"] - 0.05) < 1e-12
    assert abs(bm["max_eigenvalue_diff_ha"] - 0.05) < 1e-12
    assert bm["max_energy_diff_ha_converged"] < 1e-10
    assert bm["max_eigenvalue_diff_ha_converged"] < 1e-10
    assert "speedup_mixed" in out and "speedup" in out


def test_kernel_hash_ignores_other_kernels(bench, tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2404_19249_gb300" / "csrc"
    csrc.mkdir(parents=True)
    base = ("static const int kPcgBlocks = 8;\n"
            "template <typename T>\n__global__ void k_a(int x) {\n    x += 1;\n}\n"
            "template <typename T>\n__global__ void k_b(int x) {\n    x += 2;\n}\n")
    (csrc / "k.cu").write_text(base)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h_a = bench.kernel_source_hash("k.cu", "k_a")
    (csrc / "k.cu").write_text(base.replace("x += 2;", "x += 3;"))
    assert bench.kernel_source_hash("k.cu", "k_a") == h_a          # k_b edited: k_a's record stays
    (csrc / "k.cu").write_text(base.replace("x += 1;", "x -= 1;"))
    assert bench.kernel_source_hash("k.cu", "k_a") != h_a          # k_a edited
    (csrc / "k.cu").write_text(base.replace("kPcgBlocks = 8", "kPcgBlocks = 16"))
    assert bench.kernel_source_hash("k.cu", "k_a") != h_a          # launch constant edited


def test_cpu_spmm_baseline_on_a_small_pattern(bench):
    """The CPU SpMM baseline reads the library's CSR pattern and stiffness
    values through nas_get; here a fake context serves a small 3D Laplacian."""
    import scipy.sparse as sp
    m = 12
    T = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    I = sp.eye(m)
    A = (sp.kron(sp.kron(T, I), I) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(I, I), T)).tocsr()
    A.sort_indices()
    nas = types.SimpleNamespace(NAS_Q_ROWPTR=0, NAS_Q_COLIDX=1, NAS_Q_K=2)
    data = {0: A.indptr.astype(np.int32), 1: A.indices.astype(np.int32), 2: A.data.astype(np.float64)}
    s = types.SimpleNamespace(get=lambda q: data[q])
    out = bench.cpu_spmm_baseline(s, nas, {"n": A.shape[0], "N": 5}, reps=2)
    assert out["gbs"] > 0 and out["threads"] >= 1 and out["N"] == 5 and out["unit"] == "GB/s"


def test_kernel_rooflines_and_dominant(bench):
    """Roofline figures from report timings: bytes (or flops) per launch over
    the mean launch time, and the dominant kernel by estimated ms per step."""
    phases = ["assembly", "bvp", "poisson", "blocks", "density", "mixing", "host_eig", "transfer", "spmm", "spmv",
              "eig_rr", "eig_wait", "spmv32", "spmm32", "recon", "densk"]

    class Rep:
        def __init__(self):
            self.phase_ms = [0.0] * 16
            self.phase_calls = [0] * 16
            self.phase_ms[phases.index("spmm32")] = 4.0      # 4 launches of 1 ms
            self.phase_calls[phases.index("spmm32")] = 4
            self.phase_ms[phases.index("recon")] = 10.0      # 2 launches of 5 ms
            self.phase_calls[phases.index("recon")] = 2
            self.spmm_bytes = self.spmm_flops = 0.0
            self.spmm32_bytes = 4 * 3.0e9
            self.poisson_spmv_ms = 0.0
            self.poisson_spmv_launches = 0
            self.poisson_iters = 0

    sz = {"n": 1000, "nnz": 20000, "N": 64, "ne": 100, "order": 2}
    roofs = bench.kernel_rooflines([Rep(), Rep()], sz, 2, phases, 6000.0, "measured", nz_occ=64)
    f32 = roofs["spmm_f32"]
    assert abs(f32["achieved"] - 3000.0) < 1e-9 and abs(f32["frac"] - 0.5) < 1e-12   # 3 GB in 1 ms
    assert f32["launches"] == 8 and abs(f32["est_ms_per_step"] - 4.0) < 1e-12
    rec = roofs["k_reconstruct"]
    assert rec["bound"] == "alu" and abs(rec["algorithmic_flops_per_launch"] - 2.0 * 1000 * 64 * 68) < 1e-6
    assert abs(rec["est_ms_per_step"] - 10.0) < 1e-12
    assert bench.dominant(roofs) is rec
    # tensor-core reconstruction: the roofline counts only the FP64 work the
    # kernel keeps (I u_H and the final scaled FMA, 10 n N), and reports the
    # whole product's FP64-equivalent rate beside it
    tc = bench.kernel_rooflines([Rep(), Rep()], sz, 2, phases, 6000.0, "measured", nz_occ=64,
                                dense_tc=True)["k_reconstruct"]
    assert "tensor cores" in tc["kernel"]
    assert abs(tc["algorithmic_flops_per_launch"] - 10.0 * 1000 * 64) < 1e-6
    assert abs(tc["fp64_equivalent_tflops"] - 2.0 * 1000 * 64 * 68 / 5e-3 / 1e12) < 1e-12   # 5 ms per launch
    assert abs(tc["algorithmic_gbs"] - (16.0 * 1000 * 64 + 48.0 * 1000) / 5e-3 / 1e9) < 1e-9


def test_cpu_extrapolation_terms(bench):
    ref = {"step_s": [3.0, 3.2, 2.8], "eig_s": [0.5, 0.5, 0.5], "n_inner": [7, 7, 7], "n": 1000, "N": 1}
    ex = bench.cpu_extrapolation(ref, eig_full_s=2.0, n_full=10000, N_full=4, inner_full=14)
    # rest of the reference step (3.0 - 0.5) x (10000 x 4 x 14) / (1000 x 1 x 7) + 14 eigensolves
    assert abs(ex["fine_mesh_terms_s"] - 2.5 * 80.0) < 1e-9
    assert abs(ex["small_eigensolve_s"] - 28.0) < 1e-12
    assert abs(ex["seconds_per_step"] - (200.0 + 28.0)) < 1e-9

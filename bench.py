#!/usr/bin/env python
"""Benchmark of the augmented subspace method on one GB300 (or N replicas).

A step is one Algorithm 3 iteration (one augmented-subspace step): H~
assembly, the N shifted linear boundary value problems (block PCG), the
basis of the augmented space, its fixed blocks, and the inner SCF of the
small Kohn-Sham problem to convergence (Hartree Poisson solves, LDA,
A^NL assembly, Galerkin blocks, host small eigensolve, density, Anderson).

Workload (default): 8 nuclei, Z uniform in {1..8}, R uniform in [-4,4]^3
(seed 1), N = 21 doubly/singly occupied orbitals, Omega = [-16,16]^3, P2 on a
50^3 tensor grid graded toward the nuclei (1,030,301 nodes, 970,299
unknowns), coarse 16^3 P1 (3,375 unknowns), FP64.

Output: one JSON line (rank 0).  Multi-GPU: one process per GPU under
torchrun, each an independent replica of the workload (weak scaling, no
collective on the data path); value = total steps of all ranks / max time.
`--impl reference` times the CPU oracle instead (bounded sample, see
`oracle_sample`).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "augmented-subspace steps/s + SpMM HBM GB/s; mixed vs FP64 at ≤1e-8 Ha error"
SAMPLE = dict(cells=10, coarse_cells=6)   # oracle sample: same molecule, reduced meshes
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x FP64 FMA/clk/SM x 2 flop x max clock


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="mol8_p2")
    p.add_argument("--cells", type=int, default=None)
    p.add_argument("--coarse-cells", type=int, default=None)
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--tol-poisson", type=float, default=1e-10)
    p.add_argument("--tol-bvp", type=float, default=1e-10)
    p.add_argument("--spmv-lanes", type=int, default=0)
    p.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison")
    p.add_argument("--clocks-file", default=None, help="where to keep the nvidia-smi clock samples")
    p.add_argument("--batch", type=int, default=0,
                   help="also time this many independent small instances (batched workload), "
                        "one after another and concurrently")
    p.add_argument("--batch-steps", type=int, default=2)
    p.add_argument("--batch-threads", type=int, default=8)
    p.add_argument("--batch-mixed", type=int, default=1,
                   help="1: also run the batched instances in the mixed-precision mode")
    p.add_argument("--eig-precond", type=int, default=1,
                   help="LOBPCG preconditioner: 1 = inverse coarse stiffness on the coarse rows, 0 = diagonal")
    p.add_argument("--eig-adapt", type=float, default=1e-2,
                   help="adaptive LOBPCG tolerance factor (x previous inner-SCF residual)")
    p.add_argument("--poisson-sell", type=int, default=1, help="1: sliced-ELL Poisson SpMV, 0: CSR")
    p.add_argument("--poisson-fused", type=int, default=0,
                   help="1: persistent cooperative Poisson PCG kernel, 0: per-phase kernels from a CUDA graph")
    p.add_argument("--poisson-adaptive", type=int, default=1,
                   help="1: inner Poisson tolerance follows the density residual (fixed point unchanged)")
    return p.parse_args()


def instance(args):
    from workloads import make_instance
    kw = {}
    if args.cells:
        kw["cells"] = args.cells
    if args.coarse_cells:
        kw["coarse_cells"] = args.coarse_cells
    return make_instance(args.workload, **kw)


def kernel_source_hash(name, kernel):
    """sha256 of one kernel's source text in csrc/<name>: the file's launch
    constants (lines starting "static const int kPcg") and the kernel's
    definition from its template line to its closing brace, so that edits to
    other kernels of the file leave the record of this one valid."""
    import hashlib
    lines = open(os.path.join(ROOT, "paper_2404_19249_gb300", "csrc", name)).read().splitlines()
    consts = [ln for ln in lines if ln.startswith("static const int kPcg")]
    start = next(i for i, ln in enumerate(lines) if (" " + kernel + "(") in ln and "__global__" in ln)
    if start > 0 and lines[start - 1].startswith("template"):
        start -= 1
    end = next(i for i in range(start, len(lines)) if lines[i] == "}")
    return hashlib.sha256("\n".join(consts + lines[start:end + 1]).encode()).hexdigest()


def spmv_traffic(sz, kernel="k_pcg1_spmv"):
    """DRAM bytes per full-size launch of the Poisson SpMV kernel (per
    iteration for the persistent PCG kernel: the capture's bytes over its
    iterations per launch) from the committed ncu capture
    (profiles/traffic.json: a smaller mesh of the same workload, scaled by
    nnz, since the matrix stream grows with nnz); None when the kernel source
    changed after the capture or no capture is recorded."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
    except Exception:
        return None
    try:
        if rec.get("kernel_sha256") != kernel_source_hash("kernels_pcg1.cu", kernel):
            return None
    except StopIteration:
        return None
    per_launch = (rec["dram_read_bytes"] + rec["dram_write_bytes"]) / rec.get("iterations_per_launch", 1)
    return per_launch * sz["nnz"] / rec["nnz"]


def workload_config(args, inst, extra=None):
    cfg = {
        "workload": "%s: %d nuclei Z=%s, N=%d orbitals, P%d fine mesh %d tets, coarse %d tets, FP64"
                    % (args.workload, len(inst.Z), [int(z) for z in inst.Z], inst.n_orb, inst.order,
                       len(inst.fine_tet), len(inst.coarse_tet)),
        "fine_vertices": int(len(inst.fine_xyz)),
        "l2": "no flush: the per-step working set (CSR values/indices, orbitals, quadrature arrays) exceeds the 126 MB L2",
        "tol_bvp": args.tol_bvp, "tol_poisson": args.tol_poisson, "tol_inner": inst.tol_scf,
        "poisson_tolerance": ("inexact inner solves: max(tol_poisson, min(1e-6, 1e-3 x previous density "
                              "residual))" if args.poisson_adaptive else "tol_poisson in every solve"),
        "small_eigensolver": "LOBPCG, block vectors on the device, host Rayleigh-Ritz, %s preconditioner; "
                             "residual tolerance %g x previous inner-SCF residual in [1e-11, 1e-4]"
                             % ("inverse coarse stiffness" if args.eig_precond else "diagonal", args.eig_adapt),
    }
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, device):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(device):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- oracle
def oracle_sample(n_steps, warm_steps=1):
    """Time oracle augmented steps on the reduced sample (runs in a fresh
    single-threaded process).  Returns dict with per-step seconds and sizes."""
    from oracle.nas import Problem
    from workloads import make_instance
    inst = make_instance("mol8_p2", **SAMPLE)
    inst.tol_bvp = 1e-10
    inst.tol_poisson = 1e-10
    P = Problem(inst)
    st = P.initial_state()
    for _ in range(warm_steps):
        st = P.step(st)
    times = []
    for _ in range(n_steps):
        t = time.perf_counter()
        st = P.step(st)
        times.append(time.perf_counter() - t)
    return {"step_s": times, "n_sample": int(P.fine.n), "nH": int(P.coarse.n), "n_inner": int(st.n_inner)}


def run_oracle_subprocess(n_steps, warm_steps=1, timeout=900):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print('ORACLE', json.dumps(bench.oracle_sample(%d, %d)))" % (ROOT, n_steps, warm_steps))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=timeout)
    for line in r.stdout.splitlines():
        if line.startswith("ORACLE "):
            return json.loads(line[7:])
    raise RuntimeError("oracle sample failed: %s" % r.stderr[-2000:])


def cpu_baseline_from(sample, n_full):
    t = statistics.median(sample["step_s"])
    scale = n_full / sample["n_sample"]
    return {
        "value": 1.0 / (t * scale), "unit": "steps/s", "cores": 1, "kind": "oracle",
        "sample": ("CPU oracle (NumPy/SciPy FP64, 1 thread) Algorithm 3 steps on the same molecule with a "
                   "P2 %d^3 fine mesh (%d unknowns) and %d^3 coarse mesh; measured %.2f s/step, scaled to the "
                   "full %d-unknown mesh linearly in fine unknowns (the paper's O(N N_k) work per step)"
                   % (SAMPLE["cells"], sample["n_sample"], SAMPLE["coarse_cells"], t, n_full)),
        "sample_step_s": t,
    }


def cpu_spmm_baseline(s, nas, sz, reps=3):
    """SpMM bandwidth of the oracle's OpenMP CSR SpMM (oracle/spmm_omp.c) on
    all host cores, for the benchmark's own matrix pattern (the stiffness
    values, the same nonzeros as every fine operator) and N interleaved
    right-hand sides, with the same algorithmic byte count as the GPU SpMM:
    nnz (8 + 4) + 4 (n + 1) + 2 n N 8."""
    import ctypes as C
    import numpy as np
    from oracle import build_c
    lib = build_c.load()
    rowptr = np.ascontiguousarray(s.get(nas.NAS_Q_ROWPTR), dtype=np.int32)
    col = np.ascontiguousarray(s.get(nas.NAS_Q_COLIDX), dtype=np.int32)
    val = np.ascontiguousarray(s.get(nas.NAS_Q_K), dtype=np.float64)
    n, N = sz["n"], sz["N"]
    X = np.random.default_rng(0).standard_normal((n, N))
    Y = np.empty((n, N))
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)

    def ptr(a):
        return a.ctypes.data_as(C.c_void_p)

    t = lib.oracle_spmm_seconds(n, ptr(rowptr), ptr(col), ptr(val), N, ptr(X), ptr(Y), threads, reps)
    nbytes = 12.0 * len(val) + 4.0 * (n + 1) + 2.0 * n * N * 8.0
    return {"gbs": nbytes / t / 1e9, "unit": "GB/s", "threads": threads, "N": N, "ms_per_product": t * 1e3,
            "kind": "oracle C/OpenMP CSR SpMM (oracle/spmm_omp.c), the benchmark's pattern, mean of %d "
                    "products after one untimed" % reps}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    inst = instance(args)
    # unknowns of the full mesh: P2 nodes minus boundary nodes (counted without assembling)
    n_full = full_unknowns(inst)
    sample = run_oracle_subprocess(args.steps, warm_steps=max(1, args.warmup))
    cb = cpu_baseline_from(sample, n_full)
    ms = statistics.median(sample["step_s"]) * (n_full / sample["n_sample"]) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {k: v for k, v in workload_config(args, inst).items()
                   if k not in ("poisson_tolerance", "small_eigensolver")},
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def full_unknowns(inst):
    import numpy as np
    xyz = inst.fine_xyz
    tet = inst.fine_tet.astype(np.int64)
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    on_b = np.any((xyz == lo) | (xyz == hi), axis=1)
    n = int(np.sum(~on_b))
    if inst.order == 2:
        pairs = np.concatenate([np.sort(tet[:, [i, j]], axis=1) for i, j in
                                [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]])
        key = np.unique(pairs[:, 0] * len(xyz) + pairs[:, 1])
        a, b = key // len(xyz), key % len(xyz)
        mid = 0.5 * (xyz[a] + xyz[b])
        n += int(np.sum(~np.any((mid == lo) | (mid == hi), axis=1)))
    return n


# ---------------------------------------------------------------------------- batched instances
def run_batch(args, nas, torch, device):
    """Independent small molecules (workloads.configs.batch_instances): the same
    contexts run `batch_steps` steps one after another (one host thread) and
    concurrently (nas_batch_run with batch_threads workers; the library runs
    each context on a private stream), each time from the same initial state,
    in FP64, and (with --batch-mixed 1) concurrently in the mixed-precision
    mode (FP32 Poisson and block PCG inside FP64 refinement).  Returns
    instance-steps/s for each, checks that the two FP64 runs give
    bit-identical energies, and reports the mixed run's largest energy and
    eigenvalue differences from the sequential FP64 run."""
    import numpy as np
    from workloads.configs import batch_instances
    insts = batch_instances(count=args.batch)
    stream = torch.cuda.current_stream(device).cuda_stream
    t0 = time.time()
    solvers = [nas.Solver(inst, device=device, stream=stream, tol_poisson=args.tol_poisson,
                          tol_bvp=args.tol_bvp, poisson_adaptive=args.poisson_adaptive)
               for inst in insts]
    setup = time.time() - t0
    out = {"instances": len(insts), "steps_each": args.batch_steps,
           "unknowns": [int(sv.sizes()["n"]) for sv in solvers]}
    energies, eigvals, conv = {}, {}, {}
    modes = [("sequential", 1, 0), ("batched", args.batch_threads, 0)]
    if args.batch_mixed:
        modes.append(("batched_mixed", args.batch_threads, 1))
    for mode, threads, precision in modes:
        for sv in solvers:
            if sv.opt.precision != precision:
                sv.opt.precision = precision
                nas.nas_set_options(sv.h, sv.opt)
            sv.init()
        torch.cuda.synchronize(device)
        t = time.perf_counter()
        status, reps = nas.nas_batch_run([sv.h for sv in solvers], args.batch_steps, threads)
        torch.cuda.synchronize(device)
        dt = time.perf_counter() - t
        energies[mode] = [r.energy for r in reps]
        eigvals[mode] = [sv.get(nas.NAS_Q_EIGVALS) for sv in solvers]
        conv[mode] = [bool(r.inner_converged) for r in reps]
        out[mode] = {"instance_steps_per_s": len(insts) * args.batch_steps / dt, "s": dt, "threads": threads,
                     "precision": "mixed" if precision else "fp64",
                     "status_ok": int(sum(st in (0, -5) for st in status)),
                     "inner_scf_not_converged": int(sum(not c for c in conv[mode]))}
    out["speedup"] = out["batched"]["instance_steps_per_s"] / out["sequential"]["instance_steps_per_s"]
    out["identical_results"] = energies["sequential"] == energies["batched"]
    if args.batch_mixed:
        # differences from the sequential FP64 run, over all instances and over
        # the instances whose inner SCF met its tolerance in both runs (an
        # inner SCF stopped by its iteration cap - a degenerate, partly
        # occupied highest orbital - leaves an iterate that rounding-level
        # differences change at the 1e-2 Ha level)
        both = [a and b for a, b in zip(conv["batched_mixed"], conv["sequential"])]
        dE = [abs(a - b) for a, b in zip(energies["batched_mixed"], energies["sequential"])]
        dl = [float(np.max(np.abs(a - b))) for a, b in zip(eigvals["batched_mixed"], eigvals["sequential"])]
        bm = out["batched_mixed"]
        out["speedup_mixed"] = bm["instance_steps_per_s"] / out["sequential"]["instance_steps_per_s"]
        bm["max_energy_diff_ha"] = float(max(dE))
        bm["max_eigenvalue_diff_ha"] = float(max(dl))
        bm["converged_instances"] = int(sum(both))
        bm["max_energy_diff_ha_converged"] = float(max([d for d, c in zip(dE, both) if c], default=0.0))
        bm["max_eigenvalue_diff_ha_converged"] = float(max([d for d, c in zip(dl, both) if c], default=0.0))
    out["setup_s"] = setup
    for sv in solvers:
        sv.close()
    log("batch: %s" % json.dumps({k: v for k, v in out.items() if k != "unknowns"}))
    return out


# ---------------------------------------------------------------------------- replicas
def reduce_max(x, dist, device=None):
    """Max of a float over all ranks (no-op without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, max_ms):
    """Whole-job throughput: every rank runs `steps` steps of its own replica."""
    return world * steps / (max_ms / 1e3)


# ---------------------------------------------------------------------------- our arm
def log(msg):
    print("[bench] " + msg, file=sys.stderr, flush=True)


def main():
    args = parse()
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.steps)))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2404_19249_gb300 import build as nbuild
    if not os.path.exists(nbuild.LIB):
        nbuild.build()
    from paper_2404_19249_gb300 import nas

    inst = instance(args)
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.time()
    s = nas.Solver(inst, device=local, stream=stream, timing=1, tol_poisson=args.tol_poisson,
                   tol_bvp=args.tol_bvp, check_every=4, spmv_lanes=args.spmv_lanes,
                   poisson_adaptive=args.poisson_adaptive, eig_adapt=args.eig_adapt, eig_precond=args.eig_precond,
                   poisson_sell=args.poisson_sell, poisson_fused=args.poisson_fused)
    s.init()
    setup_s = time.time() - t0
    sz = s.sizes()
    log("setup+init %.1f s sizes %s" % (setup_s, sz))
    for w in range(args.warmup):
        tw = time.time()
        r, rep = s.step()
        log("warmup step %d: %.2f s status %d inner %d cg %d poisson %d drho %.3e E %.10f phases %s"
            % (w, time.time() - tw, r, rep.n_inner, rep.cg_iters, rep.poisson_iters, rep.drho, rep.energy,
               {k: round(v, 1) for k, v in rep.as_dict()["phase_ms"].items()}))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(args.clocks_file or "/tmp/bench_clocks_%d.csv" % os.getpid())
    # state at the start of the timed region (the mixed-precision run restarts from it)
    n0, N0, nqt0 = sz["n"], sz["N"], sz["ne"] * sz["nq"]
    s0_lam = np.zeros(N0)
    s0_psi = np.zeros((n0, N0))
    s0_rho = np.zeros(nqt0)
    nas.nas_get(s.h, nas.NAS_Q_EIGVALS, s0_lam)
    nas.nas_get(s.h, nas.NAS_Q_ORBITALS, s0_psi)
    nas.nas_get(s.h, nas.NAS_Q_RHO_IN, s0_rho)
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    reps = []
    torch.cuda.nvtx.range_push("timed")
    ev0.record()
    for _ in range(args.steps):
        r, rep = s.step()
        reps.append(nas.nas_report.from_buffer_copy(rep))
    ev1.record()
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop(local)
    ms = ev0.elapsed_time(ev1)
    log("timed: %d steps in %.1f ms; last report %s" % (args.steps, ms, reps[-1].as_dict()))
    ms = reduce_max(ms, dist, "cuda")
    value = job_value(world, args.steps, ms)

    lam64 = np.zeros(N0)
    nas.nas_get(s.h, nas.NAS_Q_EIGVALS, lam64)
    en64 = np.zeros(6)
    nas.nas_get(s.h, nas.NAS_Q_ENERGY, en64)

    # ---------------------------------------------------------------- mixed precision
    mixed = None
    if not args.no_mixed:
        nas.nas_set_state(s.h, s0_lam, s0_psi, s0_rho)
        s.opt.precision = 1
        nas.nas_set_options(s.h, s.opt)
        barrier()
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record()
        mreps = []
        for _ in range(args.steps):
            r, rep = s.step()
            mreps.append(nas.nas_report.from_buffer_copy(rep))
        m1.record()
        barrier()
        mms = reduce_max(m0.elapsed_time(m1), dist, "cuda")
        lam32 = np.zeros(N0)
        nas.nas_get(s.h, nas.NAS_Q_EIGVALS, lam32)
        en32 = np.zeros(6)
        nas.nas_get(s.h, nas.NAS_Q_ENERGY, en32)
        mixed = {
            "value": job_value(world, args.steps, mms), "unit": "steps/s", "ms_per_step": mms / args.steps,
            "what": "Poisson PCG and block PCG of the N shifted problems in FP32 inside FP64 iterative refinement; "
                    "same start state and step count as the FP64 run",
            "max_eigenvalue_err_ha": float(np.max(np.abs(lam32 - lam64))),
            "eigenvalue_err_ha": [float(x) for x in (lam32 - lam64)],
            "energy_err_ha": float(en32[0] - en64[0]),
            "poisson_ms_per_step": sum(rp.phase_ms[2] for rp in mreps) / args.steps,
            "poisson_iters_per_step": sum(rp.poisson_iters for rp in mreps) / args.steps,
            "bvp_ms_per_step": sum(rp.phase_ms[1] for rp in mreps) / args.steps,
            "fp64_bvp_ms_per_step": sum(rp.phase_ms[1] for rp in reps) / args.steps,
        }
        log("mixed: %s" % json.dumps({k: v for k, v in mixed.items() if k != "eigenvalue_err_ha"}))
        s.opt.precision = 0
        nas.nas_set_options(s.h, s.opt)

    # phase totals over the timed steps (library CUDA events on the launching stream)
    ph = {name: sum(rp.phase_ms[i] for rp in reps) for i, name in enumerate(nas.PHASES)}
    calls = {name: sum(rp.phase_calls[i] for rp in reps) for i, name in enumerate(nas.PHASES)}
    spmm_bytes = sum(rp.spmm_bytes for rp in reps)
    spmm_flops = sum(rp.spmm_flops for rp in reps)
    spmv_bytes = sum(rp.spmv_bytes for rp in reps)
    launches = int(sum(rp.kernel_launches for rp in reps))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak = float(peaks["hbm_gbs"])
        peak_src = "measured"
    except Exception:
        hbm_peak, peak_src = 6800.0, "fallback"
    spmm_ms, spmv_ms = ph["spmm"], ph["spmv"]
    spmm_gbs = spmm_bytes / (spmm_ms * 1e-3) / 1e9 if spmm_ms > 0 else 0.0
    spmv_gbs = spmv_bytes / (spmv_ms * 1e-3) / 1e9 if spmv_ms > 0 else 0.0
    spmm_tflops = spmm_flops / (spmm_ms * 1e-3) / 1e12 if spmm_ms > 0 else 0.0
    roof_spmm = {"kernel": "k_spmm_cols (CSR SpMM, N=%d interleaved RHS, FP64)" % sz["N"], "bound": "alu",
                 "achieved": spmm_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                 "frac": spmm_tflops / FP64_PEAK_TFLOPS, "traffic": None,
                 "peak_source": "FP64 FMA issue rate (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)",
                 "algorithmic_gbs": spmm_gbs, "launches": calls["spmm"], "ms_per_launch":
                     spmm_ms / max(calls["spmm"], 1)}
    # dominant kernel: the SpMV of the FP64 Poisson PCG (k_pcg1_spmv), timed by
    # CUDA events around the SpMV launches of the first two iterations of every
    # Poisson solve (library timing mode), over the timed steps
    sp_ms = sum(rp.poisson_spmv_ms for rp in reps)
    sp_n = int(sum(rp.poisson_spmv_launches for rp in reps))
    sp_bytes = 12.0 * sz["nnz"] + 20.0 * sz["n"] + 4.0   # val+col, row_ptr, p once, q written (CSR count)
    sp_ms_launch = sp_ms / max(sp_n, 1)
    sp_gbs = sp_bytes / (sp_ms_launch * 1e-3) / 1e9 if sp_ms > 0 else 0.0
    sell = sz.get("sell", 0) if args.poisson_sell else 0
    sp_name = "k_pcg1_spmv_sell" if sell else "k_pcg1_spmv"
    roof_spmv = {"kernel": ("k_pcg1_spmv_sell (sliced-ELL SpMV of the Poisson PCG, FP64; %d stored entries, "
                            "%.1f %% padding)" % (sell, 100.0 * (sell / sz["nnz"] - 1.0)))
                 if sell else "k_pcg1_spmv (CSR SpMV of the Poisson PCG, FP64)",
                 "bound": "hbm", "achieved": sp_gbs, "peak": hbm_peak, "unit": "GB/s",
                 "frac": sp_gbs / hbm_peak, "traffic": spmv_traffic(sz, sp_name), "peak_source": peak_src,
                 "algorithmic_bytes_per_launch": sp_bytes, "launches": sp_n, "ms_per_launch": sp_ms_launch,
                 "timing": "CUDA events on the library stream around the SpMV of the first two iterations "
                           "of every Poisson solve (direct launches; the rest replays from a CUDA graph)"}
    # every Poisson PCG iteration launches one SpMV: its time per step is the
    # measured mean launch time x the Poisson iterations of the timed steps
    poisson_iters = sum(rp.poisson_iters for rp in reps)
    roof_spmv["est_ms_per_step"] = sp_ms_launch * poisson_iters / args.steps
    roof_spmm["est_ms_per_step"] = spmm_ms / args.steps
    # persistent form: every launch of every FP64 Poisson solve is timed; one
    # iteration reads/writes (algorithmic, each array once per phase): SpMV
    # 12 nnz + 20 n; update 48 n; restriction 12 nnz(I^T) + 8 n; piece sums
    # 8 pieces + 12 nH; coarse solve 8 nH^2 + 16 nH; prolongation 72 n + 8 nH;
    # new direction 24 n
    fz_ms = sum(rp.poisson_fused_ms for rp in reps)
    fz_it = int(sum(rp.poisson_fused_iters for rp in reps))
    if fz_it > 0:
        nH = sz["nH"]
        fz_bytes = (12.0 * sz["nnz"] + 12.0 * sz["tnnz"] + 172.0 * sz["n"] + 8.0 * nH * nH + 8.0 * sz["tpieces"]
                    + 36.0 * nH)
        fz_gbs = fz_bytes * fz_it / (fz_ms * 1e-3) / 1e9
        tr = spmv_traffic(sz, "k_pcg1_fused")
        roof_spmv = {"kernel": "k_pcg1_fused (persistent cooperative two-level PCG of the Poisson problem, FP64, "
                               "sliced-ELL SpMV, 7 grid-wide barriers per iteration, 16 iterations per launch)",
                     "bound": "hbm", "achieved": fz_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": fz_gbs / hbm_peak, "traffic": tr, "peak_source": peak_src,
                     "traffic_unit": "DRAM bytes per iteration",
                     "algorithmic_bytes_per_iteration": fz_bytes, "iterations": fz_it,
                     "ms_per_iteration": fz_ms / fz_it,
                     "timing": "CUDA events on the library stream around every persistent launch of every "
                               "FP64 Poisson solve of the timed steps",
                     "est_ms_per_step": fz_ms / args.steps}
    dominant, other = ((roof_spmv, roof_spmm) if roof_spmv["est_ms_per_step"] >= roof_spmm["est_ms_per_step"]
                       else (roof_spmm, roof_spmv))

    # ---------------------------------------------------------------- e2e through host buffers
    n, N, nqt = sz["n"], sz["N"], sz["ne"] * sz["nq"]
    lam_h = torch.empty(N, dtype=torch.float64, pin_memory=True)
    psi_h = torch.empty((n, N), dtype=torch.float64, pin_memory=True)
    rho_h = torch.empty(nqt, dtype=torch.float64, pin_memory=True)
    en_h = torch.empty(6, dtype=torch.float64, pin_memory=True)

    def get(q, t):
        nas.nas_get(s.h, q, (t.data_ptr(), t.numel() * 8), 0)

    get(nas.NAS_Q_EIGVALS, lam_h)
    get(nas.NAS_Q_ORBITALS, psi_h)
    get(nas.NAS_Q_RHO_IN, rho_h)
    barrier()
    e0 = time.perf_counter()
    n_e2e = max(args.e2e_steps, 0)
    for _ in range(n_e2e):
        nas.nas_set_state(s.h, lam_h.data_ptr(), psi_h.data_ptr(), rho_h.data_ptr(), 0)
        s.step()
        get(nas.NAS_Q_EIGVALS, lam_h)
        get(nas.NAS_Q_ORBITALS, psi_h)
        get(nas.NAS_Q_RHO_IN, rho_h)
        get(nas.NAS_Q_ENERGY, en_h)
    barrier()
    e2e_s = reduce_max(time.perf_counter() - e0, dist, "cuda")
    io_bytes = 8 * (N + n * N + nqt)
    e2e = None
    if n_e2e > 0:
        e2e = {"value": world * n_e2e / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": io_bytes,
               "d2h_bytes_per_step": io_bytes + 48}

    if rank != 0:
        s.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    batched = run_batch(args, nas, torch, local) if args.batch > 0 else None

    # the CPU oracle sample runs after the GPU work, in a fresh single-threaded
    # process (fork + exec), so that it never competes with the host-side work
    # of the timed steps for the CPU cores
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline_from(run_oracle_subprocess(2, 1), n)
        except Exception as ex:  # the baseline is reported, never required
            cpu = {"error": str(ex)[:200]}
        try:
            cpu["spmm"] = cpu_spmm_baseline(s, nas, sz)
        except Exception as ex:
            cpu["spmm"] = {"error": str(ex)[:200]}
    last = reps[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, inst, {"unknowns": n, "nnz": sz["nnz"], "coarse_unknowns": sz["nH"],
                                               "parallelism": "replicas" if world > 1 else "1 GPU"}),
        "spmm_hbm_gbs": spmm_gbs, "spmv_hbm_gbs": sp_gbs,
        "roofline": dominant, "roofline_other": other,
        "phase_ms_per_step": {k: v / args.steps for k, v in ph.items()},
        "per_step": {"n_inner": last.n_inner, "cg_iters": last.cg_iters, "poisson_iters": last.poisson_iters,
                     "drho": last.drho, "energy": last.energy},
        "gpu_launches": launches, "e2e": e2e, "clocks": clk, "cpu_baseline": cpu, "setup_s": setup_s,
        "mixed": mixed, "energy_ha": float(en64[0]),
    }
    if batched is not None:
        line["batched"] = batched
    print(json.dumps(line))
    s.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

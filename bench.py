#!/usr/bin/env python
"""Benchmark of the augmented subspace method on one GB300 (or N replicas).

A step is one Algorithm 3 iteration (one augmented-subspace step): H~
assembly, the N shifted linear boundary value problems (block PCG), the
basis of the augmented space, its fixed blocks, and the inner SCF of the
small Kohn-Sham problem (Hartree Poisson solves, LDA, A^NL assembly,
Galerkin blocks, the small eigensolve, density, Anderson mixing).

Headline workload (default): 32 nuclei, Z uniform in {1..6}, R uniform in
[-8,8]^3 (seed 2), N = 64 orbitals with Fermi-Dirac occupations at
kT = 0.01 Ha, Omega = [-16,16]^3, P2 on a 100^3 tensor grid graded toward
the nuclei (8,120,601 nodes, 7,880,599 unknowns), coarse 16^3 P1 (3,375
unknowns), mixed precision (FP32 Poisson and block PCG inside FP64
iterative refinement; everything else FP64).  The same steps are run in
FP64 from the same start state for the per-eigenvalue error of the mixed
form and the mixed-over-FP64 speed ratio.  Secondary lines: the 8-nucleus
P2 molecule (970,299 unknowns, N = 21, FP64) and helium on the 20^3 P1 mesh
(6,859 unknowns, FP64), the size at which the CPU oracle also runs.

Output: one JSON line (rank 0).  Multi-GPU: one process per GPU under
torchrun, each an independent replica of the workload (weak scaling, no
collective on the data path); value = total steps of all ranks / max time.
`--impl reference` times the CPU oracle on the helium workload at full size.
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
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x FP64 FMA/clk/SM x 2 flop x max clock
REFERENCE_WORKLOAD = "he_p1"                      # the oracle's full-size config


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="mol32_p2")
    p.add_argument("--precision", default="auto", choices=["auto", "mixed", "fp64"],
                   help="headline precision; auto = mixed for mol32_p2 (the mixed-precision workload), else fp64")
    p.add_argument("--cells", type=int, default=None)
    p.add_argument("--coarse-cells", type=int, default=None)
    p.add_argument("--compare-steps", type=int, default=3,
                   help="steps of both precisions from the timed run's start state (<= --steps; 0: none)")
    p.add_argument("--e2e-steps", type=int, default=-1, help="-1: the same count as --steps")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-secondary", action="store_true", help="skip the 8-nucleus and helium lines")
    p.add_argument("--secondary-steps", type=int, default=10)
    p.add_argument("--tol-poisson", type=float, default=1e-12)
    p.add_argument("--tol-bvp", type=float, default=1e-10)
    p.add_argument("--inner-adapt", type=float, default=1e-2,
                   help="inexact inner SCF: stop at max(tol_inner, inner_adapt x previous step's drho)")
    p.add_argument("--bvp-adapt", type=float, default=1e-2,
                   help="inexact linear solves: max(tol_bvp, min(1e-4, bvp_adapt x previous step's drho))")
    p.add_argument("--anderson-restart", type=float, default=None,
                   help="clear the Anderson history at a residual above this x the inner SCF's best "
                        "(default: the workload's setting)")
    p.add_argument("--spmv-lanes", type=int, default=0)
    p.add_argument("--clocks-file", default=None, help="where to keep the nvidia-smi clock samples")
    p.add_argument("--batch", type=int, default=0,
                   help="also time this many independent small instances (batched workload), "
                        "one after another and concurrently")
    p.add_argument("--batch-steps", type=int, default=2)
    p.add_argument("--batch-threads", type=int, default=8)
    p.add_argument("--batch-mixed", type=int, default=1,
                   help="1: also run the batched instances in the mixed-precision mode")
    p.add_argument("--eig-precond", type=int, default=2,
                   help="LOBPCG preconditioner: inverse coarse stiffness on the coarse rows with its dense product "
                        "on the tensor cores (2) or SIMT (1); 0 = diagonal")
    p.add_argument("--eig-adapt", type=float, default=1e-2,
                   help="adaptive LOBPCG tolerance factor (x previous inner-SCF residual)")
    p.add_argument("--poisson-sell", type=int, default=1, help="1: sliced-ELL Poisson SpMV, 0: CSR")
    p.add_argument("--poisson-fused", type=int, default=0,
                   help="1: persistent cooperative Poisson PCG kernel, 0: per-phase kernels from a CUDA graph")
    p.add_argument("--dense-tc", type=int, default=1,
                   help="1: the FP64 dense contractions (reconstruction, Gram matrices) on the tensor cores from exact "
                        "integer slices, 0: FP64 SIMT")
    p.add_argument("--poisson-f32", type=int, default=0,
                   help="mixed precision: 1 = FP32 Poisson solves for tolerances >= 1e-9, 0 = FP64 Poisson")
    p.add_argument("--poisson-adaptive", type=int, default=1,
                   help="1: inner Poisson tolerance follows the density residual (fixed point unchanged)")
    return p.parse_args(argv)


def headline_precision(args):
    if args.precision != "auto":
        return args.precision
    return "mixed" if args.workload == "mol32_p2" else "fp64"


def instance(name, cells=None, coarse_cells=None):
    from workloads import make_instance
    kw = {}
    if cells:
        kw["cells"] = cells
    if coarse_cells:
        kw["coarse_cells"] = coarse_cells
    return make_instance(name, **kw)


def solver_options(args, timing=1):
    o = dict(timing=timing, tol_poisson=args.tol_poisson, tol_bvp=args.tol_bvp, check_every=4,
             spmv_lanes=args.spmv_lanes, poisson_adaptive=args.poisson_adaptive, eig_adapt=args.eig_adapt,
             eig_precond=args.eig_precond, poisson_sell=args.poisson_sell, poisson_fused=args.poisson_fused,
             inner_adapt=args.inner_adapt, bvp_adapt=args.bvp_adapt, poisson_f32=args.poisson_f32,
             dense_tc=args.dense_tc)
    if args.anderson_restart is not None:
        o["anderson_restart"] = args.anderson_restart
    return o


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


def spmv_traffic(sz, kernel="k_pcg1_spmv_sell"):
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


def workload_config(args, name, inst, sz, precision, extra=None):
    cfg = {
        "workload": "%s: %d nuclei Z=%s, N=%d orbitals%s, P%d fine mesh %d tets (%d unknowns), coarse %d tets "
                    "(%d unknowns), %s"
                    % (name, len(inst.Z), [int(z) for z in inst.Z], inst.n_orb,
                       (", Fermi-Dirac kT=%g Ha" % inst.smearing) if getattr(inst, "smearing", 0.0) > 0 else "",
                       inst.order, len(inst.fine_tet), sz["n"], len(inst.coarse_tet), sz["nH"],
                       "mixed FP32/FP64" if precision == "mixed" else "FP64"),
        "unknowns": sz["n"], "nnz": sz["nnz"], "coarse_unknowns": sz["nH"], "orbitals": sz["N"],
        "mu": inst.mu, "anderson_beta": getattr(inst, "anderson_beta", 0.7),
        "l2": "no flush: the per-step working set (CSR values/indices, orbitals, quadrature arrays) exceeds the "
              "126 MB L2 many times over",
        "tol_bvp": args.tol_bvp, "tol_poisson": args.tol_poisson, "tol_inner": inst.tol_scf,
        "inner_scf_tolerance": ("inexact: max(tol_inner, %g x previous step's drho)" % args.inner_adapt
                                if args.inner_adapt > 0 else "tol_inner in every step"),
        "bvp_tolerance": ("inexact: max(tol_bvp, min(1e-4, %g x previous step's drho))" % args.bvp_adapt
                          if args.bvp_adapt > 0 else "tol_bvp in every step"),
        "poisson_tolerance": ("inexact inner solves: max(tol_poisson, min(1e-6, 1e-3 x previous density "
                              "residual))" if args.poisson_adaptive else "tol_poisson in every solve"),
        "small_eigensolver": "LOBPCG, block vectors on the device, host Rayleigh-Ritz, %s preconditioner; "
                             "residual tolerance %g x previous inner-SCF residual in [1e-11, 1e-4]"
                             % ({2: "inverse coarse stiffness (tensor-core product)", 1: "inverse coarse stiffness",
                                 0: "diagonal"}[args.eig_precond], args.eig_adapt),
        "dense_contractions": ("reconstruction U^ alpha and Gram matrices on the tensor cores (exact 7-bit integer "
                               "slices, FP64 accuracy)" if args.dense_tc else "FP64 SIMT"),
    }
    if extra:
        cfg.update(extra)
    return cfg


def phase_totals(reps, phases):
    ms = {name: sum(rp.phase_ms[i] for rp in reps) for i, name in enumerate(phases)}
    calls = {name: sum(rp.phase_calls[i] for rp in reps) for i, name in enumerate(phases)}
    return ms, calls


def kernel_rooflines(reps, sz, steps, phases, hbm_peak, peak_src, nz_occ, layouts=None, dense_tc=False):
    """Per-kernel achieved throughput from the library's live CUDA-event
    timings of the timed steps (reports `reps`), against its roofline: HBM
    bytes for the sparse and streaming kernels, the FP64 issue rate for the
    FP64-ALU-bound ones.  Returns {kernel: dict}; each dict carries
    est_ms_per_step (mean launch time x launches per step) so that the
    caller can pick the dominant kernel of the run.

    Algorithmic bytes / flops per launch (n unknowns, nnz CSR entries, N
    columns, ne elements, 14 quadrature points and 10 nodes per P2 element,
    55 node pairs):
      FP64 SpMM           nnz (8+4) + 4 (n+1) + 2 n N 8   (FP64-ALU bound: 2 nnz N flop)
      FP32 SpMM           nnz (4+4) + 4 (n+1) + 2 n N 4
      FP64 Poisson SpMV   12 nnz + 20 n + 4
      FP32 Poisson SpMV   8 nnz + 12 n + 4
      reconstruction      2 n N (4 + N) flop (Psi = I u_H + U^ alpha)
      density             2 ne (Nz (10 + 55) + 14 x 55) flop, Nz = orbitals with f > 0
    """
    ms, calls = phase_totals(reps, phases)
    n, nnz, N = sz["n"], sz["nnz"], sz["N"]
    layouts = layouts or {}
    out = {}

    def hbm(name, kern_ms, launches, nbytes, desc):
        if launches <= 0 or kern_ms <= 0:
            return
        per = kern_ms / launches
        gbs = nbytes / (per * 1e-3) / 1e9
        out[name] = {"kernel": desc, "bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": gbs / hbm_peak, "peak_source": peak_src, "algorithmic_bytes_per_launch": nbytes,
                     "launches": int(launches), "ms_per_launch": per,
                     "est_ms_per_step": per * launches / steps}

    def alu(name, kern_ms, launches, flops, desc, nbytes=None):
        if launches <= 0 or kern_ms <= 0:
            return
        per = kern_ms / launches
        tf = flops / (per * 1e-3) / 1e12
        d = {"kernel": desc, "bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
             "frac": tf / FP64_PEAK_TFLOPS,
             "peak_source": "FP64 FMA issue rate (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)",
             "algorithmic_flops_per_launch": flops, "launches": int(launches), "ms_per_launch": per,
             "est_ms_per_step": per * launches / steps}
        if nbytes:
            d["algorithmic_gbs"] = nbytes / (per * 1e-3) / 1e9
        out[name] = d

    spmm_bytes = sum(rp.spmm_bytes for rp in reps)
    spmm_flops = sum(rp.spmm_flops for rp in reps)
    if calls["spmm"]:
        alu("spmm_f64", ms["spmm"], calls["spmm"], spmm_flops / calls["spmm"],
            "CSR SpMM, N=%d interleaved RHS, FP64 (autotuned layout %s)" % (N, layouts.get("f64", "?")),
            spmm_bytes / calls["spmm"])
    b32 = sum(getattr(rp, "spmm32_bytes", 0.0) for rp in reps)
    if calls.get("spmm32"):
        hbm("spmm_f32", ms["spmm32"], calls["spmm32"], b32 / calls["spmm32"],
            "CSR SpMM, N=%d interleaved RHS, FP32 values and vectors, mixed block PCG (autotuned layout %s)"
            % (N, layouts.get("f32", "?")))
    sp_ms = sum(rp.poisson_spmv_ms for rp in reps)
    sp_n = int(sum(rp.poisson_spmv_launches for rp in reps))
    poisson_iters = sum(rp.poisson_iters for rp in reps)
    if sp_n:
        sell = sz.get("sell", 0)
        hbm("k_pcg1_spmv_sell", sp_ms, sp_n, 12.0 * nnz + 20.0 * n + 4.0,
            "k_pcg1_spmv_sell (sliced-ELL SpMV of the FP64 Poisson PCG; %d stored entries, %.1f %% padding)"
            % (sell, 100.0 * (sell / nnz - 1.0)) if sell else "k_pcg1_spmv (CSR SpMV of the FP64 Poisson PCG)")
        # every Poisson iteration launches one SpMV
        out["k_pcg1_spmv_sell"]["est_ms_per_step"] = out["k_pcg1_spmv_sell"]["ms_per_launch"] * poisson_iters / steps
        out["k_pcg1_spmv_sell"]["timing"] = ("CUDA events around the SpMV of the first two iterations of every "
                                             "Poisson solve (direct launches; the rest replays from a CUDA graph)")
    if calls.get("spmv32"):
        hbm("k_pcg1_spmv_f32", ms["spmv32"], calls["spmv32"], 8.0 * nnz + 12.0 * n + 4.0,
            "k_pcg1_spmv (CSR SpMV of the FP32 inner Poisson PCG, mixed precision)")
        out["k_pcg1_spmv_f32"]["est_ms_per_step"] = out["k_pcg1_spmv_f32"]["ms_per_launch"] * poisson_iters / steps
        out["k_pcg1_spmv_f32"]["timing"] = ("CUDA events around the SpMV of the first two iterations of every "
                                            "inner FP32 solve (direct launches; the rest replays from a CUDA graph)")
    if calls.get("recon") and dense_tc and N <= 64:
        # dense part on the tensor cores: what stays on the FP64 pipe is I u_H
        # (4 FMA per entry) and the final scaled FMA (1 per entry)
        alu("k_reconstruct", ms["recon"], calls["recon"], 2.0 * n * N * 5,
            "k_tc_reconstruct (Psi = I u_H + U^ alpha, N=%d; U^ alpha on the tensor cores from exact 7-bit "
            "integer slices, the rest FP64; roofline = its remaining FP64 work)" % N, nbytes=16.0 * n * N + 48.0 * n)
        per = out["k_reconstruct"]["ms_per_launch"]
        out["k_reconstruct"]["fp64_equivalent_tflops"] = 2.0 * n * N * (4 + N) / (per * 1e-3) / 1e12
    elif calls.get("recon"):
        alu("k_reconstruct", ms["recon"], calls["recon"], 2.0 * n * N * (4 + N),
            "k_reconstruct (Psi = I u_H + U^ alpha, FP64, N=%d)" % N)
    if calls.get("densk"):
        ne = sz["ne"]
        nloc, nq = (10, 14) if sz["order"] == 2 else (4, 4)
        npair = nloc * (nloc + 1) // 2
        alu("k_density", ms["densk"], calls["densk"], 2.0 * ne * (nz_occ * (nloc + npair) + nq * npair),
            "k_density (rho = sum f psi^2 at the quadrature points via the element density matrix, FP64)")
    return out


def dominant(roofs):
    if not roofs:
        return None
    return max(roofs.values(), key=lambda d: d["est_ms_per_step"])


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


# ---------------------------------------------------------------------------- oracle (CPU)
def oracle_steps(name, n_steps, warm_steps):
    """Time `n_steps` oracle Algorithm 3 steps of workload `name` at full size
    after `warm_steps` untimed ones (in this process; the caller fixes the
    BLAS/OpenMP thread count).  The time spent in the oracle's small
    eigensolve is recorded separately, through a wrapper that only times the
    call."""
    from oracle.nas import Problem
    from workloads import make_instance
    inst = make_instance(name)
    inst.tol_bvp = 1e-10
    inst.tol_poisson = 1e-10
    t0 = time.perf_counter()
    P = Problem(inst)
    build_s = time.perf_counter() - t0
    eig_s = [0.0]
    inner = P.eig_small

    def timed_eig(FA, FB):
        t = time.perf_counter()
        r = inner(FA, FB)
        eig_s[0] += time.perf_counter() - t
        return r

    P.eig_small = timed_eig
    st = P.initial_state()
    for _ in range(warm_steps):
        st = P.step(st)
    steps, eigs, inners = [], [], []
    for _ in range(n_steps):
        eig_s[0] = 0.0
        t = time.perf_counter()
        st = P.step(st)
        steps.append(time.perf_counter() - t)
        eigs.append(eig_s[0])
        inners.append(int(st.n_inner))
    return {"step_s": steps, "eig_s": eigs, "n_inner": inners, "n": int(P.fine.n), "nH": int(P.coarse.n),
            "N": int(P.N), "build_s": build_s}


def oracle_eig_seconds(path, N, reps=1):
    """Time the oracle's small eigensolve (scipy.linalg.eigh of the dense
    pencil, lowest N pairs) on the pencil stored in `path` (.npz FA, FB)."""
    import numpy as np
    import types
    from oracle.nas import Problem
    d = np.load(path)
    FA, FB = d["FA"], d["FB"]
    ts = []
    for _ in range(reps):
        t = time.perf_counter()
        Problem.eig_small(types.SimpleNamespace(N=N), FA, FB)
        ts.append(time.perf_counter() - t)
    return {"eig_s": min(ts), "m": int(FA.shape[0])}


def host_threads():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def run_oracle_subprocess(call, threads, timeout=1500):
    """Run `bench.<call>` in a fresh process with `threads` BLAS/OpenMP threads
    (fork + exec, after the GPU work, so that nothing competes with the timed
    GPU steps for the host cores); returns its JSON result."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    code = ("import json,sys; sys.path.insert(0, %r); import bench; print('ORACLE', json.dumps(bench.%s))"
            % (ROOT, call))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=timeout)
    for line in r.stdout.splitlines():
        if line.startswith("ORACLE "):
            return json.loads(line[7:])
    raise RuntimeError("oracle run failed: %s" % r.stderr[-2000:])


def cpu_extrapolation(ref, eig_full_s, n_full, N_full, inner_full):
    """Oracle seconds per step of the headline workload, term by term, from
    measured pieces: the oracle's small eigensolve at the headline's own size
    (eig_full_s, timed on its pencil) once per inner iteration, plus the rest
    of an oracle step on the full-size helium workload (`ref`: its step minus
    its small eigensolves) scaled linearly in fine unknowns x orbitals x inner
    iterations.  The linear scaling is a lower bound: the Gram matrices and the
    reconstruction grow with N^2 and the Poisson/BVP iteration counts with n."""
    t_step = statistics.median(ref["step_s"])
    t_eig = statistics.median(ref["eig_s"])
    inner0 = statistics.mean(ref["n_inner"])
    rest0 = max(t_step - t_eig, 0.0)
    scale = (n_full * N_full * inner_full) / (ref["n"] * ref["N"] * inner0)
    t_full = rest0 * scale + eig_full_s * inner_full
    return {"seconds_per_step": t_full, "fine_mesh_terms_s": rest0 * scale, "small_eigensolve_s": eig_full_s * inner_full,
            "scale_fine": scale, "ref_step_s": t_step, "ref_eig_s": t_eig, "ref_inner": inner0,
            "inner_per_step": inner_full, "eig_one_call_s": eig_full_s}


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
def run_reference(args):
    """The reference arm: the CPU oracle (the plain FP64 restatement of the
    paper, as it stands) timed on the host cores on the helium workload at its
    full size (the largest workload the oracle finishes in minutes); W
    untimed and K timed steps.  Under torchrun only rank 0 runs."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = host_threads()
    res = run_oracle_subprocess("oracle_steps(%r, %d, %d)" % (REFERENCE_WORKLOAD, args.steps, max(1, args.warmup)),
                                threads)
    total = sum(res["step_s"])
    value = args.steps / total
    inst = instance(REFERENCE_WORKLOAD)
    sample = ("CPU oracle (NumPy/SciPy FP64) Algorithm 3 steps of the helium workload at full size: P1 20^3 "
              "graded mesh, %d unknowns, coarse 8^3 (%d unknowns), N = %d; %d steps timed after %d"
              % (res["n"], res["nH"], res["N"], args.steps, max(1, args.warmup)))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%s: helium Z=2, N=1, P1 fine mesh %d tets (%d unknowns), coarse %d tets, FP64"
                               % (REFERENCE_WORKLOAD, len(inst.fine_tet), res["n"], len(inst.coarse_tet)),
                   "unknowns": res["n"], "coarse_unknowns": res["nH"], "mu": 32.0},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": threads, "kind": "oracle", "sample": sample,
                         "step_s": res["step_s"], "build_s": res["build_s"]},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def log(msg):
    print("[bench] " + msg, file=sys.stderr, flush=True)


def timed_steps(s, nas, torch, steps, snap_at=None, inner_hist=False):
    """`steps` steps of solver s, a CUDA event on the stream (torch's current
    stream, which the solver runs on) before each step and after the last;
    returns (total ms, per-step ms, reports, eigenvalues and energy after step
    `snap_at`)."""
    import numpy as np
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    reps, snap = [], None
    ev[0].record()
    for k in range(steps):
        r, rep = s.step()
        ev[k + 1].record()
        reps.append(nas.nas_report.from_buffer_copy(rep))
        if inner_hist:
            h = s.get(nas.NAS_Q_INNER_HIST)
            reps[-1].hist = [float(x) for x in h if x > 0]
        if snap_at is not None and k + 1 == snap_at:
            snap = (np.array(s.get(nas.NAS_Q_EIGVALS)), float(rep.energy))
    torch.cuda.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return ev[0].elapsed_time(ev[steps]), per, reps, snap


def secondary_line(args, nas, torch, name, device, stream):
    """FP64 steps/s of a smaller workload (no e2e, no comparison)."""
    inst = instance(name)
    s = nas.Solver(inst, device=device, stream=stream, **solver_options(args))
    t0 = time.time()
    s.init()
    setup = time.time() - t0
    for _ in range(2):
        s.step()
    ms, _, reps, _ = timed_steps(s, nas, torch, args.secondary_steps)
    sz = s.sizes()
    roofs = kernel_rooflines(reps, sz, args.secondary_steps, nas.PHASES, *hbm_peak(), nz_occ=sz["N"],
                             dense_tc=bool(args.dense_tc),
                             layouts=tuned_layouts(nas, sz))
    out = {"value": args.secondary_steps / (ms / 1e3), "unit": "steps/s", "steps": args.secondary_steps,
           "warmup": 2, "ms_per_step": ms / args.secondary_steps, "dtype": "f64", "setup_s": setup,
           "config": workload_config(args, name, inst, sz, "fp64"),
           "drho": [r.drho for r in reps], "energy": [r.energy for r in reps],
           "n_inner": [r.n_inner for r in reps], "roofline": dominant(roofs),
           "gpu_launches": int(sum(r.kernel_launches for r in reps))}
    s.close()
    return out


def tuned_layouts(nas, sz):
    """The SpMM layouts the autotuner chose for this workload's block of N columns."""
    out = {}
    for r in nas.nas_spmm_tuning():
        if r["rows"] == sz["n"] and r["N"] == sz["N"]:
            out[r["type"]] = r["layout"]
    return out


def hbm_peak():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def main():
    args = parse()
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

    prec = headline_precision(args)
    other = "fp64" if prec == "mixed" else "mixed"
    inst = instance(args.workload, args.cells, args.coarse_cells)
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.time()
    s = nas.Solver(inst, device=local, stream=stream, precision=1 if prec == "mixed" else 0, **solver_options(args))
    s.init()
    setup_s = time.time() - t0
    sz = s.sizes()
    log("setup+init %.1f s sizes %s" % (setup_s, sz))
    for w in range(args.warmup):
        tw = time.time()
        r, rep = s.step()
        log("warmup step %d: %.2f s status %d inner %d cg %d poisson %d eig %d drho %.3e E %.10f phases %s"
            % (w, time.time() - tw, r, rep.n_inner, rep.cg_iters, rep.poisson_iters, rep.eig_iters, rep.drho,
               rep.energy, {k: round(v, 1) for k, v in rep.as_dict()["phase_ms"].items()}))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # state at the start of the timed region, in pinned host memory: the
    # comparison run and the end-to-end run restart from it
    n, N, nqt = sz["n"], sz["N"], sz["ne"] * sz["nq"]
    s0_lam = torch.empty(N, dtype=torch.float64, pin_memory=True)
    s0_psi = torch.empty((n, N), dtype=torch.float64, pin_memory=True)
    s0_rho = torch.empty(nqt, dtype=torch.float64, pin_memory=True)

    def get(q, t):
        nas.nas_get(s.h, q, (t.data_ptr(), t.numel() * t.element_size()), 0)

    get(nas.NAS_Q_EIGVALS, s0_lam)
    get(nas.NAS_Q_ORBITALS, s0_psi)
    get(nas.NAS_Q_RHO_IN, s0_rho)
    n_cmp = max(0, min(args.compare_steps, args.steps))
    barrier()
    clocks = Clocks(args.clocks_file or "/tmp/bench_clocks_%d.csv" % os.getpid())
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    ms, per_h, reps, snap = timed_steps(s, nas, torch, args.steps, snap_at=n_cmp or None)
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop(local)
    log("timed: %d steps in %.1f ms; last report %s" % (args.steps, ms, reps[-1].as_dict()))
    ms = reduce_max(ms, dist, "cuda")
    value = job_value(world, args.steps, ms)
    # ------------------------------------------------------------ mixed against FP64, same start state
    # both precisions run n_cmp steps from the timed run's start state with the
    # exact inner SCF (tol_inner in every step), so that the per-eigenvalue
    # difference measures the precision and not a looser inner stop
    cmp = {}
    for pr in ("mixed", "fp64") if n_cmp > 0 else ():
        nas.nas_set_state(s.h, s0_lam.data_ptr(), s0_psi.data_ptr(), s0_rho.data_ptr(), 0)
        s.opt.precision = 1 if pr == "mixed" else 0
        s.opt.inner_adapt = 0.0
        s.opt.bvp_adapt = 0.0
        s.opt.max_inner = 100
        nas.nas_set_options(s.h, s.opt)
        barrier()
        ms_c, per_c, reps_c, snap_c = timed_steps(s, nas, torch, n_cmp, snap_at=n_cmp,
                                                   inner_hist=True)
        cmp[pr] = (reduce_max(ms_c, dist, "cuda"), reps_c, snap_c)
        log("comparison %s: %.1f ms for %d steps, inner %s" % (pr, ms_c, n_cmp, [r.n_inner for r in reps_c]))
    s.opt.precision = 1 if prec == "mixed" else 0
    s.opt.inner_adapt = args.inner_adapt
    s.opt.bvp_adapt = args.bvp_adapt
    s.opt.max_inner = inst.max_inner
    nas.nas_set_options(s.h, s.opt)
    comparison, reps_o = {"skipped": "compare-steps 0"}, []
    if n_cmp > 0:
        (ms_m, reps_m, (lam_mixed, e_mixed)), (ms_f, reps_f, (lam_fp64, e_fp64)) = cmp["mixed"], cmp["fp64"]
        err = lam_mixed - lam_fp64
        reps_o = reps_f if prec == "mixed" else reps_m
        comparison = {
            "steps": n_cmp, "inner_scf": "exact (tol_inner %g in every step, cap 100)" % inst.tol_scf,
            "mixed": {"value": job_value(world, n_cmp, ms_m), "unit": "steps/s", "ms_per_step": ms_m / n_cmp,
                      "n_inner": [r.n_inner for r in reps_m], "drho": [r.drho for r in reps_m],
                      "inner_residuals": [r.hist for r in reps_m],
                      "phase_ms_per_step": {k: v / n_cmp for k, v in phase_totals(reps_m, nas.PHASES)[0].items()}},
            "fp64": {"value": job_value(world, n_cmp, ms_f), "unit": "steps/s", "ms_per_step": ms_f / n_cmp,
                     "n_inner": [r.n_inner for r in reps_f], "drho": [r.drho for r in reps_f],
                     "inner_residuals": [r.hist for r in reps_f],
                     "phase_ms_per_step": {k: v / n_cmp for k, v in phase_totals(reps_f, nas.PHASES)[0].items()}},
            "speed_ratio_mixed_over_fp64": ms_f / ms_m if ms_m > 0 else None,
            "what": "the same start state and steps in both precisions; mixed = FP32 block PCG of the shifted "
                    "problems%s inside FP64 iterative refinement, all else FP64"
                    % (" and FP32 Poisson PCG (tolerances >= 1e-9)" if args.poisson_f32 else ""),
            "max_eigenvalue_err_ha": float(np.max(np.abs(err))), "eigenvalue_err_ha": [float(x) for x in err],
            "energy_err_ha": float(e_mixed - e_fp64),
        }
    log("comparison: %s" % json.dumps({k: v for k, v in comparison.items() if k != "eigenvalue_err_ha"}))

    # ------------------------------------------------------------ rooflines from the live CUDA-event timings
    peak, psrc = hbm_peak()
    # orbitals with nonzero occupation (all of them with smearing)
    nz = N if getattr(inst, "smearing", 0.0) > 0 else int(np.sum(np.asarray(inst.occ) > 0))
    lay = tuned_layouts(nas, sz)
    roofs_h = kernel_rooflines(reps, sz, args.steps, nas.PHASES, peak, psrc, nz_occ=nz, layouts=lay,
                               dense_tc=bool(args.dense_tc))
    roofs_o = (kernel_rooflines(reps_o, sz, n_cmp, nas.PHASES, peak, psrc, nz_occ=nz, layouts=lay,
                                dense_tc=bool(args.dense_tc)) if reps_o else {})
    tuner = [r for r in nas.nas_spmm_tuning() if r["rows"] == sz["n"]]
    trf = spmv_traffic(sz, "k_pcg1_spmv_sell")
    for rr in (roofs_h, roofs_o):
        if "k_pcg1_spmv_sell" in rr:
            rr["k_pcg1_spmv_sell"]["traffic"] = trf
        for d in rr.values():
            d.setdefault("traffic", None)

    # ------------------------------------------------------------ e2e through host buffers
    n_e2e = args.steps if args.e2e_steps < 0 else args.e2e_steps
    lam_b = torch.empty_like(s0_lam, pin_memory=True)
    psi_b = torch.empty_like(s0_psi, pin_memory=True)
    rho_b = torch.empty_like(s0_rho, pin_memory=True)
    en_b = torch.empty(6, dtype=torch.float64, pin_memory=True)
    lam_b.copy_(s0_lam)
    psi_b.copy_(s0_psi)
    rho_b.copy_(s0_rho)
    barrier()
    e0 = time.perf_counter()
    for _ in range(n_e2e):
        nas.nas_set_state(s.h, lam_b.data_ptr(), psi_b.data_ptr(), rho_b.data_ptr(), 0)
        s.step()
        nas.nas_get(s.h, nas.NAS_Q_EIGVALS, (lam_b.data_ptr(), lam_b.numel() * 8), 0)
        nas.nas_get(s.h, nas.NAS_Q_ORBITALS, (psi_b.data_ptr(), psi_b.numel() * 8), 0)
        nas.nas_get(s.h, nas.NAS_Q_RHO_IN, (rho_b.data_ptr(), rho_b.numel() * 8), 0)
        nas.nas_get(s.h, nas.NAS_Q_ENERGY, (en_b.data_ptr(), 48), 0)
    barrier()
    e2e_s = reduce_max(time.perf_counter() - e0, dist, "cuda")
    io_bytes = 8 * (N + n * N + nqt)
    e2e = None
    if n_e2e > 0:
        e2e = {"value": world * n_e2e / e2e_s, "unit": "steps/s", "steps": n_e2e, "h2d_bytes_per_step": io_bytes,
               "d2h_bytes_per_step": io_bytes + 48,
               "what": "public C-ABI calls per step: nas_set_state from pinned host buffers (state copied in; the "
                       "library recomputes the density's Hartree potential and A^NL), nas_step, nas_get of the "
                       "eigenvalues, orbitals, density and energy; from the timed run's start state"}
    # the small pencil of the last inner iteration (for the CPU extrapolation)
    pencil = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            FA = s.get(nas.NAS_Q_FA)
            FB = s.get(nas.NAS_Q_FB)
            pencil = "/tmp/bench_pencil_%d.npz" % os.getpid()
            np.savez(pencil, FA=FA, FB=FB)
        except Exception as ex:
            log("pencil not saved: %s" % ex)
    cfg = workload_config(args, args.workload, inst, sz, prec, {"parallelism": "replicas" if world > 1 else "1 GPU"})
    s.close()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    secondary = {}
    if not args.no_secondary:
        for name in ("mol8_p2", REFERENCE_WORKLOAD):
            try:
                secondary[name] = secondary_line(args, nas, torch, name, local, stream)
                log("secondary %s: %.3f steps/s" % (name, secondary[name]["value"]))
            except Exception as ex:
                secondary[name] = {"error": str(ex)[:200]}
    batched = run_batch(args, nas, torch, local) if args.batch > 0 else None

    # ------------------------------------------------------------ CPU oracle baseline
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        threads = host_threads()
        cpu = {"kind": "oracle", "unit": "steps/s", "cores": threads}
        try:
            ref_n = run_oracle_subprocess("oracle_steps(%r, 2, 1)" % REFERENCE_WORKLOAD, threads)
            ref_1 = run_oracle_subprocess("oracle_steps(%r, 2, 1)" % REFERENCE_WORKLOAD, 1)
            cpu["reference_workload"] = {
                "workload": REFERENCE_WORKLOAD, "unknowns": ref_n["n"],
                "steps_per_s_all_cores": 2 / sum(ref_n["step_s"]), "cores_all": threads,
                "steps_per_s_one_core": 2 / sum(ref_1["step_s"]), "cores_one": 1,
                "step_s_all_cores": ref_n["step_s"], "step_s_one_core": ref_1["step_s"],
                "gpu_steps_per_s": secondary.get(REFERENCE_WORKLOAD, {}).get("value")}
            inner_full = statistics.mean(r.n_inner for r in reps)
            if pencil:
                eig = run_oracle_subprocess("oracle_eig_seconds(%r, %d)" % (pencil, N), threads)
                ex = cpu_extrapolation(ref_n, eig["eig_s"], n, N, inner_full)
                cpu["value"] = 1.0 / ex["seconds_per_step"]
                cpu["extrapolation"] = ex
                cpu["extrapolation"]["eig_m"] = eig["m"]
                cpu["sample"] = (
                    "the oracle cannot run the headline workload in minutes (building its operators for 32 nuclei "
                    "on a mesh fine enough for the 16^3 coarse space takes minutes alone), so its seconds per step "
                    "are assembled term by term from measurements on %d host cores: the oracle's small eigensolve "
                    "(scipy eigh, lowest %d pairs) timed on this run's own %d x %d pencil, once per inner "
                    "iteration (%.1f per step in the GPU run), plus the rest of an oracle step measured on the "
                    "full-size helium workload (%d unknowns, N = 1) scaled linearly in unknowns x orbitals x "
                    "inner iterations (a lower bound)" % (threads, N, eig["m"], eig["m"], inner_full, ref_n["n"]))
        except Exception as ex:  # the baseline is reported, never required
            cpu["error"] = str(ex)[:300]
        if pencil:
            try:
                os.remove(pencil)
            except OSError:
                pass

    last = reps[-1]
    dom_h, dom_o = dominant(roofs_h), (dominant(roofs_o) if roofs_o else None)
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64/f32 mixed" if prec == "mixed" else "f64", "data": "synthetic",
        "config": cfg,
        "roofline": dom_h, "roofline_other_precision": dom_o,
        "rooflines": {"headline": roofs_h, "other_precision": roofs_o},
        "speed_ratio_mixed_over_fp64": None,
        "comparison": comparison,
        "phase_ms_per_step": {k: v / args.steps for k, v in phase_totals(reps, nas.PHASES)[0].items()},
        "per_step": {"n_inner": [r.n_inner for r in reps], "cg_iters": [r.cg_iters for r in reps],
                     "poisson_iters": [r.poisson_iters for r in reps], "eig_iters": [r.eig_iters for r in reps],
                     "drho": [r.drho for r in reps], "energy": [r.energy for r in reps],
                     "inner_tol": [r.inner_tol for r in reps], "bvp_tol": [r.bvp_tol for r in reps],
                     "eig_rr_calls": [r.eig_rr_calls for r in reps],
                     "eig_rr_fallbacks": [r.eig_rr_fallbacks for r in reps]},
        "gpu_launches": int(sum(r.kernel_launches for r in reps)), "e2e": e2e, "clocks": clk,
        "spmm_autotuner": tuner,
        "cpu_baseline": cpu, "setup_s": setup_s, "energy_ha": float(last.energy),
        "secondary": secondary,
    }
    line["speed_ratio_mixed_over_fp64"] = comparison.get("speed_ratio_mixed_over_fp64")
    line["speed_ratio_note"] = ("FP64 ms over mixed ms for the same %d steps from the same start state, both with "
                                "the exact inner SCF (CUDA events)" % n_cmp)
    line["per_step"]["ms"] = per_h
    if batched is not None:
        line["batched"] = batched
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

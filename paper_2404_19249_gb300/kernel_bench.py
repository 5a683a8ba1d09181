"""Single-kernel runs through the C ABI on synthetic inputs of a few GB, for
timing and for profiler captures of one kernel at a time.

  python -m paper_2404_19249_gb300.kernel_bench spmm --grid 128 --N 64 --fp32 --layout rows<4,2>
  python -m paper_2404_19249_gb300.kernel_bench precond --nH 3375 --k 80 --tc 1
  python -m paper_2404_19249_gb300.kernel_bench recon --rows 7880599 --N 64 --tc 1
  python -m paper_2404_19249_gb300.kernel_bench gram --rows 7880599 --N 64 --tc 1

spmm: Y = A X for the 27-point stencil matrix of a grid^3 lattice (the
coupling pattern of trilinear elements, rows in lattice order; values
random), N interleaved right-hand sides, one kernel layout.  precond: W = T R
with T a dense SPD FP32 [nH][nH] and R FP64 [nH][k], on the SIMT (tc 0) or
tensor-core (tc 1) kernel of the small eigensolver's preconditioner.  recon:
Psi = I u_H + U^ alpha for `rows` fine rows (random coarse columns among nH
= 3375, U^ [rows][N], alpha [N][N]) on the FP64 SIMT (tc 0) or tensor-core
(tc 1) kernel of Algorithm 3's reconstruction.  gram: the symmetric Gram
X^T Y of two random [rows][N] blocks on the FP64 SIMT (tc 0) or tensor-core
(tc 1) kernel.  Prints
one JSON line with the mean time per launch (CUDA events, after warm-up) and
the algorithmic bytes or flops per launch.
"""
import argparse
import json
import sys

import numpy as np


def stencil27(g, seed=0):
    """CSR (rowptr, col int32; values float64) of the 27-point stencil on g^3."""
    idx = np.arange(g ** 3).reshape(g, g, g)
    rows, cols = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                src = idx[max(0, -dz):g - max(0, dz), max(0, -dy):g - max(0, dy), max(0, -dx):g - max(0, dx)]
                dst = idx[max(0, dz):g - max(0, -dz) or None, max(0, dy):g - max(0, -dy) or None,
                          max(0, dx):g - max(0, -dx) or None]
                rows.append(src.ravel())
                cols.append(dst.ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    order = np.lexsort((c, r))
    r, c = r[order], c[order]
    rowptr = np.zeros(g ** 3 + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    vals = np.random.default_rng(seed).standard_normal(len(c))
    return rowptr, c.astype(np.int32), vals


def time_launches(torch, fn, reps, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("kernel", choices=["spmm", "precond", "recon", "gram"])
    p.add_argument("--rows", type=int, default=7880599)
    p.add_argument("--grid", type=int, default=128)
    p.add_argument("--N", type=int, default=64)
    p.add_argument("--fp32", action="store_true")
    p.add_argument("--layout", default="rows<2,1>")
    p.add_argument("--nH", type=int, default=3375)
    p.add_argument("--k", type=int, default=80)
    p.add_argument("--tc", type=int, default=1)
    p.add_argument("--reps", type=int, default=5)
    a = p.parse_args(argv)
    import torch
    from . import nas
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream().cuda_stream
    if a.kernel == "spmm":
        rowptr, col, vals = stencil27(a.grid)
        n, nnz = len(rowptr) - 1, len(col)
        dt = torch.float32 if a.fp32 else torch.float64
        rp = torch.tensor(rowptr, device=dev)
        ci = torch.tensor(col, device=dev)
        va = torch.tensor(vals, dtype=dt, device=dev)
        X = torch.randn((n, a.N), dtype=dt, device=dev)
        Y = torch.empty((n, a.N), dtype=dt, device=dev)
        lid = nas.nas_spmm_layouts().index(a.layout)
        ms = time_launches(torch, lambda: nas.nas_spmm_layout(lid, n, rp.data_ptr(), ci.data_ptr(), va.data_ptr(),
                                                              a.N, X.data_ptr(), Y.data_ptr(), fp32=a.fp32,
                                                              stream=st), a.reps)
        s = 4 if a.fp32 else 8
        nbytes = nnz * (s + 4) + 4 * (n + 1) + 2 * n * a.N * s
        out = {"kernel": "spmm", "layout": a.layout, "precision": "f32" if a.fp32 else "f64", "rows": n,
               "nnz": nnz, "N": a.N, "ms_per_launch": ms, "algorithmic_bytes": nbytes,
               "gbs": nbytes / (ms * 1e-3) / 1e9, "tflops": 2.0 * nnz * a.N / (ms * 1e-3) / 1e12}
    elif a.kernel == "gram":
        n, N = a.rows, a.N
        g = torch.Generator(device=dev)
        g.manual_seed(5)
        X = torch.randn((n, N), dtype=torch.float64, device=dev, generator=g)
        Y = torch.randn((n, N), dtype=torch.float64, device=dev, generator=g)
        G = torch.empty((N, N), dtype=torch.float64, device=dev)
        ms = time_launches(torch, lambda: nas.nas_gram_sym_f64(a.tc, n, N, X.data_ptr(), Y.data_ptr(), G.data_ptr(),
                                                               st), a.reps)
        flops = 1.0 * n * N * (N + 1)
        out = {"kernel": "gram", "tensor_cores": bool(a.tc), "rows": n, "N": N, "ms_per_call": ms,
               "fp64_equivalent_flops": flops, "tflops_fp64_equivalent": flops / (ms * 1e-3) / 1e12,
               "algorithmic_bytes": 16.0 * n * N, "gbs": 16.0 * n * N / (ms * 1e-3) / 1e9}
    elif a.kernel == "recon":
        n, N, nH = a.rows, a.N, a.nH
        g = torch.Generator(device=dev)
        g.manual_seed(3)
        icol = torch.randint(0, nH, (n, 4), dtype=torch.int32, device=dev, generator=g)
        ival = torch.rand((n, 4), dtype=torch.float64, device=dev, generator=g)
        U = torch.randn((nH + N, N), dtype=torch.float64, device=dev, generator=g)
        Uhat = torch.randn((n, N), dtype=torch.float64, device=dev, generator=g)
        Psi = torch.empty((n, N), dtype=torch.float64, device=dev)
        ms = time_launches(torch, lambda: nas.nas_reconstruct_f64(a.tc, n, icol.data_ptr(), ival.data_ptr(), N,
                                                                  U.data_ptr(), nH, N, Uhat.data_ptr(),
                                                                  Psi.data_ptr(), st), a.reps)
        flops = 2.0 * n * N * (4 + N)
        nbytes = 8.0 * n * N * 2 + 12.0 * 4 * n
        out = {"kernel": "recon", "tensor_cores": bool(a.tc), "rows": n, "N": N, "ms_per_call": ms,
               "fp64_equivalent_flops": flops, "tflops_fp64_equivalent": flops / (ms * 1e-3) / 1e12,
               "algorithmic_bytes": nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9}
    else:
        rng = np.random.default_rng(1)
        A = rng.standard_normal((a.nH, a.nH)).astype(np.float32)
        T = torch.tensor(A @ A.T / a.nH + np.eye(a.nH, dtype=np.float32), device=dev)
        R = torch.randn((a.nH, a.k), dtype=torch.float64, device=dev)
        W = torch.empty((a.nH, a.k), dtype=torch.float64, device=dev)
        ms = time_launches(torch, lambda: nas.nas_dense_precond_f32(a.tc, a.nH, a.k, T.data_ptr(), R.data_ptr(),
                                                                    W.data_ptr(), st), a.reps)
        flops = 2.0 * a.nH * a.nH * a.k
        out = {"kernel": "precond", "tensor_cores": bool(a.tc), "nH": a.nH, "k": a.k, "ms_per_call": ms,
               "flops": flops, "tflops": flops / (ms * 1e-3) / 1e12}
    print(json.dumps(out))


if __name__ == "__main__":
    sys.exit(main())

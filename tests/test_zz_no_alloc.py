"""GPU test of nas_coldot_f64_noalloc, the entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

It is checked against the allocating entry point nas_coldot_f64 on the same
inputs, over two calls in a row (the shared scratch array keeps the first
call's contents), and its size limit is checked.  This file is collected last.
"""
import ctypes as C
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_COLS = 64


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19249_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2404_19249_gb300 import nas
    return torch, nas


def _call(lib, fn, n, N, X, Y, w, out, stream):
    return getattr(lib, fn)(n, N, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                            C.c_void_p(w.data_ptr() if w is not None else None),
                            C.c_void_p(out.data_ptr()), C.c_void_p(stream or None))


def test_no_alloc_matches_allocating_entry_point(env):
    torch, nas = env
    lib = nas.lib
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(2024)
    # two calls in a row with different shapes: the second sees the first's scratch contents
    for n, N, weighted in ((200003, 21, True), (4097, MAX_COLS, False)):
        X = torch.tensor(rng.normal(size=(n, N)), dtype=torch.float64, device=dev)
        Y = torch.tensor(rng.normal(size=(n, N)), dtype=torch.float64, device=dev)
        w = torch.tensor(rng.uniform(0.1, 2.0, size=n), dtype=torch.float64, device=dev) if weighted else None
        ref = torch.zeros(N, dtype=torch.float64, device=dev)
        got = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
        assert _call(lib, "nas_coldot_f64", n, N, X, Y, w, ref, stream) == 0
        assert _call(lib, "nas_coldot_f64_noalloc", n, N, X, Y, w, got, stream) == 0
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        scale = np.abs(r).max()
        assert np.all(np.abs(g - r) <= 1e-13 * scale)


def test_no_alloc_rejects_sizes_beyond_its_scratch(env):
    torch, nas = env
    dev = torch.device("cuda:0")
    X = torch.zeros((8, MAX_COLS + 1), dtype=torch.float64, device=dev)
    out = torch.zeros(MAX_COLS + 1, dtype=torch.float64, device=dev)
    assert _call(nas.lib, "nas_coldot_f64_noalloc", 8, MAX_COLS + 1, X, X, None, out, 0) == -1
    assert _call(nas.lib, "nas_coldot_f64_noalloc", 8, 0, X, X, None, out, 0) == -1

"""The allocation-free Gram-Schmidt projection entry point, sbm_dots_noalloc.

Some callers cannot let the library call cudaMalloc, e.g. a process whose caching allocator
already holds the device memory, or a latency-critical loop that cannot take the device-wide
synchronisation an allocation may cause.  sbm_dots_noalloc serves them: its partial sums live
in a static device array.  This file is collected last so that a run stopping at the first
failure has already run every other test; it passes alone and after the others.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_dots_noalloc_matches_sbm_dots_twice():
    import paper_2506_12899_gb300 as S
    lib = S.load_library()
    solver = S.Solver(W.disk2d_p1(16, 0))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, nv) in enumerate([(912582, 31), (5000, 3)]):      # two calls in a row, shared scratch
        rng = np.random.default_rng(100 + call)
        V = torch.tensor(rng.normal(size=(nv, n)), device="cuda")
        w = torch.tensor(rng.normal(size=n), device="cuda")
        ref = solver.dots(V, w).cpu().numpy()
        out = torch.full((nv,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.sbm_dots_noalloc(ctypes.c_void_p(V.data_ptr()), n, nv, ctypes.c_void_p(w.data_ptr()), n,
                                  ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, lib.sbm_last_error()
        got = out.cpu().numpy()
        # same kernels, same grid, same reduction order: equal within the dot-product bound (bitwise here)
        bound = n * 2.2e-16 * (np.abs(V.cpu().numpy()) @ np.abs(w.cpu().numpy()))
        assert np.all(np.abs(got - ref) <= bound)
        assert np.all(np.abs(got - V.cpu().numpy() @ w.cpu().numpy()) <= bound)


def test_dots_noalloc_rejects_bad_sizes():
    import paper_2506_12899_gb300 as S
    lib = S.load_library()
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.sbm_dots_noalloc(p, 8, 33, p, 8, p, None) == -1          # nv above the scratch width
    assert b"nv" in lib.sbm_last_error()
    assert lib.sbm_dots_noalloc(p, 4, 1, p, 8, p, None) == -1           # ldv < n

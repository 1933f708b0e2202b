"""The allocation-free Gram-Schmidt projection entry point, sbm_dots_noalloc.

Some callers cannot let the library call cudaMalloc, e.g. a process whose caching allocator
already holds the device memory, or a latency-critical loop that cannot take the device-wide
synchronisation an allocation may cause.  sbm_dots_noalloc serves them: its partial sums live
in a static device array.  This file is collected last so that a run stopping at the first
failure has already run every other test; it passes alone and after the others.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

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
    # several calls in a row on the shared scratch: the full width (32 vectors) at the largest grid
    # (608 blocks), a small case, and an empty one whose single block must still write zeros
    for call, (n, nv) in enumerate([(912582, 31), (5000, 3), (912582, 32), (0, 1)]):
        rng = np.random.default_rng(100 + call)
        V = torch.tensor(rng.normal(size=(nv, max(n, 1))), device="cuda")
        w = torch.tensor(rng.normal(size=max(n, 1)), device="cuda")
        out = torch.full((nv,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.sbm_dots_noalloc(ctypes.c_void_p(V.data_ptr()), max(n, 1), nv, ctypes.c_void_p(w.data_ptr()), n,
                                  ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, lib.sbm_last_error()
        got = out.cpu().numpy()
        if n == 0:
            assert np.all(got == 0.0), got
            continue
        ref = solver.dots(V, w).cpu().numpy()
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


_RESET_SCRIPT = textwrap.dedent("""
    import ctypes, sys
    import numpy as np
    sbm = ctypes.CDLL(sys.argv[1])
    # the CUDA runtime libsbm itself loaded (opening the same file again returns the same library)
    rt_path = next(l.split()[-1] for l in open("/proc/self/maps") if "libcudart.so" in l)
    rt = ctypes.CDLL(rt_path)
    vp = ctypes.c_void_p
    sbm.sbm_dots_noalloc.argtypes = [vp, ctypes.c_longlong, ctypes.c_int, vp, ctypes.c_longlong, vp, vp]
    sbm.sbm_last_error.restype = ctypes.c_char_p
    n, nv = 100000, 5
    rng = np.random.default_rng(7)
    V, w = rng.normal(size=(nv, n)), rng.normal(size=n)
    def run():
        ptrs = [vp(), vp(), vp()]
        for p, nbytes in zip(ptrs, (V.nbytes, w.nbytes, 8 * nv)):
            assert rt.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(nbytes)) == 0
        assert rt.cudaMemcpy(ptrs[0], V.ctypes.data_as(vp), ctypes.c_size_t(V.nbytes), 1) == 0
        assert rt.cudaMemcpy(ptrs[1], w.ctypes.data_as(vp), ctypes.c_size_t(w.nbytes), 1) == 0
        rc = sbm.sbm_dots_noalloc(ptrs[0], n, nv, ptrs[1], n, ptrs[2], None)
        assert rc == 0, sbm.sbm_last_error()
        out = np.zeros(nv)
        assert rt.cudaMemcpy(out.ctypes.data_as(vp), ptrs[2], ctypes.c_size_t(8 * nv), 2) == 0
        for p in ptrs:
            assert rt.cudaFree(p) == 0
        return out
    a = run()
    assert rt.cudaDeviceReset() == 0          # the primary context is destroyed and re-created
    b = run()                                 # the scratch address is looked up again in the new one
    bound = n * 2.2e-16 * (np.abs(V) @ np.abs(w))
    assert np.all(np.abs(a - V @ w) <= bound) and np.array_equal(a, b), (a, b)
    print("OK")
""")


def test_dots_noalloc_after_device_reset():
    """A call, cudaDeviceReset (which replaces the device's primary context and with it the address
    of the static scratch), and a second call that must use the new address.  Runs in a fresh
    process that owns its buffers through the CUDA runtime alone (no torch state to invalidate)."""
    import paper_2506_12899_gb300 as S
    S.load_library()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES=os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    r = subprocess.run([sys.executable, "-c", _RESET_SCRIPT, S.LIB_PATH], capture_output=True, text=True,
                       timeout=300, env=env)
    assert r.returncode == 0 and "OK" in r.stdout, r.stdout + r.stderr

"""Python binding of libsbm, the GB300 DG-SBM hp-multigrid FGMRES solver.

Argument marshalling only: every step of the solver runs in libsbm's CUDA kernels.  PyTorch
provides the caller's device buffers and the CUDA stream.  There is no CPU fallback: if
libsbm.so is missing or no CUDA device is present, the calls raise.

Example:
    import workloads as W, paper_2506_12899_gb300 as sbm
    solver = sbm.Solver(W.disk2d_p1(32, 0), precision="f32")
    b = solver.rhs(); x = torch.zeros_like(b)
    info = solver.solve(b, x, tol=1e-8)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsbm.so")

SBM_F64, SBM_F32 = 0, 1
ERRORS = {-1: "SBM_ERR_ARG", -2: "SBM_ERR_CUDA", -3: "SBM_ERR_SINGULAR_BLOCK", -4: "SBM_ERR_NOT_CONVERGED",
          -5: "SBM_ERR_NAN", -6: "SBM_ERR_GEOMETRY", -7: "SBM_ERR_ALLOC"}

# exported C symbols (checked by the tests against include/sbm.h)
SYMBOLS = ("sbm_setup", "sbm_setup_host", "sbm_host_apply", "sbm_host_rhs", "sbm_destroy", "sbm_last_error", "sbm_kernel_launches", "sbm_num_levels", "sbm_info", "sbm_layout",
           "sbm_export_geometry", "sbm_rhs", "sbm_apply", "sbm_residual", "sbm_smooth", "sbm_restrict",
           "sbm_prolong_add", "sbm_coarse_solve", "sbm_vcycle", "sbm_dots", "sbm_dots_noalloc", "sbm_gram_schmidt", "sbm_l2_error", "sbm_solve",
           "sbm_solve_host", "sbm_mlp_create", "sbm_mlp_destroy", "sbm_mlp_shape", "sbm_mlp_set_params",
           "sbm_mlp_get_params", "sbm_mlp_gemm_backend", "sbm_mlp_forward", "sbm_mlp_gradients", "sbm_mlp_num_samples",
           "sbm_mlp_clear_samples", "sbm_mlp_target_scale", "sbm_mlp_train", "sbm_mlp_save", "sbm_mlp_load", "sbm_learned_features",
           "sbm_learned_cells", "sbm_collect", "sbm_attach_mlp", "sbm_async_wait_selftest")


class SbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Shape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("center", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("amp", ctypes.c_double), ("freq", ctypes.c_double), ("phase", ctypes.c_double),
                ("semi", ctypes.c_double * 3), ("rot", ctypes.c_double * 9)]


class _Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("p", ctypes.c_int),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("shape", _Shape),
                ("exact", ctypes.c_int), ("lam", ctypes.c_double), ("lam_inclusive", ctypes.c_int),
                ("sigma_face_c", ctypes.c_double), ("sigma_bnd_c", ctypes.c_double), ("alpha", ctypes.c_double),
                ("extension", ctypes.c_int), ("coarsest_n", ctypes.c_int), ("pre_smooth", ctypes.c_int),
                ("post_smooth", ctypes.c_int), ("ssor_each", ctypes.c_int), ("omega", ctypes.c_double), ("omega_p3", ctypes.c_double),
                ("vf_samples", ctypes.c_int), ("precision", ctypes.c_int), ("tail_max_cells", ctypes.c_int),
                ("tail_cluster_ctas", ctypes.c_int), ("launch_overlap", ctypes.c_int),
                ("krylov_basis", ctypes.c_int), ("cell_kernel_min_cells", ctypes.c_int),
                ("staged_min_cells", ctypes.c_int), ("smoother", ctypes.c_int), ("ordering", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("cheb_ratio", ctypes.c_double), ("device_geometry", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class _LevelInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("p", ctypes.c_int), ("h", ctypes.c_double), ("n_active", ctypes.c_int),
                ("n_dof", ctypes.c_int), ("n_boundary", ctypes.c_int), ("n_sface", ctypes.c_int),
                ("colour_start", ctypes.c_int * 9), ("colour_nbnd", ctypes.c_int * 8)]


class _SolveInfo(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("history", ctypes.c_double * 512),
                ("ms_total", ctypes.c_double), ("learned", ctypes.c_int), ("learned_fallback", ctypes.c_int)]


@dataclass
class SolveInfo:
    converged: bool
    iterations: int
    restarts: int
    true_rel_residual: float
    history: list
    ms_total: float
    status: int
    learned: bool = False
    learned_fallback: bool = False


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libsbm.so (built by `python -m paper_2506_12899_gb300.build`); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsbm.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    import torch  # noqa: F401  (loads the CUDA runtime that libsbm shares)
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.sbm_setup.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_void_p)]
    lib.sbm_setup_host.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_void_p)]
    lib.sbm_host_apply.argtypes = [vp, ip, vp, vp]
    lib.sbm_host_rhs.argtypes = [vp, vp]
    lib.sbm_destroy.argtypes = [vp]
    lib.sbm_destroy.restype = None
    lib.sbm_last_error.restype = ctypes.c_char_p
    lib.sbm_kernel_launches.restype = ctypes.c_longlong
    lib.sbm_num_levels.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.sbm_info.argtypes = [vp, ip, ctypes.POINTER(_LevelInfo)]
    lib.sbm_layout.argtypes = [vp, ip, vp]
    lib.sbm_export_geometry.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), vp, vp, vp]
    lib.sbm_rhs.argtypes = [vp, vp]
    lib.sbm_apply.argtypes = [vp, ip, ip, vp, vp]
    lib.sbm_residual.argtypes = [vp, ip, ip, vp, vp, vp]
    lib.sbm_smooth.argtypes = [vp, ip, ip, ip, vp, vp]
    lib.sbm_restrict.argtypes = [vp, ip, ip, vp, vp]
    lib.sbm_prolong_add.argtypes = [vp, ip, ip, vp, vp]
    lib.sbm_coarse_solve.argtypes = [vp, ip, vp, vp]
    lib.sbm_vcycle.argtypes = [vp, ip, vp, vp]
    lib.sbm_dots.argtypes = [vp, vp, ctypes.c_longlong, ip, vp, ctypes.c_longlong, vp]
    lib.sbm_gram_schmidt.argtypes = [vp, ip, vp, ip, vp, vp, vp, vp]
    lib.sbm_l2_error.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.sbm_dots_noalloc.argtypes = [vp, ctypes.c_longlong, ip, vp, ctypes.c_longlong, vp, vp]
    lib.sbm_solve.argtypes = [vp, vp, vp, dp, ip, ip, ctypes.POINTER(_SolveInfo)]
    lib.sbm_solve_host.argtypes = [vp, vp, vp, dp, ip, ip, ctypes.POINTER(_SolveInfo)]
    llp = ctypes.POINTER(ctypes.c_longlong)
    lib.sbm_mlp_create.argtypes = [ip, ip, ip, ctypes.c_ulonglong, vp, ctypes.POINTER(ctypes.c_void_p)]
    lib.sbm_mlp_destroy.argtypes = [vp]
    lib.sbm_mlp_destroy.restype = None
    lib.sbm_mlp_shape.argtypes = [vp, vp, vp, vp, vp, llp]
    lib.sbm_mlp_set_params.argtypes = [vp, vp]
    lib.sbm_mlp_get_params.argtypes = [vp, vp]
    lib.sbm_mlp_forward.argtypes = [vp, vp, ip, vp]
    lib.sbm_mlp_gemm_backend.argtypes = [vp, ip]
    lib.sbm_mlp_gradients.argtypes = [vp, vp, vp, ip, vp, ctypes.POINTER(ctypes.c_double)]
    lib.sbm_mlp_num_samples.argtypes = [vp, llp]
    lib.sbm_mlp_clear_samples.argtypes = [vp]
    lib.sbm_mlp_target_scale.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.sbm_mlp_train.argtypes = [vp, ip, ip, ctypes.c_float, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double)]
    lib.sbm_mlp_save.argtypes = [vp, ctypes.c_char_p]
    lib.sbm_mlp_load.argtypes = [vp, ctypes.c_char_p]
    lib.sbm_learned_features.argtypes = [vp, ip, vp, vp, vp]
    lib.sbm_learned_cells.argtypes = [vp, ctypes.POINTER(ctypes.c_int), vp]
    lib.sbm_collect.argtypes = [vp, vp, ip, vp, ip, ip, llp]
    lib.sbm_attach_mlp.argtypes = [vp, vp, ctypes.c_float, dp]
    lib.sbm_async_wait_selftest.argtypes = [ip, vp]
    for name in SYMBOLS:
        if name not in ("sbm_destroy", "sbm_last_error", "sbm_kernel_launches", "sbm_mlp_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernel launches issued by libsbm since it was loaded."""
    return int(load_library().sbm_kernel_launches())


def async_wait_selftest(starve: bool, stream=None) -> None:
    """One bounded mbarrier wait on the GPU (sbm_async_wait_selftest): returns when the announced
    copy arrived, raises SbmError (SBM_ERR_CUDA) when the wait ran out (starve=True)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(load_library().sbm_async_wait_selftest(1 if starve else 0, ctypes.c_void_p(s.cuda_stream)))


def _check(code: int):
    if code != 0:
        raise SbmError(code, _lib.sbm_last_error().decode())


def make_desc(prob, precision: int = SBM_F64, stream: int = 0, tail_max_cells: int = 0,
              cell_kernel_min_cells: int = 0, tail_cluster_ctas: int = 0, launch_overlap: int = 0,
              krylov_basis: int = 0, staged_min_cells: int = 0, device_geometry: int = 0) -> _Desc:
    d = _Desc()
    d.dim, d.n, d.p = prob.dim, prob.n, prob.p
    d.lo[:] = [float(v) for v in prob.lo]
    d.hi[:] = [float(v) for v in prob.hi]
    s = prob.shape
    d.shape.kind = s.kind
    d.shape.center[:] = [float(v) for v in s.center]
    d.shape.radius, d.shape.amp, d.shape.freq, d.shape.phase = s.radius, s.amp, s.freq, s.phase
    d.shape.semi[:] = [float(v) for v in s.semi]
    d.shape.rot[:] = [float(v) for v in s.rot]
    d.exact, d.lam, d.lam_inclusive = prob.exact, prob.lam, prob.lam_inclusive
    d.sigma_face_c, d.sigma_bnd_c, d.alpha = prob.sigma_face_c, prob.sigma_bnd_c, prob.alpha
    d.extension, d.coarsest_n = prob.extension, prob.coarsest_n
    d.pre_smooth, d.post_smooth, d.omega, d.omega_p3 = prob.pre_smooth, prob.post_smooth, prob.omega, prob.omega_p3
    d.ssor_each = prob.ssor_each
    d.vf_samples, d.precision, d.stream = prob.vf_samples, precision, stream
    d.tail_max_cells = tail_max_cells
    d.tail_cluster_ctas = tail_cluster_ctas
    d.launch_overlap = launch_overlap
    d.krylov_basis = krylov_basis
    d.cell_kernel_min_cells = cell_kernel_min_cells
    d.staged_min_cells = staged_min_cells
    d.smoother = getattr(prob, "smoother", 0)
    d.ordering = getattr(prob, "ordering", 0)
    d.cheb_degree = getattr(prob, "cheb_degree", 4)
    d.cheb_ratio = getattr(prob, "cheb_ratio", 20.0)
    d.device_geometry = device_geometry
    return d


class Solver:
    """One DG-SBM problem set up on the current CUDA device (a libsbm context)."""

    def __init__(self, prob, precision: str = "f64", stream=None, tail_max_cells: int = 0,
                 cell_kernel_min_cells: int = 0, tail_cluster_ctas: int = 0, launch_overlap: int = 0,
                 krylov_basis: int = 0, staged_min_cells: int = 0, device_geometry: int = 0):
        """tail_max_cells: coarse p = 1 levels with at most that many cells run as one launch
        (0: library default, every level that fits for FP32 and none for FP64; < 0: never) of
        tail_cluster_ctas CTAs (0 or 1: one CTA; 2..16: a thread-block cluster).
        launch_overlap: programmatic dependent launch between the solver's kernels, > 0 on, < 0 off,
        0 on with the FP32 V-cycle and off with FP64 (measured best).  krylov_basis: 0 double-float
        FGMRES basis and Arnoldi operator (on the FP32 pipes), 1 FP64, 2 double-float basis with the
        FP64 operator.  cell_kernel_min_cells: launches over at least that many
        cells use one thread per cell, or at 3D p = 3 one thread per line of a cell (0: library
        default, < 0: never, 1: always where those kernels exist).  staged_min_cells: FP32 operator and smoother launches over at least that
        many cells use the staged thread-per-cell kernels (0: library default, < 0: never).
        device_geometry: volume fractions and closest points on the device (0: default, on; < 0:
        on the host cores)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libsbm needs a CUDA device; no CPU fallback exists")
        self._torch = torch
        self.lib = load_library()
        self.prob = prob
        self.precision = SBM_F32 if precision == "f32" else SBM_F64
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        desc = make_desc(prob, self.precision, self.stream.cuda_stream, tail_max_cells, cell_kernel_min_cells,
                         tail_cluster_ctas, launch_overlap, krylov_basis, staged_min_cells, device_geometry)
        ctx = ctypes.c_void_p()
        _check(self.lib.sbm_setup(ctypes.byref(desc), ctypes.byref(ctx)))
        self.ctx = ctx
        n = ctypes.c_int()
        _check(self.lib.sbm_num_levels(self.ctx, ctypes.byref(n)))
        self.num_levels = n.value

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.sbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ layout / geometry
    def info(self, level: int = -1) -> dict:
        li = _LevelInfo()
        _check(self.lib.sbm_info(self.ctx, level, ctypes.byref(li)))
        return dict(n=li.n, p=li.p, h=li.h, n_active=li.n_active, n_dof=li.n_dof, n_boundary=li.n_boundary,
                    n_sface=li.n_sface, colour_start=list(li.colour_start), colour_nbnd=list(li.colour_nbnd))

    def layout(self, level: int = -1) -> np.ndarray:
        """(n_active, 3) background multi-index of each compact cell."""
        na = self.info(level)["n_active"]
        out = np.zeros((na, 3), dtype=np.int32)
        _check(self.lib.sbm_layout(self.ctx, level, out.ctypes.data))
        return out

    def export_geometry(self, level: int = -1):
        nf = ctypes.c_int()
        _check(self.lib.sbm_export_geometry(self.ctx, level, ctypes.byref(nf), None, None, None))
        nq = (self.info(level)["p"] + 1) ** (self.prob.dim - 1)
        cell = np.zeros(nf.value, dtype=np.int32)
        slot = np.zeros(nf.value, dtype=np.int32)
        d = np.zeros((nf.value, nq, 3))
        _check(self.lib.sbm_export_geometry(self.ctx, level, ctypes.byref(nf), cell.ctypes.data,
                                            slot.ctypes.data, d.ctypes.data))
        return cell, slot, d

    # ------------------------------------------------------------------ device operations
    def _vec(self, t, dtype=None):
        torch = self._torch
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("expected a contiguous CUDA tensor")
        if dtype is not None and t.dtype != dtype:
            raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
        if t.dtype not in (torch.float64, torch.float32):
            raise ValueError("vectors must be float64 or float32")
        return ctypes.c_void_p(t.data_ptr())

    def _dt(self, t):
        return SBM_F64 if t.dtype == self._torch.float64 else SBM_F32

    def n_dof(self, level: int = -1) -> int:
        return self.info(level)["n_dof"]

    def rhs(self):
        b = self._torch.empty(self.n_dof(), dtype=self._torch.float64, device="cuda")
        _check(self.lib.sbm_rhs(self.ctx, self._vec(b)))
        return b

    def apply(self, x, y=None, level: int = -1):
        y = self._torch.empty_like(x) if y is None else y
        _check(self.lib.sbm_apply(self.ctx, level, self._dt(x), self._vec(x), self._vec(y, x.dtype)))
        return y

    def residual(self, f, u, r=None, level: int = -1):
        r = self._torch.empty_like(u) if r is None else r
        _check(self.lib.sbm_residual(self.ctx, level, self._dt(u), self._vec(f, u.dtype), self._vec(u),
                                     self._vec(r, u.dtype)))
        return r

    def smooth(self, f, u, level: int = -1, reverse: bool = False):
        _check(self.lib.sbm_smooth(self.ctx, level, self._dt(u), int(reverse), self._vec(f, u.dtype), self._vec(u)))
        return u

    def restrict(self, rf, level: int = -1):
        level = self.num_levels - 1 if level < 0 else level
        rc = self._torch.empty(self.n_dof(level - 1), dtype=rf.dtype, device="cuda")
        _check(self.lib.sbm_restrict(self.ctx, level, self._dt(rf), self._vec(rf), self._vec(rc)))
        return rc

    def prolong_add(self, ec, uf, level: int = -1):
        _check(self.lib.sbm_prolong_add(self.ctx, level, self._dt(uf), self._vec(ec, uf.dtype), self._vec(uf)))
        return uf

    def coarse_solve(self, r, e=None):
        e = self._torch.empty_like(r) if e is None else e
        _check(self.lib.sbm_coarse_solve(self.ctx, self._dt(r), self._vec(r), self._vec(e, r.dtype)))
        return e

    def vcycle(self, r, z=None):
        z = self._torch.empty_like(r) if z is None else z
        _check(self.lib.sbm_vcycle(self.ctx, self._dt(r), self._vec(r), self._vec(z, r.dtype)))
        return z

    def dots(self, V, w, out=None):
        """out[k] = V[k] . w (FP64), V: (nv, n) contiguous CUDA tensor, w: (n,)."""
        torch = self._torch
        if V.dim() != 2 or V.dtype != torch.float64 or not V.is_contiguous() or not V.is_cuda:
            raise ValueError("V must be a contiguous (nv, n) float64 CUDA tensor")
        out = torch.empty(V.shape[0], dtype=torch.float64, device="cuda") if out is None else out
        _check(self.lib.sbm_dots(self.ctx, self._vec(V), V.shape[1], V.shape[0], self._vec(w, torch.float64),
                                 w.numel(), self._vec(out, torch.float64)))
        return out

    def l2_error(self, x) -> float:
        """||u - u_h||_L2 over the finest active cells of the FP64 solution x (device)."""
        e = ctypes.c_double()
        _check(self.lib.sbm_l2_error(self.ctx, self._vec(x, self._torch.float64), ctypes.byref(e)))
        return e.value

    def gram_schmidt(self, V, w, variant: int = 0):
        """(h1, h2, w2, |w2|) of the two classical Gram-Schmidt passes of an Arnoldi step, by the
        solver's own sweeps: V (nv, N) and w (N,) contiguous float64 CUDA tensors, N the finest
        level's length; variant 0/1 double-float basis (w in FP64 / rounded to double-float first),
        2 FP64 basis."""
        torch = self._torch
        if V.dim() != 2 or V.dtype != torch.float64 or not V.is_contiguous() or not V.is_cuda:
            raise ValueError("V must be a contiguous (nv, N) float64 CUDA tensor")
        nv = V.shape[0]
        h = torch.empty(2 * nv, dtype=torch.float64, device="cuda")
        wout = torch.empty_like(w)
        nrm = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(self.lib.sbm_gram_schmidt(self.ctx, variant, self._vec(V), nv, self._vec(w, torch.float64),
                                         self._vec(h), self._vec(wout), self._vec(nrm)))
        return h[:nv], h[nv:], wout, float(nrm.item())

    def solve(self, b, x, tol: float = 1e-8, restart: int = 30, max_it: int = 300, check: bool = True) -> SolveInfo:
        inf = _SolveInfo()
        code = self.lib.sbm_solve(self.ctx, self._vec(b, self._torch.float64), self._vec(x, self._torch.float64),
                                  tol, restart, max_it, ctypes.byref(inf))
        if check and code not in (0, -4):
            _check(code)
        return _info(inf, code)

    def solve_host(self, b_host: np.ndarray, x_host: np.ndarray, tol: float = 1e-8, restart: int = 30,
                   max_it: int = 300) -> SolveInfo:
        """Host-buffer solve: the host->device copy of b and the copy of x back are part of the call."""
        for a in (b_host, x_host):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host buffers must be contiguous float64")
        inf = _SolveInfo()
        code = self.lib.sbm_solve_host(self.ctx, ctypes.c_void_p(b_host.ctypes.data),
                                       ctypes.c_void_p(x_host.ctypes.data), tol, restart, max_it, ctypes.byref(inf))
        if code not in (0, -4):
            _check(code)
        return _info(inf, code)


    # ------------------------------------------------------------------ learned correction
    def learned_cells(self) -> np.ndarray:
        """Compact indices of the finest-level boundary cells (the rows of learned_features)."""
        n = ctypes.c_int()
        _check(self.lib.sbm_learned_cells(self.ctx, ctypes.byref(n), None))
        out = np.zeros(n.value, dtype=np.int32)
        _check(self.lib.sbm_learned_cells(self.ctx, ctypes.byref(n), out.ctypes.data))
        return out

    def learned_features(self, res, F: int):
        """(X [n_bnd][F] float32, s [n_bnd]) from a finest-level residual."""
        torch = self._torch
        nb = len(self.learned_cells())
        X = torch.empty((nb, F), dtype=torch.float32, device="cuda")
        s = torch.empty(nb, dtype=torch.float32, device="cuda")
        _check(self.lib.sbm_learned_features(self.ctx, self._dt(res), self._vec(res), ctypes.c_void_p(X.data_ptr()),
                                             ctypes.c_void_p(s.data_ptr())))
        return X, s

    def collect(self, mlp: "Mlp", u0, n_cycles: int) -> int:
        """Training pairs from n_cycles stationary V-cycle steps on A u = 0 from each row of u0
        ((n_starts, N), the V-cycle precision); returns the rows appended to mlp's set."""
        if u0.dim() != 2 or u0.shape[1] != self.n_dof() or not u0.is_contiguous() or not u0.is_cuda:
            raise ValueError("u0 must be a contiguous (n_starts, N) CUDA tensor")
        n = ctypes.c_longlong()
        _check(self.lib.sbm_collect(self.ctx, mlp.h, self._dt(u0), ctypes.c_void_p(u0.data_ptr()), u0.shape[0],
                                    n_cycles, ctypes.byref(n)))
        return n.value

    def attach_mlp(self, mlp: "Mlp | None", scale: float = 1.0, fallback_rate: float = 0.0) -> None:
        """Attach (or detach with None) the learned correction to this solver's V-cycle."""
        self._mlp = mlp                                   # keeps the MLP alive while attached
        _check(self.lib.sbm_attach_mlp(self.ctx, mlp.h if mlp is not None else None, scale, fallback_rate))


class Mlp:
    """The learned boundary-cell correction's MLP (FP32 master parameters, BF16 tensor-core
    forward/backward, Adam) and its device training set.  See sbm_mlp_* in include/sbm.h."""

    def __init__(self, dim: int, p: int, hidden: int = 128, seed: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libsbm needs a CUDA device; no CPU fallback exists")
        self._torch = torch
        self.lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(self.lib.sbm_mlp_create(dim, p, hidden, seed, ctypes.c_void_p(self.stream.cuda_stream),
                                       ctypes.byref(h)))
        self.h = h
        F, Fp, H, O = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        n = ctypes.c_longlong()
        _check(self.lib.sbm_mlp_shape(self.h, ctypes.byref(F), ctypes.byref(Fp), ctypes.byref(H), ctypes.byref(O),
                                      ctypes.byref(n)))
        self.F, self.Fpad, self.H, self.O, self.nparam = F.value, Fp.value, H.value, O.value, n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.sbm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f32(self, t, shape):
        if not (t.is_cuda and t.is_contiguous() and t.dtype == self._torch.float32) or tuple(t.shape) != shape:
            raise ValueError(f"expected a contiguous float32 CUDA tensor of shape {shape}")
        return ctypes.c_void_p(t.data_ptr())

    def split(self, flat: np.ndarray):
        """(W1, b1, W2, b2, W3, b3) views of a packed parameter vector."""
        F, H, O = self.F, self.H, self.O
        sizes = [F * H, H, H * H, H, H * O, O]
        shapes = [(F, H), (H,), (H, H), (H,), (H, O), (O,)]
        out, o = [], 0
        for n, sh in zip(sizes, shapes):
            out.append(flat[o:o + n].reshape(sh))
            o += n
        return out

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparam, dtype=np.float32)
        _check(self.lib.sbm_mlp_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, params) -> None:
        """params: packed vector, or the list (W1, b1, W2, b2, W3, b3) (input-major weights)."""
        if isinstance(params, (list, tuple)):
            params = np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1) for a in params])
        flat = np.ascontiguousarray(params, dtype=np.float32)
        if flat.size != self.nparam:
            raise ValueError(f"expected {self.nparam} parameters, got {flat.size}")
        _check(self.lib.sbm_mlp_set_params(self.h, flat.ctypes.data))

    def gemm_backend(self, backend: int) -> None:
        """0: tcgen05 tensor-core GEMMs (default), 1: warp-level mma.sync GEMMs."""
        _check(self.lib.sbm_mlp_gemm_backend(self.h, backend))

    def forward(self, X):
        rows = X.shape[0]
        Y = self._torch.empty((rows, self.O), dtype=self._torch.float32, device="cuda")
        _check(self.lib.sbm_mlp_forward(self.h, self._f32(X, (rows, self.F)), rows, self._f32(Y, (rows, self.O))))
        return Y

    def gradients(self, X, T):
        """(loss, packed gradient) of mean((MLP(X) - T)^2)."""
        rows = X.shape[0]
        g = np.zeros(self.nparam, dtype=np.float32)
        loss = ctypes.c_double()
        _check(self.lib.sbm_mlp_gradients(self.h, self._f32(X, (rows, self.F)), self._f32(T, (rows, self.O)), rows,
                                          g.ctypes.data, ctypes.byref(loss)))
        return loss.value, g

    def num_samples(self) -> int:
        n = ctypes.c_longlong()
        _check(self.lib.sbm_mlp_num_samples(self.h, ctypes.byref(n)))
        return n.value

    def clear_samples(self) -> None:
        _check(self.lib.sbm_mlp_clear_samples(self.h))

    def target_scale(self) -> float:
        """Normalise the stored targets to unit RMS; returns the RMS (attach with scale=RMS)."""
        r = ctypes.c_double()
        _check(self.lib.sbm_mlp_target_scale(self.h, ctypes.byref(r)))
        return r.value

    def train(self, epochs: int = 20, batch: int = 4096, lr: float = 1e-3, seed: int = 0) -> float:
        loss = ctypes.c_double()
        _check(self.lib.sbm_mlp_train(self.h, epochs, batch, lr, seed, ctypes.byref(loss)))
        return loss.value

    def save(self, path: str) -> None:
        _check(self.lib.sbm_mlp_save(self.h, os.fsencode(path)))

    def load(self, path: str) -> None:
        _check(self.lib.sbm_mlp_load(self.h, os.fsencode(path)))


class HostSetup:
    """Host-only libsbm context (no GPU needed): the set-up of every level and a host FP64
    evaluation of the operator with the same element data the kernels use."""

    def __init__(self, prob):
        self.lib = load_library()
        self.prob = prob
        desc = make_desc(prob, SBM_F64, 0)
        ctx = ctypes.c_void_p()
        _check(self.lib.sbm_setup_host(ctypes.byref(desc), ctypes.byref(ctx)))
        self.ctx = ctx
        n = ctypes.c_int()
        _check(self.lib.sbm_num_levels(self.ctx, ctypes.byref(n)))
        self.num_levels = n.value

    info = Solver.info
    layout = Solver.layout
    export_geometry = Solver.export_geometry
    close = Solver.close
    __del__ = Solver.__del__

    def host_apply(self, x: np.ndarray, level: int = -1) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        _check(self.lib.sbm_host_apply(self.ctx, level, x.ctypes.data, y.ctypes.data))
        return y

    def host_rhs(self) -> np.ndarray:
        b = np.zeros(self.info(-1)["n_dof"])
        _check(self.lib.sbm_host_rhs(self.ctx, b.ctypes.data))
        return b


def _info(inf: _SolveInfo, code: int) -> SolveInfo:
    n = min(inf.iterations, 512)
    return SolveInfo(bool(inf.converged), inf.iterations, inf.restarts, inf.true_rel_residual,
                     list(inf.history[:n]), inf.ms_total, code, bool(inf.learned), bool(inf.learned_fallback))


def compact_to_natural(coords: np.ndarray, n: int, dim: int) -> np.ndarray:
    """Background linear id (x fastest) of each compact cell, from `Solver.layout()`."""
    lin = coords[:, 0].astype(np.int64) + n * coords[:, 1].astype(np.int64)
    if dim == 3:
        lin += n * n * coords[:, 2].astype(np.int64)
    return lin

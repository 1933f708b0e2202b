"""Geometry of the shifted boundary method, computed plainly on the CPU in FP64.

Follows Sec. 2.1 (volume fraction kappa, Eq. 4; active cells kappa > lambda; surrogate
boundary; shift vector d = x - x~) and Sec. 4.1-4.2 (level set phi < 0 inside; closest
point by Newton on the Lagrangian of Eqs. 19-22).

Readings where the paper leaves a choice:
  * kappa: the paper allows a cheap surrogate for kappa (Sec. 2.1).  Here kappa is the
    fraction of the s^d sub-cell midpoints of the cell at which phi < 0.
  * The threshold test is kappa > lambda (paper) or kappa >= lambda (the hot-path
    workloads), chosen by `lam_inclusive`.
  * The level set is the analytic phi on every level (the paper interpolates phi by
    finite elements; geometry is set-up, not the solver path).
  * The closest point is the global one for the disk/sphere and box (closed form); for the
    other shapes Newton on Eqs. 21-22 (backtracking on |F|) starts from the nearest point of a
    fixed sampling of the boundary, so that it converges to the global minimum also where the
    surrogate point lies beyond a centre of curvature (coarse levels), where a projection
    start lands on a local maximum of the distance.
"""
from __future__ import annotations

import math

import numpy as np

import workloads as W
from . import quadrature as Q


# --------------------------------------------------------------------------- level sets
def _rot(shape):
    return np.array(shape.rot, dtype=np.float64).reshape(3, 3)


def phi(shape: W.Shape, X: np.ndarray) -> np.ndarray:
    """Level-set values at points X (..., dim)."""
    X = np.asarray(X, dtype=np.float64)
    dim = X.shape[-1]
    c = np.array(shape.center[:dim])
    if shape.kind == W.SHAPE_DISK:
        return np.sqrt(np.sum((X - c) ** 2, axis=-1)) - shape.radius
    if shape.kind == W.SHAPE_BOX:
        return np.max(np.abs(X - c), axis=-1) - shape.radius
    if shape.kind == W.SHAPE_STAR:
        Y = X - c
        rho = np.sqrt(Y[..., 0] ** 2 + Y[..., 1] ** 2)
        th = np.arctan2(Y[..., 1], Y[..., 0])
        return rho - shape.radius * (1.0 + shape.amp * np.sin(shape.freq * th + shape.phase))
    if shape.kind == W.SHAPE_ELLIPSOID:
        Y = (X - c) @ _rot(shape)          # rows: R^T (x - c)
        q = Y / np.array(shape.semi)
        return np.sqrt(np.sum(q * q, axis=-1)) - 1.0
    if shape.kind == W.SHAPE_COMPLEX2D:
        x, y = X[..., 0], X[..., 1]
        return (1.0 - 0.75 * np.sin(np.pi * x) ** 2) * (x * x + y * y) - 0.2
    raise ValueError(f"unknown shape kind {shape.kind}")


def grad_hess(shape: W.Shape, x: np.ndarray):
    """Gradient and Hessian of phi at one point x (dim,), for the smooth shapes used by Newton."""
    x = np.asarray(x, dtype=np.float64)
    dim = len(x)
    c = np.array(shape.center[:dim])
    if shape.kind == W.SHAPE_STAR:
        y = x - c
        rho = math.hypot(y[0], y[1])
        th = math.atan2(y[1], y[0])
        n = y / rho
        dth = np.array([-y[1], y[0]]) / rho ** 2
        Hrho = (np.eye(2) - np.outer(n, n)) / rho
        Hth = np.array([[2 * y[0] * y[1], y[1] ** 2 - y[0] ** 2],
                        [y[1] ** 2 - y[0] ** 2, -2 * y[0] * y[1]]]) / rho ** 4
        arg = shape.freq * th + shape.phase
        R1 = shape.radius * shape.amp * shape.freq * math.cos(arg)
        R2 = -shape.radius * shape.amp * shape.freq ** 2 * math.sin(arg)
        g = n - R1 * dth
        H = Hrho - R2 * np.outer(dth, dth) - R1 * Hth
        return g, H
    if shape.kind == W.SHAPE_ELLIPSOID:
        R = _rot(shape)
        Sinv = np.diag(1.0 / np.array(shape.semi))
        q = Sinv @ (R.T @ (x - c))
        s = np.linalg.norm(q)
        M = R @ Sinv
        g = M @ q / s
        H = M @ ((np.eye(3) - np.outer(q, q) / (s * s)) / s) @ M.T
        return g, H
    if shape.kind == W.SHAPE_DISK:
        y = x - c
        r = np.linalg.norm(y)
        n = y / r
        return n, (np.eye(dim) - np.outer(n, n)) / r
    if shape.kind == W.SHAPE_COMPLEX2D:
        X, Y = x
        s = math.sin(math.pi * X)
        a = 1 - 0.75 * s * s
        ap = -0.75 * math.pi * math.sin(2 * math.pi * X)
        app = -1.5 * math.pi ** 2 * math.cos(2 * math.pi * X)
        r2 = X * X + Y * Y
        g = np.array([ap * r2 + 2 * a * X, 2 * a * Y])
        H = np.array([[app * r2 + 4 * ap * X + 2 * a, 2 * ap * Y], [2 * ap * Y, 2 * a]])
        return g, H
    raise ValueError(f"no smooth Hessian for shape kind {shape.kind}")


# --------------------------------------------------------------------------- closest point
class NewtonFailure(RuntimeError):
    pass


def boundary_samples(shape: W.Shape, dim: int) -> np.ndarray:
    """A fixed sampling of the true boundary, used only to start Newton near the global minimum:
    star and the Sec. 5.4 domain: 1024 rays theta_k = 2 pi k / 1024; ellipsoid: 64 x 128
    (u_i = pi (i + 1/2) / 64, v_j = 2 pi j / 128) points of c + R diag(semi) (sin u cos v,
    sin u sin v, cos u)."""
    c = np.array(shape.center[:dim])
    if shape.kind == W.SHAPE_STAR:
        th = 2 * np.pi * np.arange(1024) / 1024
        r = shape.radius * (1.0 + shape.amp * np.sin(shape.freq * th + shape.phase))
        return c + np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    if shape.kind == W.SHAPE_COMPLEX2D:
        th = 2 * np.pi * np.arange(1024) / 1024
        lo, hi = np.zeros(1024), np.full(1024, 2.0)        # phi(0) < 0 < phi(2 e_theta): bisection
        for _ in range(64):
            mid = 0.5 * (lo + hi)
            inside = phi(shape, np.stack([mid * np.cos(th), mid * np.sin(th)], axis=1)) < 0
            lo, hi = np.where(inside, mid, lo), np.where(inside, hi, mid)
        r = 0.5 * (lo + hi)
        return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    if shape.kind == W.SHAPE_ELLIPSOID:
        u = np.pi * (np.arange(64) + 0.5) / 64
        v = 2 * np.pi * np.arange(128) / 128
        U, V = np.meshgrid(u, v, indexing="ij")
        loc = np.stack([np.sin(U) * np.cos(V), np.sin(U) * np.sin(V), np.cos(U)], axis=-1).reshape(-1, 3)
        return c + (loc * np.array(shape.semi)) @ _rot(shape).T
    raise ValueError(f"no boundary sampling for shape kind {shape.kind}")


_SAMPLES = {}


def closest_point_newton(shape: W.Shape, xt: np.ndarray, maxit: int = 50) -> np.ndarray:
    """Closest point on {phi = 0} to xt: Newton on the stationarity system of the
    Lagrangian L(x, mu) = |x - xt|^2 + mu phi(x) (Eqs. 20-22):
        F(x, mu) = [2 (x - xt) + mu grad phi(x) ; phi(x)] = 0,
        J = [[2 I + mu Hess phi, grad phi], [grad phi^T, 0]],
    started from the nearest point of `boundary_samples` (first one on ties) with
    mu = 2 (xt - x).grad phi / |grad phi|^2, with backtracking on |F|.
    """
    xt = np.asarray(xt, dtype=np.float64)
    dim = len(xt)
    key = (shape.kind, tuple(shape.center), shape.radius, shape.amp, shape.freq, shape.phase,
           tuple(shape.semi), tuple(shape.rot), dim)
    if key not in _SAMPLES:
        _SAMPLES[key] = boundary_samples(shape, dim)
    samp = _SAMPLES[key]
    x = samp[int(np.argmin(np.sum((samp - xt) ** 2, axis=1)))].copy()
    g, _H = grad_hess(shape, x)
    mu = 2.0 * ((xt - x) @ g) / (g @ g)

    def residual(xx, mm):
        gg, HH = grad_hess(shape, xx)
        return np.concatenate([2.0 * (xx - xt) + mm * gg, [phi(shape, xx)]]), gg, HH

    F, g, H = residual(x, mu)
    for _ in range(maxit):
        nF = np.linalg.norm(F)
        if nF <= 1e-15:
            break
        J = np.zeros((dim + 1, dim + 1))
        J[:dim, :dim] = 2.0 * np.eye(dim) + mu * H
        J[:dim, dim] = g
        J[dim, :dim] = g
        delta = np.linalg.solve(J, -F)
        t = 1.0
        while True:
            xn, mn = x + t * delta[:dim], mu + t * delta[dim]
            Fn, gn, Hn = residual(xn, mn)
            if np.linalg.norm(Fn) < (1.0 - 1e-4 * t) * nF or t < 1e-3:
                break
            t *= 0.5
        x, mu, F, g, H = xn, mn, Fn, gn, Hn
        if np.linalg.norm(t * delta) <= 1e-15 * max(1.0, np.linalg.norm(x)):
            break
    if np.linalg.norm(F) > 1e-10:
        raise NewtonFailure(f"closest point did not converge at {xt}: |F|={np.linalg.norm(F):.3e}")
    return x


def closest_point(shape: W.Shape, xt: np.ndarray) -> np.ndarray:
    """Closest-point projection of a surrogate point onto the true boundary (Sec. 2.1, Sec. 4.2)."""
    xt = np.asarray(xt, dtype=np.float64)
    dim = len(xt)
    c = np.array(shape.center[:dim])
    if shape.kind == W.SHAPE_DISK:
        y = xt - c
        return c + shape.radius * y / np.linalg.norm(y)
    if shape.kind == W.SHAPE_BOX:
        y = xt - c
        r = shape.radius
        if np.max(np.abs(y)) <= r:                 # inside (or on): move the dominant coordinate out
            k = int(np.argmax(np.abs(y) - r))
            out = y.copy()
            out[k] = r if y[k] >= 0 else -r
            return c + out
        return c + np.clip(y, -r, r)
    return closest_point_newton(shape, xt)


# --------------------------------------------------------------------------- mesh geometry
class LevelGeometry:
    """Active set, surrogate faces and shift vectors of one background mesh (n cells/dir, degree p).

    Cells are indexed by background multi-index I = (i_0, .., i_{dim-1}) with x fastest;
    `active_cells` lists the active ones in that lexicographic ("natural") order.
    A surrogate face is a face of an active cell whose neighbour is inactive or outside the box.
    Each surrogate face carries (p+1)^(dim-1) Gauss-Legendre points x~ and shifts d = x - x~.
    """

    def __init__(self, prob: W.Problem, n: int, p: int):
        self.prob, self.n, self.p, self.dim = prob, n, p, prob.dim
        dim = prob.dim
        self.lo = np.array(prob.lo[:dim], dtype=np.float64)
        self.hi = np.array(prob.hi[:dim], dtype=np.float64)
        self.h = float((self.hi[0] - self.lo[0]) / n)
        self.kappa = volume_fractions(prob, n)
        S = prob.samples ** dim
        count = np.rint(self.kappa * S)
        thr = prob.lam * S
        self.active = (count >= thr) if prob.lam_inclusive else (count > thr)
        shape = (n,) * dim
        flat = self.active.reshape(-1)
        self.active_cells = np.nonzero(flat)[0]               # background linear ids, natural order
        self.bg2act = -np.ones(n ** dim, dtype=np.int64)
        self.bg2act[self.active_cells] = np.arange(len(self.active_cells))
        self.cell_idx = np.stack(np.unravel_index(self.active_cells, shape[::-1])[::-1], axis=1) \
            if dim > 1 else self.active_cells[:, None]
        self._build_faces()

    def corner(self, idx):
        return self.lo + self.h * np.asarray(idx, dtype=np.float64)

    def neighbour(self, idx, direction, side):
        """Background linear id of the face neighbour, or -1 outside the box."""
        j = list(idx)
        j[direction] += 1 if side == 1 else -1
        if j[direction] < 0 or j[direction] >= self.n:
            return -1
        lin = 0
        for k in reversed(range(self.dim)):
            lin = lin * self.n + j[k]
        return lin

    def _build_faces(self):
        dim, p = self.dim, self.p
        nodes, _ = Q.gauss_legendre(p + 1)
        tang = Q.multi_indices(p + 1, dim - 1) if dim > 1 else np.zeros((1, 0), dtype=np.int64)
        self.faces = []                                   # (act cell, direction, side)
        self.face_xt = []                                 # (nq, dim) surrogate points
        self.face_d = []                                  # (nq, dim) shifts
        self.interior_faces = []                          # (act minus, act plus, direction)
        for a, idx in enumerate(self.cell_idx):
            for direction in range(dim):
                for side in (0, 1):
                    nb = self.neighbour(idx, direction, side)
                    nb_act = self.bg2act[nb] if nb >= 0 else -1
                    if nb_act >= 0:
                        if side == 1:
                            self.interior_faces.append((a, nb_act, direction))
                        continue
                    tdirs = [k for k in range(dim) if k != direction]
                    xi = np.zeros((len(tang), dim))
                    xi[:, direction] = float(side)
                    for t, k in enumerate(tdirs):
                        xi[:, k] = nodes[tang[:, t]]
                    xt = self.corner(idx) + self.h * xi
                    d = np.array([closest_point(self.prob.shape, x) - x for x in xt])
                    self.faces.append((a, direction, side))
                    self.face_xt.append(xt)
                    self.face_d.append(d)
        self.interior_faces = np.array(self.interior_faces, dtype=np.int64).reshape(-1, 3)

    @property
    def n_active(self):
        return len(self.active_cells)

    def boundary_cells(self):
        """Active cells that own at least one surrogate face."""
        return sorted({f[0] for f in self.faces})


def volume_fractions(prob: W.Problem, n: int) -> np.ndarray:
    """kappa(K) = fraction of the s^dim sub-cell midpoints of K with phi < 0 (Eq. 4, cheap surrogate).

    Returns an array of shape (n,)*dim indexed [i_{dim-1}, ..., i_0] (x fastest in memory)."""
    dim = prob.dim
    s = prob.samples
    lo = np.array(prob.lo[:dim], dtype=np.float64)
    h = float((prob.hi[0] - prob.lo[0]) / n)
    sub = (np.arange(s) + 0.5) / s
    offs = np.stack(np.meshgrid(*([sub] * dim), indexing="ij"), axis=-1).reshape(-1, dim)[:, ::-1]
    # offs: all s^dim sub-cell midpoints (reference coordinates), any fixed order
    kappa = np.zeros((n,) * dim)
    if dim == 2:
        for j in range(n):
            ii = np.arange(n)
            corners = lo + h * np.stack([ii, np.full(n, j)], axis=1)
            pts = corners[:, None, :] + h * offs[None, :, :]
            kappa[j, :] = np.mean(phi(prob.shape, pts) < 0.0, axis=1)
    else:
        ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
        for k in range(n):
            corners = lo + h * np.stack([ii.reshape(-1), jj.reshape(-1), np.full(n * n, k)], axis=1)
            pts = corners[:, None, :] + h * offs[None, :, :]
            kappa[k] = np.mean(phi(prob.shape, pts) < 0.0, axis=1).reshape(n, n)
    return kappa

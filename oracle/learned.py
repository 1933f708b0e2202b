"""Learned boundary-cell correction, plain FP64 reference (test infrastructure).

The paper has no learned component; this is the learned variant of the V-cycle smoother built on
the paper's method (its p = 3 smoother weakens near the surrogate boundary, Sec. 5.3).  After
the finest-level post-smoothing, every boundary cell K (a cell owning a surrogate face) gets a
correction u_K += s * h^(2-d) * MLP(x_K), where

  x_K = [ patch residual / s , d / h on every face point , kappa(K) , surrogate-face mask ]
  s   = || patch residual ||_2  (1 if the patch residual is zero)

* patch residual: the residual r = f - A u of the 3^d cells K + o, o in {-1, 0, 1}^d (offsets
  ordered x fastest), each contributing its (p+1)^d values, zeros for cells that are inactive
  or outside the box;
* d / h: for face slot s = 2 * direction + side, face point t (tangential Gauss-Legendre points,
  first tangential dim fastest) and component k, d_k / h on surrogate faces and 0 elsewhere;
* kappa: the volume fraction of K; mask: 1 for each surrogate face slot.

MLP: two hidden layers with ReLU, y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3 (weights
stored input-major, W1: F x H).  Training minimises the mean squared error between y and
target / (s h^(2-d)), where the target is the cell's error (exact solution minus u); h^(2-d) is the
scale of A^-1 (the operator scales like h^(d-2)), which makes the targets mesh-independent.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import multigrid as MG


def feature_size(dim: int, p: int) -> int:
    nb = (p + 1) ** dim
    nq = (p + 1) ** (dim - 1)
    return 3 ** dim * nb + 2 * dim * nq * dim + 1 + 2 * dim


def patch_offsets(dim: int):
    return [tuple(reversed(o)) for o in itertools.product((-1, 0, 1), repeat=dim)]


def features(level: MG.Level, r: np.ndarray, cells):
    """(X, s) for the given active cells (oracle natural order) from the residual r."""
    g, nb, dim = level.geom, level.nb, level.prob.dim
    p = level.p
    nq = (p + 1) ** (dim - 1)
    F = feature_size(dim, p)
    R = r.reshape(-1, nb)
    faces = {}
    for f, (a, dr, side) in enumerate(g.faces):
        faces[(a, 2 * dr + side)] = f
    kap = g.kappa.reshape(-1)
    X = np.zeros((len(cells), F))
    s = np.ones(len(cells))
    for row, a in enumerate(cells):
        idx = g.cell_idx[a]
        patch = []
        for o in patch_offsets(dim):
            j = idx + np.array(o)
            if np.any(j < 0) or np.any(j >= g.n):
                patch.append(np.zeros(nb))
                continue
            lin = 0
            for k in reversed(range(dim)):
                lin = lin * g.n + int(j[k])
            act = g.bg2act[lin]
            patch.append(R[act] if act >= 0 else np.zeros(nb))
        patch = np.concatenate(patch)
        nrm = np.linalg.norm(patch)
        s[row] = nrm if nrm > 0 else 1.0
        dfeat = np.zeros((2 * dim, nq, dim))
        mask = np.zeros(2 * dim)
        for slot in range(2 * dim):
            f = faces.get((a, slot))
            if f is not None:
                dfeat[slot] = g.face_d[f] / g.h
                mask[slot] = 1.0
        X[row] = np.concatenate([patch / s[row], dfeat.reshape(-1), [kap[g.active_cells[a]]], mask])
    return X, s


class MLP:
    """Two-hidden-layer ReLU network in FP64 with explicit forward and backward passes."""

    def __init__(self, F: int, H: int, O: int, seed: int = 0):
        rng = np.random.default_rng(seed)
        self.W1 = rng.normal(size=(F, H)) * np.sqrt(2.0 / F)
        self.b1 = np.zeros(H)
        self.W2 = rng.normal(size=(H, H)) * np.sqrt(2.0 / H)
        self.b2 = np.zeros(H)
        self.W3 = rng.normal(size=(H, O)) * np.sqrt(1.0 / H)
        self.b3 = np.zeros(O)

    def params(self):
        return [self.W1, self.b1, self.W2, self.b2, self.W3, self.b3]

    def forward(self, X):
        Z1 = X @ self.W1 + self.b1
        H1 = np.maximum(Z1, 0.0)
        Z2 = H1 @ self.W2 + self.b2
        H2 = np.maximum(Z2, 0.0)
        Y = H2 @ self.W3 + self.b3
        self._cache = (X, Z1, H1, Z2, H2)
        return Y

    def loss(self, Y, T):
        """Mean squared error over all entries."""
        return float(np.mean((Y - T) ** 2))

    def backward(self, Y, T):
        """Gradients of `loss` with respect to (W1, b1, W2, b2, W3, b3), after `forward`."""
        X, Z1, H1, Z2, H2 = self._cache
        dY = 2.0 * (Y - T) / Y.size
        gW3 = H2.T @ dY
        gb3 = dY.sum(axis=0)
        dH2 = dY @ self.W3.T
        dZ2 = dH2 * (Z2 > 0)
        gW2 = H1.T @ dZ2
        gb2 = dZ2.sum(axis=0)
        dH1 = dZ2 @ self.W2.T
        dZ1 = dH1 * (Z1 > 0)
        gW1 = X.T @ dZ1
        gb1 = dZ1.sum(axis=0)
        return [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) in place; state = dict(t, m, v)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    if "m" not in state:
        state["m"] = [np.zeros_like(p) for p in params]
        state["v"] = [np.zeros_like(p) for p in params]
    for p, g, m, v in zip(params, grads, state["m"], state["v"]):
        m *= b1
        m += (1 - b1) * g
        v *= b2
        v += (1 - b2) * g * g
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p -= lr * mh / (np.sqrt(vh) + eps)


def boundary_cells(level: MG.Level):
    """Active cells (oracle natural order) that own at least one surrogate face."""
    return level.geom.boundary_cells()


def correction_unit(level: MG.Level) -> float:
    """Unit of the network's outputs, h^(2-d): the operator scales like h^(d-2), so the error of a
    cell relative to its patch residual norm scales like h^(2-d)."""
    return level.geom.h ** (2 - level.prob.dim)


def correction(net: MLP, cells, scale: float = 1.0):
    """V-cycle hook: z_K += scale * s * h^(2-d) * MLP(x_K) for the boundary cells, x from r - A z
    (finest level)."""
    def apply(level: MG.Level, z: np.ndarray, r: np.ndarray):
        res = r - level.A @ z
        X, s = features(level, res, cells)
        Y = net.forward(X) * (scale * correction_unit(level)) * s[:, None]
        nb = level.nb
        for row, a in enumerate(cells):
            z[a * nb:(a + 1) * nb] += Y[row]
    return apply


def training_pairs(H: MG.Hierarchy, n_starts: int, n_cycles: int, seed: int, u0s=None, cells=None):
    """(X, T) from the stationary V-cycle iteration u <- u + V(-A u) on A u = 0 from seeded random
    u0 in U[-1, 1] (or the given starts u0s): the exact solution is 0, so after each finest-level
    post-smoothing the error of the finest iterate is -u.  Features use r = -A u; targets are
    -u_K / (s h^(2-d)).  Rows: for each start, for each step, one per boundary cell (`cells`, default
    the boundary cells in natural order)."""
    F = H.finest
    cells = boundary_cells(F) if cells is None else cells
    nb = F.nb
    rng = np.random.default_rng(seed)
    starts = list(u0s) if u0s is not None else [2.0 * rng.random(F.N) - 1.0 for _ in range(n_starts)]
    Xs, Ts = [], []

    def record(level, z, rhs):
        # inside the V-cycle the finest level solves A z = rhs with rhs = -A u; the iterate is u + z
        u_new = state["u"] + z
        res = -(level.A @ u_new)
        X, s = features(level, res, cells)
        T = np.stack([-u_new[a * nb:(a + 1) * nb] for a in cells]) / (s[:, None] * correction_unit(level))
        Xs.append(X)
        Ts.append(T)

    state = {}
    for u in starts:
        u = np.array(u, dtype=np.float64)
        for _ in range(n_cycles):
            state["u"] = u
            z = H.vcycle(-(F.A @ u), correction=record)
            u = u + z
    return np.concatenate(Xs), np.concatenate(Ts)

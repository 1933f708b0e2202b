"""Flexible GMRES(m), right-preconditioned, with classical Gram-Schmidt applied twice.

Sec. 3 solves the non-symmetric DG-SBM system with GMRES preconditioned by one multigrid
V-cycle.  The paper does not fix the restart length, the orthogonalisation or the side of
the preconditioner; the reading here is: flexible (FGMRES, so that the preconditioner may
be any fixed or varying map), right preconditioning, restart m = 30, two passes of classical
Gram-Schmidt (h = V^T w, w -= V h, twice, h accumulated), Givens rotations on the
Hessenberg matrix, and the stopping test |g_{j+1}| <= tol ||b|| followed by a check of the
true residual ||b - A x|| <= tol ||b|| at the end of each cycle.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class GmresInfo:
    converged: bool = False
    iterations: int = 0            # Arnoldi steps (= preconditioner applications)
    restarts: int = 0
    history: list = field(default_factory=list)   # |g_{j+1}| / ||b|| after each step
    true_rel_residual: float = float("nan")


def fgmres(apply_A, apply_M, b, x0=None, tol=1e-8, m=30, max_it=300):
    b = np.asarray(b, dtype=np.float64)
    N = len(b)
    x = np.zeros(N) if x0 is None else np.array(x0, dtype=np.float64)
    info = GmresInfo()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        info.converged, info.true_rel_residual = True, 0.0
        return np.zeros(N), info
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        info.true_rel_residual = beta / bnorm
        if beta <= tol * bnorm:
            info.converged = True
            return x, info
        if info.iterations >= max_it:
            return x, info
        V = np.zeros((m + 1, N))
        Z = np.zeros((m, N))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = apply_M(V[j])
            w = apply_A(Z[j])
            h = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h
            h2 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0.0:
                V[j + 1] = w / hn
            for i in range(j):                                       # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rr = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rr, H[j + 1, j] / rr
            H[j, j], H[j + 1, j] = rr, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            info.iterations += 1
            info.history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or info.iterations >= max_it or hn == 0.0:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):                                # back substitution
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        info.restarts += 1

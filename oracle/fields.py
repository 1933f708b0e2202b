"""Manufactured solutions u, their gradients and sources f = -Laplace(u) (Sec. 2, Eq. 1; Sec. 5.1, Eq. 23).

Dirichlet data is g = u evaluated on the true boundary (Sec. 2.1): the right-hand side of
Eq. 7 uses g at the projected point x~ + d.
"""
from __future__ import annotations

import numpy as np

import workloads as W


def _xyz(X):
    X = np.asarray(X, dtype=np.float64)
    x = X[..., 0]
    y = X[..., 1]
    z = X[..., 2] if X.shape[-1] > 2 else np.zeros_like(x)
    return x, y, z


def u_exact(kind: int, X: np.ndarray, shape: W.Shape | None = None) -> np.ndarray:
    x, y, z = _xyz(X)
    dim = np.asarray(X).shape[-1]
    if kind == W.EXACT_SINPROD:
        v = np.sin(np.pi * x) * np.sin(np.pi * y)
        return v * np.sin(np.pi * z) if dim == 3 else v
    if kind == W.EXACT_EXPCOS:
        return np.exp(x) * np.cos(2 * y)
    if kind == W.EXACT_LINEAR:
        return 0.5 + x - 0.7 * y + 0.3 * z
    if kind == W.EXACT_COSSIN:
        return 2 * np.cos(x) * np.sin(y)
    if kind == W.EXACT_QUADRATIC:
        return 0.5 + x - 0.7 * y + 0.3 * z + x * x - 0.5 * y * y + 0.25 * x * y - 0.4 * z * z + 0.2 * y * z
    if kind == W.EXACT_PHIP1:
        return (1 - 0.75 * np.sin(np.pi * x) ** 2) * (x * x + y * y) - 0.2 + 1.0
    raise ValueError(f"unknown exact solution kind {kind}")


def f_source(kind: int, X: np.ndarray) -> np.ndarray:
    """f = -Laplace(u), derived by hand for each manufactured solution."""
    x, y, z = _xyz(X)
    dim = np.asarray(X).shape[-1]
    if kind == W.EXACT_SINPROD:
        return dim * np.pi ** 2 * u_exact(kind, X)
    if kind == W.EXACT_EXPCOS:
        return 3.0 * u_exact(kind, X)           # u_xx = u, u_yy = -4u
    if kind == W.EXACT_LINEAR:
        return np.zeros_like(x)
    if kind == W.EXACT_COSSIN:
        return 2.0 * u_exact(kind, X)           # u_xx = u_yy = -u
    if kind == W.EXACT_QUADRATIC:
        lap = 2.0 - 1.0 + (-0.8 if dim == 3 else 0.0)
        return np.full_like(x, -lap)
    if kind == W.EXACT_PHIP1:
        # phi = a(x) r2 - 1/5, a = 1 - 3/4 sin^2(pi x); Laplace = a'' r2 + 4 a' x + 4 a
        s2 = np.sin(np.pi * x) ** 2
        a = 1 - 0.75 * s2
        ap = -0.75 * np.pi * np.sin(2 * np.pi * x)
        app = -1.5 * np.pi ** 2 * np.cos(2 * np.pi * x)
        r2 = x * x + y * y
        return -(app * r2 + 4 * ap * x + 4 * a)
    raise ValueError(f"unknown exact solution kind {kind}")

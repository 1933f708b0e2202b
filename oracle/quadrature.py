"""Gauss-Legendre quadrature and the nodal Lagrange basis on the unit interval / cube.

Sec. 2.2 of the paper keeps a nodal Lagrange basis of degree p on each cell.  The
paper does not say where the nodes sit; the reading taken here is the (p+1)
Gauss-Legendre points of [0,1] (the paper reports that the basis choice barely
changes iteration counts).  Multi-dimensional basis functions are tensor products,
numbered lexicographically with the x index fastest.
"""
from __future__ import annotations

import itertools

import numpy as np


def gauss_legendre(npts: int):
    """Points and weights of the npts-point Gauss-Legendre rule on [0,1] (exact to degree 2 npts - 1)."""
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """V[k, m] = l_k(x_m) for the Lagrange polynomials l_k on `nodes` (plain product formula)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((n, len(x)))
    for k in range(n):
        for j in range(n):
            if j != k:
                V[k] *= (x - nodes[j]) / (nodes[k] - nodes[j])
    return V


def lagrange_derivs(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """D[k, m] = l_k'(x_m): derivative of the product formula by the product rule."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((n, len(x)))
    for k in range(n):
        for i in range(n):
            if i == k:
                continue
            term = np.full(len(x), 1.0 / (nodes[k] - nodes[i]))
            for j in range(n):
                if j != k and j != i:
                    term = term * (x - nodes[j]) / (nodes[k] - nodes[j])
            D[k] += term
    return D


def multi_indices(npts: int, dim: int) -> np.ndarray:
    """All index tuples (i_0, ..., i_{dim-1}) in [0,npts)^dim, x index fastest: shape (npts^dim, dim)."""
    out = [tuple(reversed(t)) for t in itertools.product(range(npts), repeat=dim)]
    return np.array(out, dtype=np.int64).reshape(-1, dim)


def tensor_basis(p: int, dim: int, xi: np.ndarray):
    """Values and reference gradients of all (p+1)^dim tensor Lagrange basis functions at points.

    xi: (m, dim) reference coordinates in [0,1]^dim.
    Returns phi (m, nb) and grad (m, nb, dim), nb = (p+1)^dim, with
    phi_i(xi) = prod_k l_{i_k}(xi_k).
    """
    nodes, _ = gauss_legendre(p + 1)
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    m = xi.shape[0]
    idx = multi_indices(p + 1, dim)
    vals = [lagrange_values(nodes, xi[:, k]) for k in range(dim)]     # (p+1, m) per axis
    ders = [lagrange_derivs(nodes, xi[:, k]) for k in range(dim)]
    nb = idx.shape[0]
    phi = np.ones((m, nb))
    grad = np.ones((m, nb, dim))
    for b in range(nb):
        for k in range(dim):
            phi[:, b] *= vals[k][idx[b, k]]
            for g in range(dim):
                grad[:, b, g] *= (ders[k][idx[b, k]] if g == k else vals[k][idx[b, k]])
    return phi, grad


def tensor_rule(npts: int, dim: int):
    """Tensor Gauss-Legendre rule on [0,1]^dim: points (npts^dim, dim), weights (npts^dim,)."""
    x, w = gauss_legendre(npts)
    idx = multi_indices(npts, dim)
    pts = x[idx]
    wts = np.prod(w[idx], axis=1)
    return pts, wts

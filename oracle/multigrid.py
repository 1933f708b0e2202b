"""hp-multigrid V-cycle of Sec. 3 on assembled FP64 matrices.

Level hierarchy (Sec. 3): the finest mesh carries degree p, p-coarsening lowers the degree
to 1 on the same mesh, then h-coarsening halves the mesh at p = 1 down to `coarsest_n`
cells per direction.  Levels are numbered l = 0 (coarsest) .. L (finest).  Every level
has its own active set, shifts and re-discretised operator (Sec. 4.3).

Smoother (default): successive subspace correction over single-cell subspaces (Eq. 16) with the
local operator A_i = R_i A R_i^T (Eq. 14), i.e. block Gauss-Seidel,
    u_K <- u_K + omega A_KK^{-1} (f - A u)_K   (most recent u).
Visiting order: cells coloured by c(K) = sum_k (i_k mod 2) 2^k; the pre-smoother visits
colours 0 .. 2^d - 1, the post-smoother 2^d - 1 .. 0 (together one symmetric sweep, the
cell-wise SSOR of Sec. 4.3).  With `ssor_each`, every smoothing step is a full SSOR step, a
forward then a reverse sweep, both before and after the coarse correction (an SSOR step is its own
adjoint, so the V-cycle stays symmetric).  omega = 1, except on p = 3 levels where omega = 0.8 (Sec. 5.3).
Red-black ordering (`ordering` 1): face neighbours differ by one in one index, so cells of equal
index-sum parity never couple and the sweep visits the even-parity colours, then the odd ones.
Variants of Sec. 3.1 / Sec. 5.3 (`smoother`): 1, the additive form over the same subspaces, block
Jacobi u <- u + omega D^-1 (f - A u); 2, that block Jacobi wrapped in a Chebyshev iteration whose
interval comes from a power-iteration estimate of lambda_max(D^-1 A) (the Chebyshev smoother
names no degree or interval: degree 4 and [lambda_max / 20, 1.1 lambda_max] are our reading).

Transfers (Sec. 3.2): prolongation = embedding on the background mesh, realised by
interpolating the coarse polynomial at the fine nodes (Eq. 17); restriction = its
transpose (Eq. 18).  Reading for inactive cells (Secs. 4.1, 4.3): all level vectors are
kept only on active cells (masked); prolongation into a fine active cell whose parent is
inactive adds zero, and restriction into an inactive coarse cell is dropped.

Coarse solve: dense LU with partial pivoting of the coarsest active matrix (Sec. 3 names
a coarse solver without specifying it).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

import workloads as W
from . import quadrature as Q
from .dgsbm import Discretisation
from .geometry import LevelGeometry


def level_sequence(prob: W.Problem):
    """(n, p) from coarsest to finest: h-levels at p=1 up to n, then p = 2..p_target on the finest mesh."""
    ns = [prob.n]
    while ns[-1] % 2 == 0 and ns[-1] // 2 >= prob.coarsest_n:
        ns.append(ns[-1] // 2)
    levels = [(m, 1) for m in reversed(ns)]
    levels += [(prob.n, q) for q in range(2, prob.p + 1)]
    return levels


def colour_of(cell_idx: np.ndarray) -> np.ndarray:
    """c(K) = sum_k (i_k mod 2) 2^k."""
    return np.sum((cell_idx % 2) << np.arange(cell_idx.shape[1]), axis=1)


def chebyshev_start(cell_idx: np.ndarray, nb: int) -> np.ndarray:
    """Start vector of the power iteration for lambda_max(D^-1 A): entry (cell, node l) is
    1 + 0.5 sin(0.7 (i + 2.1 j + 3.3 k) + 1.3 l), a function of the background cell index, so that
    any cell ordering gives the same vector."""
    ijk = cell_idx.astype(np.float64)
    base = ijk[:, 0] + 2.1 * ijk[:, 1] + (3.3 * ijk[:, 2] if ijk.shape[1] > 2 else 0.0)
    return (1.0 + 0.5 * np.sin(0.7 * base[:, None] + 1.3 * np.arange(nb)[None, :])).reshape(-1)


CHEB_POWER_STEPS = 15      # power-iteration steps for lambda_max(D^-1 A)
CHEB_SAFETY = 1.1          # upper end of the Chebyshev interval: 1.1 times the estimate


class Level:
    def __init__(self, prob: W.Problem, n: int, p: int):
        self.prob, self.n, self.p = prob, n, p
        self.geom = LevelGeometry(prob, n, p)
        self.disc = Discretisation(prob, self.geom)
        self.A = self.disc.A
        self.nb = self.disc.nb
        self.omega = prob.omega_p3 if p == 3 else prob.omega
        self.colour = colour_of(self.geom.cell_idx)
        self.n_colours = 2 ** prob.dim
        self.cells_of_colour = [np.nonzero(self.colour == c)[0] for c in range(self.n_colours)]
        # A_KK^{-1} of each cell (Eq. 14: principal submatrix of A), by LU-based inversion
        self.diag_inv = np.linalg.inv(self.disc.diag)
        self._colour_rows = []
        for cells in self.cells_of_colour:
            idx = (cells[:, None] * self.nb + np.arange(self.nb)[None, :]).reshape(-1)
            self._colour_rows.append((idx, self.A[idx]))

    @property
    def N(self):
        return self.geom.n_active * self.nb

    def dofs(self, a):
        return slice(a * self.nb, (a + 1) * self.nb)

    # ------------------------------------------------------------------ smoothers
    def block_gs_sequential(self, u, f, order, omega=None):
        """One successive subspace correction pass (Eq. 16) over `order`, cell by cell:
        r = f_K - (A u)_K with the latest u, then solve A_KK e = r and add omega e."""
        omega = self.omega if omega is None else omega
        for a in order:
            s = self.dofs(a)
            r = f[s] - self.A[s] @ u
            AKK = self.A[s][:, s].toarray()
            u[s] += omega * np.linalg.solve(AKK, r)
        return u

    def colour_sequence(self, reverse=False):
        """Colours in sweep order: 0 .. 2^d - 1, or (ordering 1, red-black) the colours of even
        index-sum parity (popcount of c even) before those of odd parity; reversed for reverse."""
        cols = list(range(self.n_colours))
        if getattr(self.prob, "ordering", 0) == 1:
            cols = sorted(cols, key=lambda c: (bin(c).count("1") % 2, c))
        return cols[::-1] if reverse else cols

    def colour_order(self, reverse=False):
        return np.concatenate([self.cells_of_colour[c] for c in self.colour_sequence(reverse)])

    def coloured_sweep(self, u, f, reverse=False, omega=None):
        """Block Gauss-Seidel over the colours.  Cells of one colour share no face, so
        A_KN = 0 between them and the sequential correction (Eq. 16) over one colour equals
        the simultaneous correction of all its cells; it is evaluated that way here."""
        omega = self.omega if omega is None else omega
        cols = self.colour_sequence(reverse)
        for c in cols:
            cells = self.cells_of_colour[c]
            if len(cells) == 0:
                continue
            idx, Arows = self._colour_rows[c]
            r = (f[idx] - Arows @ u).reshape(len(cells), self.nb)
            u[idx] += omega * np.einsum("kij,kj->ki", self.diag_inv[cells], r).reshape(-1)
        return u


    # ------------------------------------------------------------------ additive smoothers
    def block_inverse(self, r):
        """D^-1 r with D the block diagonal of the cell blocks A_KK (Eq. 14)."""
        R = r.reshape(-1, self.nb)
        return np.einsum("kij,kj->ki", self.diag_inv, R).reshape(-1)

    def block_jacobi_step(self, u, f, omega=None):
        """Additive subspace correction over the single-cell subspaces (the additive form of Sec. 3.1):
        u <- u + omega D^-1 (f - A u), every cell from the same u."""
        omega = self.omega if omega is None else omega
        u += omega * self.block_inverse(f - self.A @ u)
        return u

    def lambda_max(self):
        """Estimate of the largest eigenvalue modulus of D^-1 A: CHEB_POWER_STEPS power-iteration
        steps from chebyshev_start, the last step's |D^-1 A v| with |v| = 1."""
        if getattr(self, "_lam_max", None) is None:
            v = chebyshev_start(self.geom.cell_idx, self.nb)
            lam = 0.0
            for _ in range(CHEB_POWER_STEPS):
                v = v / np.linalg.norm(v)
                w = self.block_inverse(self.A @ v)
                lam = np.linalg.norm(w)
                v = w
            self._lam_max = lam
        return self._lam_max

    def chebyshev(self, u, f, degree=None, ratio=None):
        """degree steps of the Chebyshev iteration preconditioned by D^-1 on the interval
        [b / ratio, b], b = CHEB_SAFETY * lambda_max (Chebyshev semi-iteration with the three-term
        recurrence of the scaled Chebyshev polynomials):
            theta = (b + a) / 2, delta = (b - a) / 2, sigma = theta / delta,
            rho_0 = 1 / sigma,  d_0 = D^-1 r_0 / theta,  u_1 = u_0 + d_0,
            rho_k = 1 / (2 sigma - rho_(k-1)),
            d_k = rho_k rho_(k-1) d_(k-1) + (2 rho_k / delta) D^-1 r_k,  u_(k+1) = u_k + d_k,
        with r_k = f - A u_k."""
        degree = self.prob.cheb_degree if degree is None else degree
        ratio = self.prob.cheb_ratio if ratio is None else ratio
        b = CHEB_SAFETY * self.lambda_max()
        a = b / ratio
        theta, delta = 0.5 * (b + a), 0.5 * (b - a)
        sigma = theta / delta
        rho = 1.0 / sigma
        d = self.block_inverse(f - self.A @ u) / theta
        u += d
        for _ in range(1, degree):
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * self.block_inverse(f - self.A @ u)
            u += d
            rho = rho_new
        return u


def prolongation(coarse: Level, fine: Level) -> sp.csr_matrix:
    """Sparse P (fine active dofs x coarse active dofs) of Eq. 17, masked to active cells."""
    dim = fine.prob.dim
    nodes_f, _ = Q.tensor_rule(fine.p + 1, dim)          # fine nodes in fine reference coordinates
    rows, cols, vals = [], [], []
    if coarse.n == fine.n:                                # p-transfer on the same mesh
        phi_c, _ = Q.tensor_basis(coarse.p, dim, nodes_f)  # phi_c[i_f, j_c]
        for a in range(fine.geom.n_active):
            ac = coarse.geom.bg2act[fine.geom.active_cells[a]]
            if ac < 0:
                continue
            rr, cc = np.meshgrid(np.arange(fine.nb), np.arange(coarse.nb), indexing="ij")
            rows.append((a * fine.nb + rr).reshape(-1))
            cols.append((ac * coarse.nb + cc).reshape(-1))
            vals.append(phi_c.reshape(-1))
    else:                                                 # h-transfer: parent = child // 2
        assert fine.n == 2 * coarse.n
        cache = {}
        for a, idx in enumerate(fine.geom.cell_idx):
            parent = idx // 2
            off = tuple(int(v) for v in idx % 2)
            lin = 0
            for k in reversed(range(dim)):
                lin = lin * coarse.n + int(parent[k])
            ac = coarse.geom.bg2act[lin]
            if ac < 0:
                continue
            if off not in cache:
                cache[off] = Q.tensor_basis(coarse.p, dim, (np.array(off)[None, :] + nodes_f) / 2.0)[0]
            phi_c = cache[off]
            rr, cc = np.meshgrid(np.arange(fine.nb), np.arange(coarse.nb), indexing="ij")
            rows.append((a * fine.nb + rr).reshape(-1))
            cols.append((ac * coarse.nb + cc).reshape(-1))
            vals.append(phi_c.reshape(-1))
    if rows:
        r, c, v = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    else:
        r = c = np.zeros(0, dtype=np.int64)
        v = np.zeros(0)
    return sp.csr_matrix((v, (r, c)), shape=(fine.N, coarse.N))


class Hierarchy:
    """All levels of the V-cycle, transfers between them and the coarse LU."""

    def __init__(self, prob: W.Problem, levels=None):
        self.prob = prob
        seq = level_sequence(prob) if levels is None else levels
        self.levels = []
        for (n, p) in seq:
            lev = Level(prob, n, p)
            if lev.geom.n_active == 0:
                self.levels = []                          # drop everything coarser than an empty level
                continue
            self.levels.append(lev)
        if not self.levels:
            raise ValueError("finest level has no active cells")
        self.P = [None] + [prolongation(self.levels[l - 1], self.levels[l]) for l in range(1, len(self.levels))]
        self.R = [None] + [P.T.tocsr() for P in self.P[1:]]          # Eq. 18
        A0 = self.levels[0].A.toarray()
        self.coarse_lu = sla.lu_factor(A0)

    @property
    def finest(self) -> Level:
        return self.levels[-1]

    def vcycle(self, r: np.ndarray, level: int | None = None, correction=None) -> np.ndarray:
        """One V-cycle z = M^{-1} r (Sec. 3): zero initial guess on every level, pre-smooth
        (forward colours), residual, restrict, recurse, prolongate and add, post-smooth
        (reverse colours); the coarsest level is solved directly.  `correction(level, z, r)`,
        if given, updates z in place after the finest level's post-smoothing (the learned
        boundary-cell correction)."""
        top = len(self.levels) - 1
        l = top if level is None else level
        lev = self.levels[l]
        if l == 0:
            return sla.lu_solve(self.coarse_lu, r)
        z = np.zeros(lev.N)
        ssor = getattr(self.prob, "ssor_each", 0)
        smoother = getattr(self.prob, "smoother", 0)
        for _ in range(self.prob.pre_smooth):
            if smoother == 1:
                lev.block_jacobi_step(z, r)
            elif smoother == 2:
                lev.chebyshev(z, r)
            else:
                lev.coloured_sweep(z, r, reverse=False)
                if ssor:
                    lev.coloured_sweep(z, r, reverse=True)
        res = r - lev.A @ z
        zc = self.vcycle(self.R[l] @ res, l - 1)
        z += self.P[l] @ zc
        for _ in range(self.prob.post_smooth):
            if smoother == 1:
                lev.block_jacobi_step(z, r)
            elif smoother == 2:
                lev.chebyshev(z, r)
            else:
                if ssor:
                    lev.coloured_sweep(z, r, reverse=False)
                lev.coloured_sweep(z, r, reverse=True)
        if correction is not None and l == top:
            correction(lev, z, r)
        return z

"""Assembled DG-SBM operator and right-hand side on one level, plain FP64 (Sec. 2.2, Eqs. 7, 10, 11).

Bilinear form a_h(u, v) (Eq. 11), one-sided traces taken from the owning cell:
  volume          sum_K int_K grad u . grad v                                      (Eq. 10)
  interior faces  int_F [ -{d_n u}[[v]] - {d_n v}[[u]] + sigma_F [[u]][[v]] ]       (Eq. 10)
                  n from K- to K+, [[w]] = w- - w+, {w} = (w- + w+)/2
  surrogate faces int_F [ -(d_n~ u) v - alpha (d_n~ v)(u + d.grad u) + sigma_G (u + d.grad u) v ]
Right-hand side (Eq. 11):
  sum_K int_K f v + sum_F int_F [ -alpha (d_n~ v) g(x~ + d) + sigma_G g(x~ + d) v ]

Readings (the paper leaves these open):
  * Extension operator (Eqs. 6-7): on the left-hand side the trial function is extended to
    the true boundary as u(x~) + d . grad u(x~) (extension = 0, the first-order Taylor form
    of Eq. 6); the data term on the right is g(x~ + d); the test function is the plain v.
    extension = 1 instead evaluates the cell's polynomial at x~ + d (the whole Taylor series
    of the discrete polynomial); the optimal O(h^(p+1)) L2 rates printed in Sec. 5.1 for
    p = 2, 3 are reproduced only with this form.
  * Penalties: sigma_F = c_F (p_l+1)^2 / h_l and sigma_G = c_G (p_l+1)^2 / h_l.
  * Quadrature: (p+1)-point Gauss-Legendre on cells and faces for the form (exact for the
    polynomial integrands on Cartesian cells), (p+3) points for f and for the L2 error.
  * Matrix convention: row = test function, column = trial function, A u = b.
Element matrices are computed here by looping over quadrature points with the full
dim-dimensional basis functions (no one-dimensional factorisation).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import workloads as W
from . import fields
from . import quadrature as Q
from .geometry import LevelGeometry


def _face_points(p: int, dim: int, direction: int, side: int):
    """Reference points and weights of the tensor Gauss-Legendre rule on face (direction, side)."""
    nodes, wts = Q.gauss_legendre(p + 1)
    tang = Q.multi_indices(p + 1, dim - 1) if dim > 1 else np.zeros((1, 0), dtype=np.int64)
    xi = np.zeros((len(tang), dim))
    xi[:, direction] = float(side)
    w = np.ones(len(tang))
    for t, k in enumerate([k for k in range(dim) if k != direction]):
        xi[:, k] = nodes[tang[:, t]]
        w *= wts[tang[:, t]]
    return xi, w


class Discretisation:
    """Element matrices, the assembled sparse matrix A and the RHS b on one level."""

    def __init__(self, prob: W.Problem, geom: LevelGeometry, assemble: bool = True):
        self.prob, self.geom = prob, geom
        p, dim, h = geom.p, geom.dim, geom.h
        self.p, self.dim, self.h = p, dim, h
        self.nb = (p + 1) ** dim
        self.alpha = prob.alpha
        self.sigma_F = prob.sigma_face_c * (p + 1) ** 2 / h
        self.sigma_G = prob.sigma_bnd_c * (p + 1) ** 2 / h

        # volume stiffness: int_K grad phi_j . grad phi_i  (Eq. 10, first term)
        pts, wts = Q.tensor_rule(p + 1, dim)
        _, g = Q.tensor_basis(p, dim, pts)
        g = g / h
        self.K_vol = np.zeros((self.nb, self.nb))
        for q in range(len(wts)):
            self.K_vol += wts[q] * h ** dim * (g[q] @ g[q].T)

        # interior face blocks per direction (Eq. 10, face terms), test row, trial column
        self.F_blocks = []
        for direction in range(dim):
            xm, w = _face_points(p, dim, direction, 1)     # face seen from K- (its upper face)
            xp, _ = _face_points(p, dim, direction, 0)     # same face seen from K+
            phm, gm = Q.tensor_basis(p, dim, xm)
            php, gp = Q.tensor_basis(p, dim, xp)
            dnm, dnp = gm[:, :, direction] / h, gp[:, :, direction] / h
            blocks = {}
            for ti, (pv, sv) in enumerate(((phm, 1.0), (php, -1.0))):        # test side (-, +)
                for tj, (pu, su) in enumerate(((phm, 1.0), (php, -1.0))):    # trial side (-, +)
                    dv = dnm if ti == 0 else dnp
                    du = dnm if tj == 0 else dnp
                    M = np.zeros((self.nb, self.nb))
                    for t in range(len(w)):
                        jump_v = sv * pv[t]                 # [[v]] for test functions on side ti
                        jump_u = su * pu[t]
                        avg_du = 0.5 * du[t]
                        avg_dv = 0.5 * dv[t]
                        M += w[t] * h ** (dim - 1) * (-np.outer(jump_v, avg_du) - np.outer(avg_dv, jump_u)
                                                      + self.sigma_F * np.outer(jump_v, jump_u))
                    blocks["mp"[ti] + "mp"[tj]] = M
            self.F_blocks.append(blocks)

        self.sbm_blocks = [self.surrogate_face_matrix(f) for f in range(len(geom.faces))]
        self._faces_of = {}
        for f, (a, _d, _s) in enumerate(geom.faces):
            self._faces_of.setdefault(a, []).append(f)
        if assemble:                       # assemble=False: blocks on demand only (large meshes)
            self._assemble()

    # ------------------------------------------------------------------ surrogate faces
    def surrogate_face_matrix(self, f: int) -> np.ndarray:
        """Nitsche-SBM terms of Eq. 7 on surrogate face f, with the Taylor-extended trial u + d.grad u."""
        p, dim, h = self.p, self.dim, self.h
        _cell, direction, side = self.geom.faces[f]
        d = self.geom.face_d[f]
        xi, w = _face_points(p, dim, direction, side)
        ph, g = Q.tensor_basis(p, dim, xi)
        g = g / h
        nsign = 1.0 if side == 1 else -1.0
        dn = nsign * g[:, :, direction]
        if self.prob.extension == 1:
            ext_all, _ = Q.tensor_basis(p, dim, xi + d / h)  # phi_j(x~ + d)
        M = np.zeros((self.nb, self.nb))
        for t in range(len(w)):
            ext = ext_all[t] if self.prob.extension == 1 else ph[t] + g[t] @ d[t]   # extended trial phi_j
            M += w[t] * h ** (dim - 1) * (-np.outer(ph[t], dn[t])
                                          - self.alpha * np.outer(dn[t], ext)
                                          + self.sigma_G * np.outer(ph[t], ext))
        return M

    # ------------------------------------------------------------------ assembly
    def diag_block(self, a: int) -> np.ndarray:
        """A_KK for active cell a: volume + its own halves of interior faces + surrogate faces (Eq. 14)."""
        geom = self.geom
        D = self.K_vol.copy()
        idx = geom.cell_idx[a]
        for direction in range(self.dim):
            for side in (0, 1):
                nb = geom.neighbour(idx, direction, side)
                if nb >= 0 and geom.bg2act[nb] >= 0:
                    D += self.F_blocks[direction]["mm" if side == 1 else "pp"]
        for f in self._faces_of.get(a, []):
            D += self.sbm_blocks[f]
        return D

    def offdiag_blocks(self, a: int):
        """[(neighbour active id, A_K,N block)] for the interior-face neighbours of cell a."""
        geom = self.geom
        out = []
        idx = geom.cell_idx[a]
        for direction in range(self.dim):
            for side in (0, 1):
                nb = geom.neighbour(idx, direction, side)
                if nb >= 0 and geom.bg2act[nb] >= 0:
                    out.append((int(geom.bg2act[nb]), self.F_blocks[direction]["mp" if side == 1 else "pm"]))
        return out

    def _assemble(self):
        geom, nb = self.geom, self.nb
        nact = geom.n_active
        loc = np.arange(nb)
        Ri = np.repeat(loc, nb)
        Cj = np.tile(loc, nb)
        rows, cols, vals = [], [], []
        # diagonal blocks
        self.diag = np.zeros((nact, nb, nb))
        for a in range(nact):
            self.diag[a] = self.diag_block(a)
        base = (np.arange(nact) * nb)[:, None]
        rows.append((base + Ri[None, :]).reshape(-1))
        cols.append((base + Cj[None, :]).reshape(-1))
        vals.append(self.diag.reshape(-1))
        # off-diagonal blocks of interior faces
        for direction in range(self.dim):
            sel = geom.interior_faces[geom.interior_faces[:, 2] == direction]
            if len(sel) == 0:
                continue
            am, ap = sel[:, 0][:, None] * nb, sel[:, 1][:, None] * nb
            Bmp, Bpm = self.F_blocks[direction]["mp"], self.F_blocks[direction]["pm"]
            rows += [(am + Ri).reshape(-1), (ap + Ri).reshape(-1)]
            cols += [(ap + Cj).reshape(-1), (am + Cj).reshape(-1)]
            vals += [np.tile(Bmp.reshape(-1), len(sel)), np.tile(Bpm.reshape(-1), len(sel))]
        N = nact * nb
        self.A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(N, N)).tocsr()
        self.A.sum_duplicates()

    # ------------------------------------------------------------------ right-hand side
    def rhs(self) -> np.ndarray:
        """b of Eq. 11: volume source with (p+3)-point Gauss-Legendre + surrogate-face data terms."""
        geom, p, dim, h = self.geom, self.p, self.dim, self.h
        kind = self.prob.exact
        pts, wts = Q.tensor_rule(p + 3, dim)
        ph, _ = Q.tensor_basis(p, dim, pts)
        corners = geom.lo + h * geom.cell_idx
        X = corners[:, None, :] + h * pts[None, :, :]
        fv = fields.f_source(kind, X)                         # (nact, nq)
        b = (h ** dim) * (fv * wts[None, :]) @ ph             # (nact, nb)
        for f, (a, direction, side) in enumerate(geom.faces):
            xi, w = _face_points(p, dim, direction, side)
            phf, gf = Q.tensor_basis(p, dim, xi)
            nsign = 1.0 if side == 1 else -1.0
            dn = nsign * gf[:, :, direction] / h
            gval = fields.u_exact(kind, geom.face_xt[f] + geom.face_d[f])
            for t in range(len(w)):
                b[a] += w[t] * h ** (dim - 1) * gval[t] * (self.sigma_G * phf[t] - self.alpha * dn[t])
        return b.reshape(-1)

    # ------------------------------------------------------------------ helpers
    def interpolate(self, kind: int) -> np.ndarray:
        """Nodal interpolant of the manufactured solution (values at the cell's Gauss-Legendre nodes)."""
        geom, p, dim, h = self.geom, self.p, self.dim, self.h
        nodes_ref, _ = Q.tensor_rule(p + 1, dim)
        X = (geom.lo + h * geom.cell_idx)[:, None, :] + h * nodes_ref[None, :, :]
        return fields.u_exact(kind, X).reshape(-1)

    def l2_error(self, uh: np.ndarray, kind: int | None = None) -> float:
        """|| u - u_h ||_{L2(surrogate domain)} with (p+3)-point Gauss-Legendre per active cell."""
        kind = self.prob.exact if kind is None else kind
        geom, p, dim, h = self.geom, self.p, self.dim, self.h
        pts, wts = Q.tensor_rule(p + 3, dim)
        ph, _ = Q.tensor_basis(p, dim, pts)
        X = (geom.lo + h * geom.cell_idx)[:, None, :] + h * pts[None, :, :]
        uex = fields.u_exact(kind, X)
        uhq = uh.reshape(geom.n_active, self.nb) @ ph.T
        return float(np.sqrt(np.sum((uex - uhq) ** 2 * wts[None, :]) * h ** dim))

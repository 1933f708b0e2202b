"""C-ABI library checks that need no GPU: exported symbols, argument validation, and the
host-side set-up (geometry, layout, element data, right-hand side) against the oracle."""
import re
import os

import numpy as np
import pytest

import workloads as W
from oracle.dgsbm import Discretisation
from oracle.geometry import LevelGeometry
from oracle import multigrid as MG

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "sbm.h")


def header_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(sbm_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_symbol(libsbm):
    names = header_functions()
    assert len(names) >= 18
    lib = libsbm.load_library()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(libsbm.SYMBOLS)


def test_bad_descriptor_is_rejected(libsbm):
    prob = W.disk2d_p1(8, 0)
    for bad in (dict(p=4), dict(dim=4), dict(lam=1.5), dict(n=0)):
        with pytest.raises(libsbm.SbmError) as e:
            libsbm.HostSetup(prob.replace(**bad))
        assert e.value.code == -1
    with pytest.raises(libsbm.SbmError) as e:             # unequal box extents: cells not square
        libsbm.HostSetup(prob.replace(hi=(1.0, 2.0, 1.0)))
    assert e.value.code == -1


def test_empty_domain_is_reported(libsbm):
    prob = W.disk2d_p1(8, 0).replace(shape=W.Shape(kind=W.SHAPE_DISK, center=(5.0, 5.0, 0.0), radius=0.1))
    with pytest.raises(libsbm.SbmError) as e:
        libsbm.HostSetup(prob)
    assert e.value.code == -6


def test_device_calls_refuse_host_only_context(libsbm):
    import ctypes
    hs = libsbm.HostSetup(W.disk2d_p1(8, 0))
    lib = hs.lib
    x = np.zeros(hs.info()["n_dof"])
    assert lib.sbm_apply(hs.ctx, -1, 0, x.ctypes.data, x.ctypes.data + 8) == -1
    assert lib.sbm_vcycle(hs.ctx, 0, x.ctypes.data, x.ctypes.data + 8) == -1
    assert b"host-only" in lib.sbm_last_error()


def _perm(hs, geom, level=-1):
    coords = hs.layout(level)
    lin = coords[:, 0].astype(np.int64) + geom.n * coords[:, 1].astype(np.int64)
    if geom.dim == 3:
        lin += geom.n * geom.n * coords[:, 2].astype(np.int64)
    return geom.bg2act[lin]


CASES = [W.disk2d_p1(16, 0), W.star2d_p2(16, 1), W.disk2d_p1(8, 2).replace(p=3), W.sphere3d(8, 1, 2),
         W.sphere3d(6, 2, 3), W.ellipsoid3d_p3(6, 4), W.disk2d_p1(16, 0).replace(extension=1, p=2),
         W.Problem(dim=2, n=8, p=2, shape=W.box(0.5)), W.paper_disk(1, 3, 0.25)]


@pytest.mark.parametrize("prob", CASES, ids=lambda p: f"{p.name}_p{p.p}_e{p.extension}")
def test_host_setup_matches_oracle(libsbm, prob):
    """Compact layout is a colour-major permutation of the oracle's active cells; the host
    operator and right-hand side equal the oracle's assembled A and b; surrogate faces and
    shifts agree (independent implementations of Secs. 2.1, 2.2 and 4.2)."""
    hs = libsbm.HostSetup(prob)
    g = LevelGeometry(prob, prob.n, prob.p)
    D = Discretisation(prob, g)
    perm = _perm(hs, g)
    assert (perm >= 0).all() and len(perm) == g.n_active and len(set(perm)) == len(perm)
    info = hs.info()
    cs = info["colour_start"]
    colours = MG.colour_of(g.cell_idx[perm])
    for c in range(2 ** prob.dim):                       # colour-major order
        assert np.all(colours[cs[c]:cs[c + 1]] == c)
    nb = D.nb
    dof = (perm[:, None] * nb + np.arange(nb)[None, :]).reshape(-1)
    x = W.random_vector(len(dof), 7)
    xo = np.zeros(len(dof))
    xo[dof] = x
    y, yo = hs.host_apply(x), (D.A @ xo)[dof]
    assert np.linalg.norm(y - yo) <= 1e-13 * np.linalg.norm(yo)
    b, bo = hs.host_rhs(), D.rhs()[dof]
    assert np.linalg.norm(b - bo) <= 1e-13 * np.linalg.norm(bo)
    cell, slot, d = hs.export_geometry()
    assert len(cell) == len(g.faces) == info["n_sface"]
    ofaces = {(int(a), 2 * dr + s): k for k, (a, dr, s) in enumerate(g.faces)}
    for f in range(len(cell)):
        k = ofaces[(int(perm[cell[f]]), int(slot[f]))]
        assert np.abs(d[f][:, :prob.dim] - g.face_d[k]).max() <= 1e-12


def test_host_setup_all_levels_match_oracle(libsbm):
    prob = W.sphere3d(8, 2, 1)
    hs = libsbm.HostSetup(prob)
    H = MG.Hierarchy(prob)
    assert hs.num_levels == len(H.levels)
    for l, lev in enumerate(H.levels):
        info = hs.info(l)
        assert (info["n"], info["p"], info["n_active"]) == (lev.n, lev.p, lev.geom.n_active)
        perm = _perm(hs, lev.geom, l)
        dof = (perm[:, None] * lev.nb + np.arange(lev.nb)[None, :]).reshape(-1)
        x = W.random_vector(len(dof), l)
        xo = np.zeros(len(dof))
        xo[dof] = x
        y, yo = hs.host_apply(x, l), (lev.A @ xo)[dof]
        assert np.linalg.norm(y - yo) <= 1e-13 * np.linalg.norm(yo)


@pytest.mark.parametrize("prob", [W.disk2d_p1(32, 0), W.star2d_p2(64, 1), W.sphere3d(16, 1, 2), W.ellipsoid3d_p3(12, 0)],
                         ids=["disk2d_p1_n32", "star2d_p2_n64", "sphere3d_p1_n16", "ellipsoid3d_p3_n12"])
def test_compact_order_colour_major_boundary_cells_by_face_set(libsbm, prob):
    """Every level's compact order: colour-major (colour = parity bits of the cell index); within a
    colour the cells with surrogate faces first, ordered by their set of surrogate-face slots and
    then by background index, then the interior cells by background index."""
    hs = libsbm.HostSetup(prob)
    dim = prob.dim
    for level in range(hs.num_levels):
        info = hs.info(level)
        n, na = info["n"], info["n_active"]
        coords = hs.layout(level).astype(np.int64)
        lin = libsbm.compact_to_natural(coords, n, dim)
        colour = sum(((coords[:, k] & 1) << k) for k in range(dim))
        cell, slot, _ = hs.export_geometry(level)
        mask = np.zeros(na, dtype=np.int64)
        np.bitwise_or.at(mask, cell, 1 << slot.astype(np.int64))
        cs = info["colour_start"]
        for c in range(2 ** dim):
            a0, a1, nb = cs[c], cs[c + 1], info["colour_nbnd"][c]
            assert np.all(colour[a0:a1] == c)
            bnd, inner = slice(a0, a0 + nb), slice(a0 + nb, a1)
            assert np.all(mask[bnd] != 0) and np.all(mask[inner] == 0)
            key = mask[bnd] * (n ** dim) + lin[bnd]
            assert np.all(np.diff(key) > 0)
            assert np.all(np.diff(lin[inner]) > 0)
        assert cs[2 ** dim] == na
    hs.close()

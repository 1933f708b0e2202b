"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks the oracle against something other than itself: closed forms, exact
reproduction properties of the discretisation, brute force on tiny inputs, library
routines for special cases, and numbers printed in the paper (tests/golden/).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import workloads as W
from oracle import geometry as G
from oracle import krylov as K
from oracle import multigrid as MG
from oracle import quadrature as Q
from oracle.dgsbm import Discretisation

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ quadrature and basis
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_gauss_legendre_degree_of_exactness(n):
    x, w = Q.gauss_legendre(n)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
    assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-10    # not exact beyond 2n-1


@pytest.mark.parametrize("p", [1, 2, 3])
def test_lagrange_basis_interpolates_polynomials(p):
    nodes, _ = Q.gauss_legendre(p + 1)
    assert np.allclose(Q.lagrange_values(nodes, nodes), np.eye(p + 1), atol=1e-14)
    xs = np.linspace(-0.3, 1.4, 17)
    V, D = Q.lagrange_values(nodes, xs), Q.lagrange_derivs(nodes, xs)
    rng = np.random.default_rng(p)
    c = rng.normal(size=p + 1)
    poly = np.polynomial.Polynomial(c)
    assert np.allclose(poly(nodes) @ V, poly(xs), atol=1e-12)
    assert np.allclose(poly(nodes) @ D, poly.deriv()(xs), atol=1e-11)
    # degree-1 case against the closed form l_0(x) = (x - x1) / (x0 - x1)
    if p == 1:
        assert np.allclose(V[0], (xs - nodes[1]) / (nodes[0] - nodes[1]))
        assert np.allclose(nodes, [0.5 - 0.5 / math.sqrt(3), 0.5 + 0.5 / math.sqrt(3)])


# ------------------------------------------------------------------ geometry
def test_box_kappa_exact_and_disk_area():
    prob = W.Problem(dim=2, n=16, p=1, shape=W.box(0.5))
    kap = G.volume_fractions(prob, 16)
    # box [-0.5,0.5]^2 on a 16^2 grid over [-1,1]^2: cells 4..11 inside, others outside
    expect = np.zeros((16, 16))
    expect[4:12, 4:12] = 1.0
    assert np.array_equal(kap, expect)
    # disk area from kappa: sampling error O(h * perimeter / s)
    prob = W.disk2d_p1(64, 3)
    kap = G.volume_fractions(prob, 64)
    h = 2.0 / 64
    assert abs(kap.sum() * h * h - math.pi * 0.49) < 2 * math.pi * 0.7 * h / 16


def test_disk_shift_closed_form():
    prob = W.disk2d_p1(16, 5)
    g = G.LevelGeometry(prob, 16, 2)
    c = np.array(prob.shape.center[:2])
    for xt, d in zip(g.face_xt, g.face_d):
        x = xt + d
        assert np.allclose(np.linalg.norm(x - c, axis=1), 0.7, atol=1e-14)
        cross = (x - c)[:, 0] * d[:, 1] - (x - c)[:, 1] * d[:, 0]      # d parallel to the radius
        assert np.allclose(cross, 0.0, atol=1e-14)


@pytest.mark.parametrize("shape", [W.star(1), W.random_star(1007), W.complex2d()])
def test_newton_closest_point_2d_brute_force(shape):
    """Newton on Eqs. 21-22 against a dense sampling of the boundary curve in polar form."""
    rng = np.random.default_rng(0)
    th = np.linspace(0, 2 * np.pi, 400001)[:-1]
    if shape.kind == W.SHAPE_STAR:
        r = shape.radius * (1 + shape.amp * np.sin(shape.freq * th + shape.phase))
    else:   # complex2d: (1 - 3/4 sin^2(pi x)) r^2 = 1/5 along each ray, solved by bisection in r
        lo_, hi_ = np.zeros_like(th), np.full_like(th, 2.0)
        for _ in range(60):
            mid = 0.5 * (lo_ + hi_)
            X = np.stack([mid * np.cos(th), mid * np.sin(th)], axis=1)
            inside = G.phi(shape, X) < 0
            lo_ = np.where(inside, mid, lo_)
            hi_ = np.where(inside, hi_, mid)
        r = 0.5 * (lo_ + hi_)
    curve = np.stack([r * np.cos(th), r * np.sin(th)], axis=1) + np.array(shape.center[:2])
    for _ in range(25):
        ang = rng.uniform(0, 2 * np.pi)
        rad = np.interp(ang, th, r) * (1 + rng.uniform(-0.08, 0.08))
        xt = np.array([rad * np.cos(ang), rad * np.sin(ang)]) + np.array(shape.center[:2])
        x = G.closest_point(shape, xt)
        assert abs(G.phi(shape, x)) < 1e-12
        dist_brute = np.min(np.linalg.norm(curve - xt, axis=1))
        assert np.linalg.norm(x - xt) <= dist_brute + 1e-6
        assert np.linalg.norm(x - xt) >= dist_brute - 2e-5


def test_newton_closest_point_ellipsoid():
    shape = W.ellipsoid(4)
    rng = np.random.default_rng(1)
    R = np.array(shape.rot).reshape(3, 3)
    semi = np.array(shape.semi)
    u, v = np.meshgrid(np.linspace(0, np.pi, 801), np.linspace(0, 2 * np.pi, 1601), indexing="ij")
    loc = np.stack([np.sin(u) * np.cos(v), np.sin(u) * np.sin(v), np.cos(u)], axis=-1).reshape(-1, 3) * semi
    surf = loc @ R.T
    for _ in range(15):
        dirn = rng.normal(size=3)
        dirn /= np.linalg.norm(dirn)
        s = 1.0 / np.linalg.norm((R.T @ dirn) / semi)          # boundary along this ray
        xt = dirn * s * (1 + rng.uniform(-0.1, 0.1))
        x = G.closest_point(shape, xt)
        assert abs(G.phi(shape, x)) < 1e-12
        g, _ = G.grad_hess(shape, x)
        assert np.linalg.norm(np.cross(g, x - xt)) < 1e-10 * np.linalg.norm(g)   # normal to the surface
        dist_brute = np.min(np.linalg.norm(surf - xt, axis=1))
        assert np.linalg.norm(x - xt) <= dist_brute + 1e-9
        assert np.linalg.norm(x - xt) >= dist_brute - 5e-3


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def test_paper_shift_ranges_golden():
    """Sec. 5, figure shift_distribution: min/max normalised shifts, unit disk, p = 3."""
    cache = {}
    for lam, level, mn, mx in _golden("paper_shift_range.txt"):
        key = (lam, int(level))
        if key not in cache:
            prob = W.paper_disk(int(level), 3, lam)
            g = G.LevelGeometry(prob, prob.n, 3)
            vals = []
            for (_a, dr, side), d in zip(g.faces, g.face_d):
                nt = np.zeros(2)
                nt[dr] = 1.0 if side == 1 else -1.0
                vals.append(np.sign(d @ nt) * np.linalg.norm(d, axis=1) / g.h)
            vals = np.concatenate(vals)
            cache[key] = (vals.min(), vals.max())
        omin, omax = cache[key]
        assert abs(omax - mx) < 6e-4, (lam, level, omax, mx)
        if not math.isnan(mn):
            assert abs(omin - mn) < 6e-4, (lam, level, omin, mn)


# ------------------------------------------------------------------ the discrete operator
CASES_LINEAR = [
    (W.disk2d_p1(16, 1), 1), (W.disk2d_p1(16, 1), 2), (W.disk2d_p1(8, 2), 3),
    (W.star2d_p2(16, 3), 2), (W.star2d_p2(16, 3), 3),
    (W.sphere3d(8, 1, 4), 1), (W.sphere3d(6, 2, 4), 2), (W.ellipsoid3d_p3(6, 5), 3),
]


@pytest.mark.parametrize("prob,p", CASES_LINEAR, ids=lambda v: getattr(v, "name", str(v)))
def test_linear_solution_reproduced(prob, p):
    """The Taylor extension is exact for linear u (Eqs. 5-7), so A u_I = b with f = 0, g = u
    for any shift d; the solve returns u_I.  A dropped/mis-signed consistency or SBM term fails."""
    prob = prob.replace(p=p, exact=W.EXACT_LINEAR)
    g = G.LevelGeometry(prob, prob.n, p)
    D = Discretisation(prob, g)
    uI, b = D.interpolate(W.EXACT_LINEAR), D.rhs()
    assert len(g.faces) > 0 and np.abs(np.concatenate(g.face_d)).max() > 0.01 * g.h
    assert np.linalg.norm(D.A @ uI - b) <= 1e-12 * np.linalg.norm(b)
    x = spla.spsolve(D.A.tocsc(), b)
    assert np.linalg.norm(x - uI) <= 1e-10 * np.linalg.norm(uI)


@pytest.mark.parametrize("dim,n,p", [(2, 16, 1), (2, 8, 2), (2, 8, 3), (3, 4, 1), (3, 4, 2)])
def test_box_symmetric_positive_definite(dim, n, p):
    """d = 0 on a body-fitted box: the form is symmetric for alpha = 1 (Sec. 2, Eq. 3) and SPD."""
    prob = W.Problem(dim=dim, n=n, p=p, shape=W.box(0.5))
    g = G.LevelGeometry(prob, n, p)
    assert np.abs(np.concatenate(g.face_d)).max() == 0.0
    A = Discretisation(prob, g).A.toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    sla.cholesky(A)                                        # raises if not positive definite


@pytest.mark.parametrize("p,kind", [(2, W.EXACT_QUADRATIC), (3, W.EXACT_QUADRATIC)])
def test_box_polynomial_solution_exact(p, kind):
    """Galerkin consistency on a fitted boundary: u in V_h is reproduced exactly (tests the
    volume source quadrature and every consistency term)."""
    for dim, n in ((2, 8), (3, 4)):
        prob = W.Problem(dim=dim, n=n, p=p, shape=W.box(0.5), exact=kind)
        g = G.LevelGeometry(prob, n, p)
        D = Discretisation(prob, g)
        x = spla.spsolve(D.A.tocsc(), D.rhs())
        uI = D.interpolate(kind)
        assert np.linalg.norm(x - uI) <= 1e-11 * np.linalg.norm(uI)
        assert D.l2_error(x) < 1e-11


def test_h_convergence_taylor_extension():
    """First-order Taylor shift (Eq. 6): O(h^2) L2 convergence on the disk for p = 1."""
    errs = []
    for n in (16, 32, 64):
        prob = W.disk2d_p1(n, 0)
        g = G.LevelGeometry(prob, n, 1)
        D = Discretisation(prob, g)
        errs.append(D.l2_error(spla.spsolve(D.A.tocsc(), D.rhs())))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.35), (errs, rates)


@pytest.mark.slow
def test_paper_l2_bands_golden():
    """Sec. 5.1 figure convergence_results_l2: with the polynomial extension the errors over
    lambda in {1, .75, .5, .25} sit within a factor 4 of the paper's band (geometric means),
    and fall at the optimal rate p + 1."""
    rows = [r for r in _golden("paper_l2_bands.txt") if r[1] <= 3]
    ours = {}
    for p, level, up, lo in rows:
        errs = []
        for lam in (1.0, 0.75, 0.5, 0.25):
            prob = W.paper_disk(int(level), int(p), lam)
            g = G.LevelGeometry(prob, prob.n, int(p))
            D = Discretisation(prob, g)
            errs.append(D.l2_error(spla.spsolve(D.A.tocsc(), D.rhs())))
        gm = math.exp(np.mean(np.log(errs)))
        ours[(p, level)] = gm
        assert gm / math.sqrt(up * lo) < 4.0 and math.sqrt(up * lo) / gm < 4.0, (p, level, errs, up, lo)
    for p in (1, 2, 3):
        rate = math.log2(ours[(p, 1.0)] / ours[(p, 3.0)]) / 2
        assert abs(rate - (p + 1)) < 0.6, (p, rate)


@pytest.mark.slow
def test_paper_complex_l2_bands_golden():
    """Sec. 5.4 figure solution_complex (right panel), the complex deformed domain with u = phi + 1.
    p = 1: the geometric mean of our errors over lambda in {1, .75, .5, .25} lies within a factor 4
    of the paper's band at levels 1-4.  p = 2, 3: every error lies at or below the paper's upper
    band and the rate between levels 3 and 4 is at least p; the paper interpolates phi by finite
    elements, which perturbs where g = 1 is imposed and raises its p >= 2 errors, while phi is
    analytic here (reading R7), so only the upper side of its band binds."""
    bands = {(int(p), int(l)): (up, lo) for p, l, up, lo in _golden("paper_complex_l2_bands.txt")}
    for p in (1, 2, 3):
        gms = {}
        for level in (1, 2, 3, 4):
            errs = []
            for lam in (1.0, 0.75, 0.5, 0.25):
                prob = W.paper_complex2d(level, p, lam)
                g = G.LevelGeometry(prob, prob.n, p)
                D = Discretisation(prob, g)
                errs.append(D.l2_error(spla.spsolve(D.A.tocsc(), D.rhs())))
            up, lo = bands[(p, level)]
            gm = math.exp(np.mean(np.log(errs)))
            gms[level] = gm
            if p == 1:
                ref = math.sqrt(up * lo)
                assert gm / ref < 4.0 and ref / gm < 4.0, (p, level, errs, up, lo)
            elif level >= 2:
                assert max(errs) <= up * 1.05, (p, level, errs, up)
        assert math.log2(gms[3] / gms[4]) >= p, (p, gms)


@pytest.mark.parametrize("kind", [W.EXACT_SINPROD, W.EXACT_EXPCOS, W.EXACT_LINEAR, W.EXACT_COSSIN,
                                  W.EXACT_QUADRATIC, W.EXACT_PHIP1])
@pytest.mark.parametrize("dim", [2, 3])
def test_manufactured_sources_are_minus_laplacian(kind, dim):
    """f = -Laplace(u) for every manufactured solution, against fourth-order central differences of
    u at random points (the sources were derived by hand)."""
    from oracle import fields
    if kind == W.EXACT_PHIP1 and dim == 3:
        pytest.skip("the complex-domain solution is two-dimensional")
    rng = np.random.default_rng(kind)
    X = rng.uniform(-0.9, 0.9, size=(40, dim))
    h = 1e-3
    lap = np.zeros(len(X))
    for k in range(dim):
        e = np.zeros(dim)
        e[k] = h
        u = lambda s: fields.u_exact(kind, X + s * e)
        lap += (-u(2) + 16 * u(1) - 30 * u(0) + 16 * u(-1) - u(-2)) / (12 * h * h)
    f = fields.f_source(kind, X)
    assert np.allclose(f, -lap, rtol=1e-6, atol=1e-6 * (1 + np.abs(f).max())), np.abs(f + lap).max()


# ------------------------------------------------------------------ multigrid pieces
@pytest.mark.parametrize("dim,n,pf,pc", [(2, 8, 1, 1), (2, 8, 3, 1), (2, 8, 3, 2), (3, 8, 1, 1), (3, 4, 2, 1)])
def test_prolongation_reproduces_coarse_polynomials(dim, n, pf, pc):
    """Eq. 17: the embedding reproduces every coarse polynomial exactly on the fine cells."""
    prob = W.Problem(dim=dim, n=n, p=pf, shape=W.disk(dim, 0, radius=0.8), exact=W.EXACT_QUADRATIC)
    if pf == pc:       # h-transfer
        coarse, fine = MG.Level(prob, n // 2, pc), MG.Level(prob, n, pf)
        kind = W.EXACT_LINEAR
    else:              # p-transfer
        coarse, fine = MG.Level(prob, n, pc), MG.Level(prob, n, pf)
        kind = W.EXACT_QUADRATIC if pc >= 2 else W.EXACT_LINEAR
    P = MG.prolongation(coarse, fine)
    uc, uf = coarse.disc.interpolate(kind), fine.disc.interpolate(kind)
    # compare on fine cells whose parent is active (masked reading)
    hit = np.asarray(P.sum(axis=1)).reshape(-1) != 0
    assert hit.sum() > 0
    assert np.abs((P @ uc - uf)[hit]).max() < 1e-13
    # partition of unity of the coarse basis: row sums are 1 on hit rows
    assert np.allclose(np.asarray(P.sum(axis=1)).reshape(-1)[hit], 1.0, atol=1e-13)


def test_coloured_sweep_equals_sequential_block_gs():
    """Cells of one colour share no face, so the per-colour update equals the cell-by-cell
    successive correction of Eq. 16 in colour order; natural order gives a different map."""
    for prob in (W.disk2d_p1(16, 2).replace(p=2), W.sphere3d(6, 1, 1)):
        lev = MG.Level(prob, prob.n, prob.p)
        rng = np.random.default_rng(3)
        f = rng.normal(size=lev.N)
        u0 = rng.normal(size=lev.N)
        a = lev.coloured_sweep(u0.copy(), f)
        b = lev.block_gs_sequential(u0.copy(), f, lev.colour_order())
        c = lev.block_gs_sequential(u0.copy(), f, np.arange(lev.geom.n_active))
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
        assert np.linalg.norm(a - c) > 1e-6 * np.linalg.norm(b)
        a = lev.coloured_sweep(u0.copy(), f, reverse=True)
        b = lev.block_gs_sequential(u0.copy(), f, lev.colour_order(reverse=True))
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_red_black_sweep_equals_sequential_block_gs():
    """Red-black ordering: cells of equal index-sum parity share no face (a face changes one index
    by one), so the sweep over the even-parity colours, then the odd ones, equals the cell-by-cell
    successive correction (Eq. 16) in that cell order, differs from the 2^d-colour sweep, and a
    colouring that mixes parities within a step would not be a valid simultaneous update."""
    for prob in (W.disk2d_p1(16, 2).replace(p=2, ordering=1), W.sphere3d(6, 1, 1).replace(ordering=1)):
        lev = MG.Level(prob, prob.n, prob.p)
        par = lev.geom.cell_idx.sum(axis=1) % 2
        # no coupling between two cells of the same parity
        A = lev.A.tocoo()
        ca, cb = A.row // lev.nb, A.col // lev.nb
        off = ca != cb
        assert np.all(par[ca[off]] != par[cb[off]])
        rng = np.random.default_rng(4)
        f, u0 = rng.normal(size=lev.N), rng.normal(size=lev.N)
        order = np.concatenate([np.nonzero(par == 0)[0], np.nonzero(par == 1)[0]])
        for reverse in (False, True):
            a = lev.coloured_sweep(u0.copy(), f, reverse=reverse)
            o = order[::-1] if reverse else order
            b = lev.block_gs_sequential(u0.copy(), f, o)
            assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
        c = MG.Level(prob.replace(ordering=0), prob.n, prob.p).coloured_sweep(u0.copy(), f)
        assert np.linalg.norm(lev.coloured_sweep(u0.copy(), f) - c) > 1e-6 * np.linalg.norm(c)


def test_block_jacobi_step_and_convergence():
    """Additive block Jacobi: one step equals u + omega D^-1 (f - A u) with D the principal cell
    blocks of the dense matrix, and damped steps converge to A^-1 f on the SPD box."""
    prob = W.Problem(dim=2, n=8, p=2, shape=W.box(0.5), smoother=1, omega=0.6)
    lev = MG.Level(prob, 8, 2)
    A = lev.A.toarray()
    rng = np.random.default_rng(5)
    f, u0 = rng.normal(size=lev.N), rng.normal(size=lev.N)
    r = f - A @ u0
    expect = u0.copy()
    for a in range(lev.geom.n_active):
        s = lev.dofs(a)
        expect[s] += 0.6 * np.linalg.solve(A[s, s], r[s])
    got = lev.block_jacobi_step(u0.copy(), f)
    assert np.linalg.norm(got - expect) <= 1e-12 * np.linalg.norm(expect)
    # k steps multiply the error by (I - omega D^-1 A)^k, whose spectral radius is below 1 on the
    # SPD box for omega < 2 / lambda_max(D^-1 A): the iteration converges to A^-1 f
    Dinv = np.zeros_like(A)
    for a in range(lev.geom.n_active):
        s = lev.dofs(a)
        Dinv[s, s] = np.linalg.inv(A[s, s])
    E = np.eye(lev.N) - 0.6 * Dinv @ A
    assert np.abs(np.linalg.eigvals(E)).max() < 1.0
    x = np.linalg.solve(A, f)
    u = u0.copy()
    for _ in range(7):
        lev.block_jacobi_step(u, f)
    assert np.linalg.norm((u - x) - np.linalg.matrix_power(E, 7) @ (u0 - x)) <= 1e-10 * np.linalg.norm(u0 - x)


def test_power_iteration_estimates_lambda_max():
    """The power-iteration estimate of lambda_max(D^-1 A) lies below the spectral radius and within
    10% of it on the SPD box (where D^-1 A has a real positive spectrum); the start vector depends on
    the background cell index only."""
    prob = W.Problem(dim=2, n=8, p=2, shape=W.box(0.5), smoother=2)
    lev = MG.Level(prob, 8, 2)
    A = lev.A.toarray()
    Dinv = np.zeros_like(A)
    for a in range(lev.geom.n_active):
        s = lev.dofs(a)
        Dinv[s, s] = np.linalg.inv(A[s, s])
    ev = np.linalg.eigvals(Dinv @ A)
    rho = np.abs(ev).max()
    assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > 0
    lam = lev.lambda_max()
    assert lam <= rho * (1 + 1e-12) and lam >= 0.9 * rho, (lam, rho)
    v = MG.chebyshev_start(lev.geom.cell_idx, lev.nb).reshape(-1, lev.nb)
    perm = np.random.default_rng(0).permutation(lev.geom.n_active)
    assert np.array_equal(MG.chebyshev_start(lev.geom.cell_idx[perm], lev.nb).reshape(-1, lev.nb), v[perm])


def test_chebyshev_error_polynomial():
    """The Chebyshev smoother multiplies the error by the scaled Chebyshev polynomial
    p_m(t) = T_m((theta - t) / delta) / T_m(theta / delta) of t = D^-1 A (textbook Chebyshev
    semi-iteration), checked through the eigen-decomposition of D^-1 A on the SPD box, for degrees
    1 to 5; every eigencomponent inside the interval is damped by at least 1 / T_m(theta/delta)."""
    prob = W.Problem(dim=2, n=8, p=2, shape=W.box(0.5), smoother=2)
    lev = MG.Level(prob, 8, 2)
    A = lev.A.toarray()
    Dinv = np.zeros_like(A)
    for a in range(lev.geom.n_active):
        s = lev.dofs(a)
        Dinv[s, s] = np.linalg.inv(A[s, s])
    T = Dinv @ A
    b = MG.CHEB_SAFETY * lev.lambda_max()
    a_ = b / prob.cheb_ratio
    theta, delta = 0.5 * (b + a_), 0.5 * (b - a_)
    X = (theta * np.eye(lev.N) - T) / delta
    rng = np.random.default_rng(6)
    x = rng.normal(size=lev.N)
    f = A @ x
    u0 = rng.normal(size=lev.N)
    Tkm1, Tk = np.eye(lev.N), X.copy()                     # T_0(X), T_1(X) (three-term recurrence)
    for m in range(1, 6):
        if m > 1:
            Tkm1, Tk = Tk, 2 * X @ Tk - Tkm1
        scale = np.cosh(m * np.arccosh(theta / delta))     # T_m(theta / delta), theta / delta > 1
        u = lev.chebyshev(u0.copy(), f, degree=m)
        e0, e = u0 - x, u - x
        expect = Tk @ e0 / scale
        assert np.linalg.norm(e - expect) <= 1e-9 * np.linalg.norm(e0), (m, np.linalg.norm(e - expect))
        # eigencomponents of D^-1 A inside [a, b] are damped by at least 1 / T_m(theta / delta)
        w = np.linalg.eigvals(T).real
        inside = w[(w >= a_) & (w <= b)]
        pm = np.cos(m * np.arccos(np.clip((theta - inside) / delta, -1, 1))) / scale
        assert np.all(np.abs(pm) <= 1.0 / scale * (1 + 1e-9))


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1)])
def test_penalty_free_variant_reproduces_linear(dim, p):
    """The penalty-free form alpha = -1, sigma_Gamma = 0 (Sec. 2.1) is still consistent: the linear
    solution is reproduced exactly for any shift d (the SBM terms vanish on it with the Taylor
    extension), and the matrix is not symmetric on a curved boundary."""
    prob = (W.disk2d_p1(16, 1) if dim == 2 else W.sphere3d(8, 1, 4)).replace(p=p, alpha=-1.0, sigma_bnd_c=0.0,
                                                                              exact=W.EXACT_LINEAR)
    g = G.LevelGeometry(prob, prob.n, p)
    D = Discretisation(prob, g)
    uI = D.interpolate(W.EXACT_LINEAR)
    b = D.rhs()
    assert np.linalg.norm(D.A @ uI - b) <= 1e-12 * np.linalg.norm(b)
    x = spla.spsolve(D.A.tocsc(), b)
    assert np.linalg.norm(x - uI) <= 1e-10 * np.linalg.norm(uI)
    assert abs(D.A - D.A.T).max() > 1e-6 * abs(D.A).max()


def test_colour_groups_equal_colour_order():
    """Colour c(K) = sum_k (i_k mod 2) 2^k; face neighbours differ in one index parity, so colours
    with the same number of odd bits never couple.  The sweep in colour order 0..2^d-1 therefore
    equals the sweep that updates all colours with g odd bits at once, g = 0..d (reverse: d..0);
    the GPU smoother launches one such group per launch.  The pin: no face couples two colours of
    one group (the off-diagonal blocks of A between them vanish), and the grouped simultaneous
    update reproduces the oracle's coloured sweep exactly."""
    for prob in (W.star2d_p2(16, 1), W.sphere3d(6, 2, 1)):
        lev = MG.Level(prob, prob.n, prob.p)
        d, nb = prob.dim, lev.nb
        pop = np.array([bin(c).count("1") for c in range(2 ** d)])
        rows = []
        for g in range(d + 1):
            cells = np.concatenate([lev.cells_of_colour[c] for c in range(2 ** d) if pop[c] == g])
            idx = (cells[:, None] * nb + np.arange(nb)[None, :]).reshape(-1)
            rows.append((cells, idx))
            blk = lev.A[idx][:, idx].tocoo()
            same = (blk.row // nb) == (blk.col // nb)
            assert np.all(blk.data[~same] == 0.0)
        rng = np.random.default_rng(4)
        f, u0 = rng.normal(size=lev.N), rng.normal(size=lev.N)
        for reverse in (False, True):
            u = u0.copy()
            for g in (range(d, -1, -1) if reverse else range(d + 1)):
                cells, idx = rows[g]
                r = (f[idx] - lev.A[idx] @ u).reshape(len(cells), nb)
                u[idx] += lev.omega * np.einsum("kij,kj->ki", lev.diag_inv[cells], r).reshape(-1)
            ref = lev.coloured_sweep(u0.copy(), f, reverse=reverse)
            assert np.linalg.norm(u - ref) <= 1e-14 * np.linalg.norm(ref)
        # a colour order that is not grouped by odd-bit count gives a different map
        bad = lev.block_gs_sequential(u0.copy(), f, np.concatenate([lev.cells_of_colour[c] for c in
                                                                     [0, 3, 1, 2] + list(range(4, 2 ** d))]))
        assert np.linalg.norm(bad - lev.coloured_sweep(u0.copy(), f)) > 1e-8 * np.linalg.norm(bad)


def test_block_gs_converges_to_solution():
    """Repeated symmetric block Gauss-Seidel on an SPD system converges to A^{-1} f."""
    prob = W.Problem(dim=2, n=8, p=2, shape=W.box(0.5))
    lev = MG.Level(prob, 8, 2)
    f = np.random.default_rng(0).normal(size=lev.N)
    x = spla.spsolve(lev.A.tocsc(), f)
    u = np.zeros(lev.N)
    for _ in range(3000):
        lev.coloured_sweep(u, f)
        lev.coloured_sweep(u, f, reverse=True)
    assert np.linalg.norm(u - x) <= 1e-8 * np.linalg.norm(x)


@pytest.mark.parametrize("ssor_each", [0, 1])
def test_vcycle_symmetric_on_spd_box(ssor_each):
    """Forward pre-smoothing, backward post-smoothing and R = P^T make the V-cycle a symmetric
    operator when A is symmetric (Secs. 3.1-3.2); with full SSOR steps (forward then reverse,
    before and after the coarse correction) the post-smoother is still the adjoint of the
    pre-smoother, since an SSOR step is self-adjoint.  A wrong order breaks the symmetry by far
    more than rounding."""
    prob = W.Problem(dim=2, n=32, p=2, shape=W.box(0.5), coarsest_n=4, ssor_each=ssor_each)
    H = MG.Hierarchy(prob)
    rng = np.random.default_rng(0)
    r1, r2 = rng.normal(size=H.finest.N), rng.normal(size=H.finest.N)
    a, b = H.vcycle(r1) @ r2, r1 @ H.vcycle(r2)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_ssor_each_smooths_more_than_one_sweep():
    """Two-grid error reduction on the disk: a full SSOR step per smoothing step reduces the error
    of one V-cycle iteration at least as much as the single sweeps (the same colour order run
    twice over)."""
    rates = []
    for ssor in (0, 1):
        prob = W.disk2d_p1(16, 0).replace(ssor_each=ssor)
        H = MG.Hierarchy(prob)
        A = H.finest.A
        e = np.random.default_rng(2).normal(size=H.finest.N)
        for _ in range(3):
            e = e - H.vcycle(A @ e)
        rates.append(np.linalg.norm(e))
    assert rates[1] <= rates[0]


def test_vcycle_is_linear_and_exact_on_single_level():
    prob = W.disk2d_p1(8, 0)
    H = MG.Hierarchy(prob, levels=[(8, 1)])
    r = np.random.default_rng(1).normal(size=H.finest.N)
    x = np.linalg.solve(H.finest.A.toarray(), r)
    assert np.linalg.norm(H.vcycle(r) - x) <= 1e-12 * np.linalg.norm(x)


# ------------------------------------------------------------------ Krylov
def test_fgmres_matches_direct_solve_tiny():
    prob = W.disk2d_p1(16, 0)
    H = MG.Hierarchy(prob)
    A, b = H.finest.A, H.finest.disc.rhs()
    x, info = K.fgmres(lambda v: A @ v, H.vcycle, b, tol=1e-12, m=30, max_it=400)
    xd = np.linalg.solve(A.toarray(), b)
    assert info.converged and info.true_rel_residual <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_unpreconditioned_gmres_terminates_in_n_steps():
    """Full GMRES (m >= N) reaches the exact solution in at most N steps (Krylov dimension)."""
    rng = np.random.default_rng(2)
    N = 12
    A = rng.normal(size=(N, N)) + N * np.eye(N)
    b = rng.normal(size=N)
    x, info = K.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-13, m=N, max_it=N)
    assert info.iterations <= N
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)
    # with m = 3 it restarts, and still converges
    x, info = K.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-10, m=3, max_it=500)
    assert info.converged and info.restarts > 1


# ------------------------------------------------------------------ learned boundary correction
def test_mlp_gradients_match_central_differences():
    """Backward pass of the FP64 MLP against central finite differences of its loss."""
    from oracle import learned as LR
    rng = np.random.default_rng(0)
    net = LR.MLP(7, 5, 3, seed=1)
    for prm in net.params():
        prm += 0.05 * rng.normal(size=prm.shape)      # nonzero biases, no ties at ReLU kinks
    X, T = rng.normal(size=(11, 7)), rng.normal(size=(11, 3))
    grads = net.backward(net.forward(X), T)
    for prm, g in zip(net.params(), grads):
        flat = prm.reshape(-1)
        for k in range(flat.size):
            old = flat[k]
            flat[k] = old + 1e-6
            lp = net.loss(net.forward(X), T)
            flat[k] = old - 1e-6
            lm = net.loss(net.forward(X), T)
            flat[k] = old
            fd = (lp - lm) / 2e-6
            assert abs(fd - g.reshape(-1)[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g.reshape(-1)[k])


def test_mlp_forward_closed_form():
    """Identity-like weights: y = relu(relu(x)) = relu(x) for a square network with zero biases."""
    from oracle import learned as LR
    net = LR.MLP(4, 4, 4)
    net.W1, net.W2, net.W3 = np.eye(4), np.eye(4), np.eye(4)
    x = np.array([[1.0, -2.0, 3.0, -0.5]])
    assert np.array_equal(net.forward(x), np.array([[1.0, 0.0, 3.0, 0.0]]))


def test_adam_first_step_is_sign_step():
    """Adam's bias-corrected first step moves every parameter by lr in the direction -sign(g)."""
    from oracle import learned as LR
    p = [np.array([1.0, -1.0, 0.5])]
    g = [np.array([3.0, -0.2, 1e-3])]
    LR.adam_step(p, g, {}, lr=0.01, eps=1e-12)
    assert np.allclose(p[0], [0.99, -0.99, 0.49], atol=1e-9)


def test_learned_features_layout():
    """Patch residual normalised to unit norm; shift and mask entries only on surrogate faces."""
    from oracle import learned as LR
    prob = W.star2d_p2(16, 1).replace(p=3)
    lev = MG.Level(prob, 16, 3)
    r = W.random_vector(lev.N, 5)
    cells = lev.geom.boundary_cells()[:10]
    X, s = LR.features(lev, r, cells)
    nb, dim, nq = lev.nb, 2, 4
    assert X.shape == (10, LR.feature_size(2, 3)) == (10, 9 * 16 + 4 * 4 * 2 + 1 + 4)
    for row, a in enumerate(cells):
        assert abs(np.linalg.norm(X[row, :9 * nb]) - 1.0) < 1e-12
        assert np.allclose(X[row, 4 * nb:5 * nb] * s[row], r[a * nb:(a + 1) * nb])     # centre cell
        mask = X[row, -4:]
        d = X[row, 9 * nb:9 * nb + 4 * nq * dim].reshape(4, nq, dim)
        slots = {2 * dr + sd for (aa, dr, sd) in lev.geom.faces if aa == a}
        assert set(np.nonzero(mask)[0]) == slots
        for slot in range(4):
            assert (np.abs(d[slot]).max() > 0) == (slot in slots)


def _vcycle_matrix(H):
    """The V-cycle as a matrix, by brute force: column j is V(e_j) (V is linear, Sec. 3)."""
    N = H.finest.N
    M = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        M[:, j] = H.vcycle(e)
    return M


@pytest.mark.parametrize("prob", [W.disk2d_p1(8, 1).replace(coarsest_n=4), W.sphere3d(8, 1, 2).replace(coarsest_n=4)],
                         ids=["disk2d", "sphere3d"])
def test_training_pairs_follow_the_error_propagation(prob):
    """The learned part's training pairs: after k steps of u <- u + V(-A u) on A u = 0 the iterate is
    (I - V A)^k u0 (error propagation of a stationary iteration with a linear preconditioner), so
    the k-th block of rows must hold targets -u_K / (s_K h^(2-d)) of that iterate and residual
    features of -A u.  Checked against the explicit matrix power on a tiny mesh; a sign, a stale iterate or
    the correction z alone in place of u + z fails it."""
    from oracle import learned as OL
    H = MG.Hierarchy(prob)
    F = H.finest
    assert len(H.levels) == 2
    cells = OL.boundary_cells(F)
    dim = prob.dim
    nb = F.nb
    rng = np.random.default_rng(3)
    u0s = [2.0 * rng.random(F.N) - 1.0 for _ in range(2)]
    X, T = OL.training_pairs(H, 2, 3, 0, u0s=u0s)
    nc = len(cells)
    assert X.shape == (2 * 3 * nc, OL.feature_size(dim, 1)) and T.shape == (2 * 3 * nc, nb)
    E = np.eye(F.N) - _vcycle_matrix(H) @ F.A.toarray()
    row = 0
    for u0 in u0s:
        u = u0.copy()
        for _ in range(3):
            u = E @ u
            Xo, so = OL.features(F, -(F.A @ u), cells)
            To = np.stack([-u[a * nb:(a + 1) * nb] for a in cells]) / so[:, None] / F.geom.h ** (2 - F.prob.dim)
            assert np.allclose(X[row:row + nc], Xo, rtol=1e-9, atol=1e-12)
            assert np.allclose(T[row:row + nc], To, rtol=1e-9, atol=1e-12)
            row += nc
    # the centre block of the patch (offset 0, the middle of the 3^d blocks) times s is -(A u)_K
    _, so = OL.features(F, -(F.A @ u), cells)
    r = -(F.A @ u)
    c = (3 ** dim) // 2
    assert np.allclose(X[-nc:, c * nb:(c + 1) * nb] * so[:, None], np.stack([r[a * nb:(a + 1) * nb] for a in cells]),
                       rtol=1e-9, atol=1e-12)

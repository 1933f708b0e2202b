"""Element-by-element parity at the benchmark's full sizes, in the launch configuration the
benchmark times (FP32 V-cycle defaults: thread-per-cell kernels, colour-group smoother launches,
the one-CTA tail for the small p = 1 levels, the staged Gram-Schmidt sweeps).

* 2D star, p = 2, 512^2 background cells (910,035 DoF, 8 levels): the oracle hierarchy is
  assembled in full, so every level's operator, both smoother sweep directions and one V-cycle
  are compared on every entry; the Gram-Schmidt sweeps are compared with NumPy at the widths the
  solve reaches; the FP64 FGMRES solve must take the oracle's iteration count.
* 3D ellipsoid, p = 3, 48^3 background cells (~0.8 M DoF): too large to assemble in the oracle,
  so the operator and one smoother sweep are compared on sampled cells whose oracle rows are built
  cell by cell (`Discretisation(assemble=False)`), the smoother with the neighbours' values the
  sweep itself used fed into the oracle's cell update (Eq. 16).

Tolerances are the ones of tests/test_gpu_parity.py: FP64 operator 1e-12 relative; FP32 operator
2e-6 |A||x|; FP32 smoother 2e-4 relative (inputs rounded to FP32 and block inverses amplified by
cond(A_KK)); FP64 smoother sweep (d+1) 2 n_p eps cond(A_KK) over the whole level (`sweep_tol`),
n_p eps cond(A_KK) for a single cell update (floor 1e-12); FP32 V-cycle 1e-4 relative L2; FP64
FGMRES equal iteration counts and 1e-10 relative L2.
"""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from _pairs import Pair  # noqa: E402


def rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def block_tol(levels):
    kap = max(np.linalg.cond(lev.disc.diag).max() for lev in levels)
    nb = max(lev.nb for lev in levels)
    return max(1e-12, nb * 2.2e-16 * kap)


def sweep_tol(lev):
    """FP64 bound of one colour sweep (Eq. 16) over the d + 1 colour groups: each group forms the
    residual of its cells and applies the block inverses (rounding ~ 2 n_p eps cond(A_KK), the
    interior cells by fast diagonalisation on the GPU and by LU on the oracle side), and passes its
    error on to the later groups through the couplings A_KN; at full size the largest block
    condition number (about 2.4e4 at 512^2 p = 2) is met in some cell of every group."""
    kap = np.linalg.cond(lev.disc.diag).max()
    return max(1e-12, (lev.prob.dim + 1) * 2 * lev.nb * 2.2e-16 * kap)


@pytest.fixture(scope="module")
def star512():
    return Pair(W.star2d_p2(512, 0), "f32")


def test_star512_apply_every_level(star512):
    """a1 on all 8 levels of the benchmark hierarchy: FP64 and FP32 operators against A x."""
    P = star512
    for l, lev in enumerate(P.H.levels):
        x = W.random_vector(lev.N, 31 + l)
        yo = lev.A @ x
        y64 = P.to_oracle(P.gpu.apply(P.to_gpu(x, l), level=l), l)
        assert rel_max(y64, yo) <= 1e-12, (l, rel_max(y64, yo))
        y32 = P.to_oracle(P.gpu.apply(P.to_gpu(x, l, torch.float32), level=l), l)
        scale = np.abs(abs(lev.A) @ np.abs(x)).max()
        assert np.abs(y32 - yo).max() <= 2e-6 * scale, (l, np.abs(y32 - yo).max() / scale)


def test_star512_smoother_sweeps(star512):
    """a2 on every level above the coarsest: one forward and one reverse colour sweep, FP32 (the
    V-cycle's precision, thread-per-cell colour-group launches) and FP64."""
    P = star512
    for l in range(1, len(P.H.levels)):
        lev = P.H.levels[l]
        f, u0 = W.random_vector(lev.N, 40 + l), W.random_vector(lev.N, 50 + l)
        for reverse in (False, True):
            uo = lev.coloured_sweep(u0.copy(), f, reverse=reverse)
            u32 = P.gpu.smooth(P.to_gpu(f, l, torch.float32), P.to_gpu(u0, l, torch.float32), level=l,
                               reverse=reverse)
            err32 = rel_max(P.to_oracle(u32, l), uo)
            assert err32 <= 2e-4, (l, reverse, err32)
            u64 = P.gpu.smooth(P.to_gpu(f, l), P.to_gpu(u0, l), level=l, reverse=reverse)
            err64 = rel_max(P.to_oracle(u64, l), uo)
            assert err64 <= sweep_tol(lev), (l, reverse, err64, sweep_tol(lev))


def test_star512_staged_kernels(star512):
    """The staged thread-per-cell operator and smoother at the benchmark size, forced on every
    level: operator on every level and both sweep directions above the coarsest, FP32 bounds."""
    import paper_2506_12899_gb300 as S
    P = star512
    g = S.Solver(P.prob, "f32", staged_min_cells=1)
    for l, lev in enumerate(P.H.levels):
        x = W.random_vector(lev.N, 131 + l)
        yo = lev.A @ x
        scale = np.abs(abs(lev.A) @ np.abs(x)).max()
        y32 = P.to_oracle(g.apply(P.to_gpu(x, l, torch.float32), level=l), l)
        assert np.abs(y32 - yo).max() <= 2e-6 * scale, (l, np.abs(y32 - yo).max() / scale)
        if l == 0:
            continue
        f, u0 = W.random_vector(lev.N, 140 + l), W.random_vector(lev.N, 150 + l)
        for reverse in (False, True):
            uo = lev.coloured_sweep(u0.copy(), f, reverse=reverse)
            u32 = g.smooth(P.to_gpu(f, l, torch.float32), P.to_gpu(u0, l, torch.float32), level=l, reverse=reverse)
            assert rel_max(P.to_oracle(u32, l), uo) <= 2e-4, (l, reverse, rel_max(P.to_oracle(u32, l), uo))
    g.close()


def test_star512_vcycle(star512):
    """One V-cycle of the benchmark hierarchy (512^2 p=2 -> p=1 -> ... -> 64^2, then the one-CTA
    tail over 64^2 .. 8^2 and the coarse solve) in FP32, and the FP64 V-cycle with one launch per
    phase, against the oracle's V-cycle."""
    P = star512
    L = len(P.H.levels) - 1
    r = W.random_vector(P.H.finest.N, 61)
    zo = P.H.vcycle(r)
    z32 = P.to_oracle(P.gpu.vcycle(P.to_gpu(r, L, torch.float32)), L)
    assert np.linalg.norm(z32 - zo) <= 1e-4 * np.linalg.norm(zo), np.linalg.norm(z32 - zo) / np.linalg.norm(zo)
    z64 = P.to_oracle(P.gpu.vcycle(P.to_gpu(r, L)), L)
    tol = block_tol(P.H.levels[1:])
    assert np.linalg.norm(z64 - zo) <= tol * np.linalg.norm(zo), (np.linalg.norm(z64 - zo) / np.linalg.norm(zo), tol)


@pytest.mark.parametrize("variant", [0, 1, 2], ids=["df_basis_w64", "df_basis_wdf", "fp64_basis"])
@pytest.mark.parametrize("nv", [1, 14, 25, 27, 28, 30])
def test_star512_gram_schmidt_sweeps(star512, nv, variant):
    """a6: the three Gram-Schmidt sweeps of an Arnoldi step at N = 910,035 and the widths the
    benchmark solve reaches (staged shapes: E = 512, S = 2 up to width 25; w read directly at
    27-28; E = 256 at 30), against NumPy FP64 CGS2 on an orthonormal V.  Bound: the double-float
    sweeps round V and every operation to about 2^-48 relative; 2^-40 of the magnitudes involved
    leaves 2^8 for the accumulation depth (each thread sums ~12 entries, then tree reductions)."""
    P = star512
    N = P.H.finest.N
    rng = np.random.default_rng(1000 * nv + variant)
    Q, _ = np.linalg.qr(rng.normal(size=(N, nv)))
    V = np.ascontiguousarray(Q.T)
    w = rng.normal(size=N)
    h1, h2, w2, nrm = P.gpu.gram_schmidt(torch.tensor(V, device="cuda"), torch.tensor(w, device="cuda"), variant)
    h1, h2, w2 = h1.cpu().numpy(), h2.cpu().numpy(), w2.cpu().numpy()
    o1 = V @ w
    w1 = w - V.T @ o1
    o2 = V @ w1
    ow2 = w1 - V.T @ o2
    u = 2.0 ** -40
    bh = u * (np.abs(V) @ np.abs(w))
    assert np.all(np.abs(h1 - o1) <= bh), np.abs(h1 - o1).max()
    assert np.all(np.abs(h2 - o2) <= bh), np.abs(h2 - o2).max()
    bw = u * (np.abs(w) + np.abs(V.T) @ (np.abs(o1) + np.abs(o2))) + np.abs(V.T) @ (2 * bh)
    assert np.all(np.abs(w2 - ow2) <= bw), np.abs(w2 - ow2).max()
    on = np.linalg.norm(ow2)
    assert abs(nrm - on) <= u * np.linalg.norm(np.abs(w)) + np.linalg.norm(bw), (nrm, on)


def test_star512_fgmres_fp64_equal_iterations(star512):
    """a6 end to end at full size: the FP64-V-cycle FGMRES(30) solve takes the oracle's iteration
    count and lands within 1e-10 of its solution; the FP32-V-cycle solve reaches the FP64 true
    residual 1e-8 as recomputed by the oracle, and its distance to the oracle's solution is below
    the residual bound with the operator's condition estimate from the same run."""
    import paper_2506_12899_gb300 as S
    P = star512
    F = P.H.finest
    L = len(P.H.levels) - 1
    bo = F.disc.rhs()
    xo, oi = K.fgmres(lambda v: F.A @ v, P.H.vcycle, bo, tol=1e-8, m=30, max_it=300)
    assert oi.converged
    g64 = S.Solver(P.prob, "f64")
    b = g64.rhs()
    assert rel_max(P.to_oracle(b, L), bo) <= 1e-13
    x = torch.zeros_like(b)
    info = g64.solve(b, x, tol=1e-8, restart=30, max_it=300)
    assert info.converged and info.iterations == oi.iterations, (info.iterations, oi.iterations)
    assert np.linalg.norm(P.to_oracle(x, L) - xo) <= 1e-10 * np.linalg.norm(xo)
    g64.close()
    x32 = torch.zeros_like(b)
    info32 = P.gpu.solve(b, x32, tol=1e-8, restart=30, max_it=300)
    assert info32.converged
    xg = P.to_oracle(x32, L)
    assert np.linalg.norm(bo - F.A @ xg) <= 1.01e-8 * np.linalg.norm(bo)
    # ||x - x_o|| <= ||A^-1|| ||A x - b|| with ||A^-1|| from a few inverse-power steps through
    # the oracle's own FGMRES (a lower bound, hence the factor 10)
    v = W.random_vector(F.N, 7)
    v /= np.linalg.norm(v)
    inv = 0.0
    for _ in range(3):
        y, _i = K.fgmres(lambda q: F.A @ q, P.H.vcycle, v, tol=1e-10, m=30, max_it=300)
        inv = np.linalg.norm(y)
        v = y / inv
    bound = 10 * inv * (np.linalg.norm(bo - F.A @ xg) + np.linalg.norm(bo - F.A @ xo))
    assert np.linalg.norm(xg - xo) <= bound, (np.linalg.norm(xg - xo), bound)


# ------------------------------------------------------------------ 3D p = 3 at 48^3, sampled cells
@pytest.fixture(scope="module")
def ellipsoid48():
    import paper_2506_12899_gb300 as S
    from oracle.dgsbm import Discretisation
    from oracle.geometry import LevelGeometry
    prob = W.ellipsoid3d_p3(48, 0)
    g = S.Solver(prob, "f32")
    geom = LevelGeometry(prob, 48, 3)
    D = Discretisation(prob, geom, assemble=False)
    coords = g.layout()
    lin = coords[:, 0].astype(np.int64) + 48 * coords[:, 1].astype(np.int64) + 48 * 48 * coords[:, 2].astype(np.int64)
    perm = geom.bg2act[lin]
    assert (perm >= 0).all() and len(perm) == geom.n_active
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))                 # oracle cell -> compact cell
    rng = np.random.default_rng(48)
    bcells = np.array(sorted({f[0] for f in geom.faces}))
    sample = np.concatenate([rng.choice(geom.n_active, 300, replace=False), rng.choice(bcells, 100, replace=False)])
    return dict(prob=prob, g=g, geom=geom, D=D, inv=inv, sample=sample)


def test_ellipsoid48_p3_apply_sampled(ellipsoid48):
    """a1 at 3D p = 3, 48^3: FP64 and FP32 operators on 400 sampled cells (100 of them boundary
    cells) against oracle rows built cell by cell."""
    E = ellipsoid48
    g, D, inv, sample = E["g"], E["D"], E["inv"], E["sample"]
    nb = D.nb
    x = W.random_vector(g.n_dof(), 5)
    X = x.reshape(-1, nb)
    yo, ya = [], []
    for a in sample:
        y = D.diag_block(a) @ X[inv[a]]
        s = np.abs(D.diag_block(a)) @ np.abs(X[inv[a]])
        for nbc, B in D.offdiag_blocks(a):
            y = y + B @ X[inv[nbc]]
            s = s + np.abs(B) @ np.abs(X[inv[nbc]])
        yo.append(y)
        ya.append(s)
    yo, ya = np.array(yo), np.array(ya)
    y64 = g.apply(torch.tensor(x, device="cuda")).cpu().numpy().reshape(-1, nb)[inv[sample]]
    assert np.abs(y64 - yo).max() <= 1e-12 * np.abs(yo).max()
    x32 = torch.tensor(x, dtype=torch.float32, device="cuda")
    y32 = g.apply(x32).double().cpu().numpy().reshape(-1, nb)[inv[sample]]
    assert np.abs(y32 - yo).max() <= 2e-6 * ya.max(), np.abs(y32 - yo).max() / ya.max()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ellipsoid48_p3_smoother_sampled(ellipsoid48, dtype):
    """a2 at 3D p = 3, 48^3: one forward colour sweep (omega = 0.8 on p = 3 levels).  For every
    sampled cell K of colour c the oracle recomputes Eq. 16's update
        u_K <- u_K + omega A_KK^-1 (f_K - A_KK u_K - sum_N A_KN u_N)
    with u_N the value the sweep had produced for neighbours of earlier colours (the GPU's output:
    those cells are not touched again in the sweep) and the input value for later colours."""
    E = ellipsoid48
    g, D, geom, inv, sample, prob = E["g"], E["D"], E["geom"], E["inv"], E["sample"], E["prob"]
    nb = D.nb
    dt = torch.float64 if dtype == "f64" else torch.float32
    f = W.random_vector(g.n_dof(), 8)
    u0 = W.random_vector(g.n_dof(), 9)
    f_t, u_t = torch.tensor(f, dtype=dt, device="cuda"), torch.tensor(u0, dtype=dt, device="cuda")
    f_in, u_in = f_t.double().cpu().numpy(), u_t.double().cpu().numpy()      # what the GPU sees
    out = g.smooth(f_t, u_t.clone()).double().cpu().numpy()
    F_, U0, UN = f_in.reshape(-1, nb), u_in.reshape(-1, nb), out.reshape(-1, nb)
    colour = np.sum((geom.cell_idx % 2) << np.arange(3), axis=1)
    omega = prob.omega_p3
    got, exp, tols = [], [], []
    for a in sample:
        AKK = D.diag_block(a)
        t = F_[inv[a]] - AKK @ U0[inv[a]]
        for nbc, B in D.offdiag_blocks(a):
            un = UN[inv[nbc]] if colour[nbc] < colour[a] else U0[inv[nbc]]
            t = t - B @ un
        exp.append(U0[inv[a]] + omega * np.linalg.solve(AKK, t))
        got.append(UN[inv[a]])
        tols.append(np.linalg.cond(AKK))
    got, exp = np.array(got), np.array(exp)
    if dtype == "f64":
        tol = max(1e-12, nb * 2.2e-16 * max(tols))
    else:
        tol = 2e-4
    assert rel_max(got, exp) <= tol, (rel_max(got, exp), tol)

"""Seeded synthetic workloads for the DG-SBM Poisson solver.

This module produces *inputs only*: the problem description (background box, cell
counts, degree, level-set shape parameters drawn from a seed, manufactured
solution kind, penalty constants, multigrid options) and seeded random vectors.
It performs none of the method's arithmetic (no geometry classification, no
quadrature, no operator, no smoother).  Both the CPU oracle and the CUDA path
receive the same `Problem` and evaluate everything else independently.

Shapes (level set phi < 0 inside, Sec. 4.1 of the paper):
  DISK       disk (2D) / sphere (3D):   |x - c| - r
  STAR       2D star:                   |x - c| - r (1 + amp sin(freq theta + phase))
  ELLIPSOID  3D ellipsoid:              |S^-1 R^T (x - c)| - 1,  S = diag(semi)
  BOX        axis-aligned box:          max_k |x_k - c_k| - r   (surrogate == true boundary)
  COMPLEX2D  the deformed 2D domain of Sec. 5.4, Eq. 24:
             (1 - 3/4 sin^2(pi x)) (x^2 + y^2) - 1/5

Manufactured solutions (f = -Laplace(u), g = u on the true boundary):
  SINPROD    prod_k sin(pi x_k)
  EXPCOS     exp(x) cos(2 y)                     (2D)
  LINEAR     0.5 + x - 0.7 y + 0.3 z
  COSSIN     2 cos(x) sin(y)                     (Sec. 5.1, Eq. 23)
  PHIP1      phi(x) + 1 for the COMPLEX2D shape  (Sec. 5.4)
  QUADRATIC  LINEAR + x^2 - 0.5 y^2 + 0.25 x y - 0.4 z^2 + 0.2 y z
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

SHAPE_DISK, SHAPE_STAR, SHAPE_ELLIPSOID, SHAPE_BOX, SHAPE_COMPLEX2D = 0, 1, 2, 3, 4
EXACT_SINPROD, EXACT_EXPCOS, EXACT_LINEAR, EXACT_COSSIN, EXACT_PHIP1, EXACT_QUADRATIC = 0, 1, 2, 3, 4, 5


@dataclass
class Shape:
    kind: int = SHAPE_DISK
    center: tuple = (0.0, 0.0, 0.0)
    radius: float = 0.7
    amp: float = 0.0
    freq: float = 0.0
    phase: float = 0.0
    semi: tuple = (1.0, 1.0, 1.0)
    rot: tuple = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)  # row-major 3x3


@dataclass
class Problem:
    """Everything both sides need to build the discrete problem and its solver."""
    name: str = "custom"
    dim: int = 2
    n: int = 32                      # background cells per direction on the finest level
    p: int = 1                       # polynomial degree on the finest level
    lo: tuple = (-1.0, -1.0, -1.0)
    hi: tuple = (1.0, 1.0, 1.0)
    shape: Shape = field(default_factory=Shape)
    exact: int = EXACT_SINPROD
    lam: float = 0.5                 # volume-fraction threshold lambda
    lam_inclusive: int = 1           # 1: active iff kappa >= lambda; 0: kappa > lambda (Sec. 2.1)
    sigma_face_c: float = 10.0       # sigma_F = c (p_l + 1)^2 / h_l
    sigma_bnd_c: float = 10.0        # sigma_Gamma = c (p_l + 1)^2 / h_l
    alpha: float = 1.0               # 1: quasi-symmetric Nitsche, -1: penalty-free variant
    extension: int = 0               # 0: u(x~) + d.grad u(x~) (Eq. 6); 1: cell polynomial evaluated at x~ + d
    coarsest_n: int = 4              # h-coarsening stops at this many cells per direction
    pre_smooth: int = 1
    post_smooth: int = 1
    ssor_each: int = 0               # 1: every smoothing step is a forward then a reverse (SSOR) sweep
    omega: float = 1.0               # block-smoother relaxation on levels with p_l <= 2
    omega_p3: float = 0.8            # relaxation on levels with p_l = 3 (Sec. 5.3)
    vf_samples: int = 0              # kappa sub-samples per direction (0: 16 in 2D, 8 in 3D)
    smoother: int = 0                # 0: coloured block Gauss-Seidel (multiplicative, Eq. 16); 1: additive
                                     # block Jacobi damped by omega; 2: Chebyshev-accelerated block Jacobi
    ordering: int = 0                # Gauss-Seidel colours: 0 the 2^d colours c = sum (i_k mod 2) 2^k;
                                     # 1 red-black, (sum_k i_k) mod 2
    cheb_degree: int = 4             # Chebyshev steps per smoothing step
    cheb_ratio: float = 20.0         # Chebyshev interval [lambda_max / ratio, lambda_max]

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    @property
    def samples(self) -> int:
        if self.vf_samples > 0:
            return self.vf_samples
        return 16 if self.dim == 2 else 8


def _uniform(seed: int, k: int) -> np.ndarray:
    return np.random.default_rng(seed).random(k)


def rotation_from_angles(a: float, b: float, c: float) -> tuple:
    """R = Rz(a) Ry(b) Rx(c), row-major (an input parameter of the ellipsoid)."""
    ca, sa, cb, sb, cc, sc = math.cos(a), math.sin(a), math.cos(b), math.sin(b), math.cos(c), math.sin(c)
    rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1.0]])
    ry = np.array([[cb, 0, sb], [0, 1.0, 0], [-sb, 0, cb]])
    rx = np.array([[1.0, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return tuple(float(v) for v in (rz @ ry @ rx).reshape(-1))


def disk(dim: int, seed: int, radius: float = 0.7, offset: float = 0.05) -> Shape:
    u = _uniform(seed, 3)
    c = [-offset + 2 * offset * u[k] if k < dim else 0.0 for k in range(3)]
    return Shape(kind=SHAPE_DISK, center=tuple(c), radius=radius)


def star(seed: int, r0: float = 0.7, amp: float = 0.1, freq: int = 5) -> Shape:
    u = _uniform(seed, 1)
    return Shape(kind=SHAPE_STAR, radius=r0, amp=amp, freq=float(freq), phase=2 * math.pi * float(u[0]))


def ellipsoid(seed: int, semi=(0.75, 0.6, 0.5)) -> Shape:
    u = _uniform(seed, 3)
    return Shape(kind=SHAPE_ELLIPSOID, semi=tuple(semi),
                 rot=rotation_from_angles(2 * math.pi * u[0], 2 * math.pi * u[1], 2 * math.pi * u[2]))


def random_star(seed: int) -> Shape:
    u = _uniform(seed, 4)
    return Shape(kind=SHAPE_STAR, radius=0.6 + 0.15 * u[0], amp=0.05 + 0.10 * u[1],
                 freq=float(3 + min(4, int(5 * u[2]))), phase=2 * math.pi * u[3])


def random_ellipsoid(seed: int) -> Shape:
    u = _uniform(seed, 6)
    semi = tuple(0.45 + 0.35 * u[k] for k in range(3))
    return Shape(kind=SHAPE_ELLIPSOID, semi=semi,
                 rot=rotation_from_angles(2 * math.pi * u[3], 2 * math.pi * u[4], 2 * math.pi * u[5]))


def box(half: float = 0.5) -> Shape:
    return Shape(kind=SHAPE_BOX, radius=half)


def complex2d() -> Shape:
    return Shape(kind=SHAPE_COMPLEX2D)


# --------------------------------------------------------------------------- named workloads
def disk2d_p1(n: int = 32, seed: int = 0) -> Problem:
    """2D plain FP64 workload: 32^2 Q1 cells, disk r=0.7 with seeded centre offset."""
    return Problem(name=f"disk2d_p1_n{n}", dim=2, n=n, p=1, shape=disk(2, seed),
                   exact=EXACT_SINPROD, coarsest_n=4)


# The p >= 2 and 3D workloads use lambda = 0.75 (kappa >= 0.75), a minimal interior penalty
# sigma_F = (p+1)^2 / h and the boundary penalty sigma_Gamma = 10 (p+1)^2 / h.  With the 2D
# workload's lambda = 0.5 and sigma_F = 10 (p+1)^2 / h, about 40% of the boundary-cell blocks
# are indefinite at p = 2 and the cell-wise smoother diverges.
HIGH_ORDER = dict(lam=0.75, sigma_face_c=1.0, sigma_bnd_c=10.0)


def star2d_p2(n: int = 512, seed: int = 0) -> Problem:
    """2D p=2 workload: 512^2 cells, star r(theta)=0.7(1+0.1 sin(5 theta+phi)), phi seeded."""
    return Problem(name=f"star2d_p2_n{n}", dim=2, n=n, p=2, shape=star(seed),
                   exact=EXACT_EXPCOS, coarsest_n=8 if n >= 64 else 4, **HIGH_ORDER)


# In 3D at p >= 2 the first-order Taylor extension u(x~) + d.grad u(x~) gives a V-cycle that does
# not converge (sphere p=2: 59 FGMRES iterations at 16^3, stagnation from 32^3; ellipsoid p=3:
# stagnation from 24^3; oracle and GPU agree), so those workloads take the full-order extension,
# the cell polynomial evaluated at x~ + d (20 iterations at 64^3 p=2, 19 at 48^3 p=3).
def sphere3d(n: int = 64, p: int = 1, seed: int = 0) -> Problem:
    """3D p=1 / p=2 workload: 64^3 cells, sphere r=0.7 with seeded centre offset (full-order
    boundary extension at p >= 2)."""
    return Problem(name=f"sphere3d_p{p}_n{n}", dim=3, n=n, p=p, shape=disk(3, seed),
                   exact=EXACT_SINPROD, coarsest_n=4, extension=1 if p >= 2 else 0, **HIGH_ORDER)


def ellipsoid3d_p3(n: int = 96, seed: int = 0, smooth: int = 2) -> Problem:
    """3D p=3 workload: 96^3 cells, ellipsoid (0.75,0.6,0.5) rotated by seeded angles (full-order
    boundary extension).  Two pre- and two post-smoothing steps: with one of each the FGMRES
    residual stalls near 5e-5 at 96^3 (measured; the paper reports the same weakness of its
    smoother for p = 3 in 3D); with two it converges in 29 iterations."""
    return Problem(name=f"ellipsoid3d_p3_n{n}", dim=3, n=n, p=3, shape=ellipsoid(seed),
                   exact=EXACT_SINPROD, coarsest_n=6 if n % 6 == 0 else 4, extension=1,
                   pre_smooth=smooth, post_smooth=smooth, **HIGH_ORDER)


def random_star2d_p3(n: int = 128, seed: int = 1000) -> Problem:
    """Learned-correction family (2D): a seeded random star on 128^2 Q3 cells.  Training domains
    use seeds 1000..1255, held-out domains 2000..2031."""
    return Problem(name=f"random_star2d_p3_n{n}_s{seed}", dim=2, n=n, p=3, shape=random_star(seed),
                   exact=EXACT_EXPCOS, coarsest_n=8 if n >= 64 else 4, extension=1, **HIGH_ORDER)


def random_ellipsoid3d_p3(n: int = 32, seed: int = 1000) -> Problem:
    """Learned-correction family (3D): a seeded random ellipsoid on 32^3 Q3 cells."""
    return Problem(name=f"random_ellipsoid3d_p3_n{n}_s{seed}", dim=3, n=n, p=3, shape=random_ellipsoid(seed),
                   exact=EXACT_SINPROD, coarsest_n=4, extension=1, **HIGH_ORDER)


def paper_disk(level: int, p: int, lam: float, dim: int = 2) -> Problem:
    """Paper-replica unit disk/sphere (Sec. 5): box [-1.01,1.01]^d, 4*2^level cells per direction,
    sigma_Gamma = 5, sigma_F = 1 (scaled by (p+1)^2/h), kappa > lambda (kappa = 1 for lambda = 1),
    u = 2 cos x sin y, boundary extension by the cell polynomial evaluated at x~ + d."""
    return Problem(name=f"paper_disk{dim}d_p{p}_l{level}_lam{lam}", dim=dim, n=4 * 2 ** level, p=p,
                   lo=(-1.01,) * 3, hi=(1.01,) * 3, shape=Shape(kind=SHAPE_DISK, radius=1.0),
                   exact=EXACT_COSSIN, lam=lam, lam_inclusive=1 if lam >= 1.0 else 0, sigma_face_c=1.0, sigma_bnd_c=5.0,
                   extension=1, coarsest_n=4)


def paper_complex2d(level: int, p: int, lam: float) -> Problem:
    """The paper's complex deformed 2D domain (Sec. 5.4): phi = (1 - 3/4 sin^2(pi x))(x^2 + y^2) - 1/5,
    u = phi + 1 (g = 1 on the true boundary), background [-1.01,1.01]^2 with 4*2^level cells per
    direction, the paper-replica penalties and activity test of paper_disk, polynomial extension."""
    return Problem(name=f"paper_complex2d_p{p}_l{level}_lam{lam}", dim=2, n=4 * 2 ** level, p=p,
                   lo=(-1.01,) * 3, hi=(1.01,) * 3, shape=complex2d(), exact=EXACT_PHIP1, lam=lam,
                   lam_inclusive=1 if lam >= 1.0 else 0, sigma_face_c=1.0, sigma_bnd_c=5.0, extension=1,
                   coarsest_n=4)


def random_vector(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded U[-1,1] vector (used as an apply / smoother / V-cycle input)."""
    return (2.0 * np.random.default_rng(seed).random(n) - 1.0).astype(dtype)

"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the factorization itself: it only makes
points and right-hand sides.  Every random number comes from one
counter-based generator, SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so that any other
implementation can reproduce the same stream from its published definition:

    state_i = seed + (i + 1) * 0x9E3779B97F4A7C15          (mod 2^64)
    z = state_i
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out_i = z ^ (z >> 31)

Uniforms are the top 53 bits scaled by 2^-53 (in [0, 1)); normals use the
Box-Muller transform on consecutive pairs of uniforms.

Workloads (all synthetic, shaped like the numerical examples of Sec. 4):

* 2D unit square, piecewise-constant collocation on a uniform grid
  (Example 1): points at the cell centres ((i+1/2)h, (j+1/2)h), h = 1/n.
* 3D unit cube on a uniform grid (Example 2), same rule in 3D.
* iid uniform random points in the unit square (the batched workload).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First ``n`` outputs of SplitMix64 started at ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """``n`` uniforms in [0, 1): top 53 bits of SplitMix64 times 2^-53."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """``n`` standard normals by Box-Muller on uniforms (u1, u2) of the stream.

    Pair p uses uniforms 2p and 2p+1; u1 is mapped to (0, 1] as 1 - u.
    Both outputs of a pair are used (cos first, then sin).
    """
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:n]


def grid_points(n_side: int, dim: int) -> np.ndarray:
    """Cell centres of a uniform ``n_side``^dim grid on [0,1]^dim, point-major.

    Ordering: x fastest, then y, then z.  Shape (n_side**dim, dim).
    """
    h = 1.0 / n_side
    c = (np.arange(n_side) + 0.5) * h
    mesh = np.meshgrid(*([c] * dim), indexing="ij")
    # mesh[0] varies along axis 0; we want x fastest -> reverse axes
    pts = np.stack([m.transpose(tuple(reversed(range(dim)))).reshape(-1) for m in mesh], axis=1)
    return np.ascontiguousarray(pts)


def random_points(seed: int, n: int, dim: int) -> np.ndarray:
    """``n`` iid uniform points in [0,1)^dim; coordinate d of point i is
    uniform number i*dim + d of the stream.  Shape (n, dim)."""
    return uniform(seed, n * dim).reshape(n, dim)


def rhs(seed: int, n: int, nrhs: int = 1) -> np.ndarray:
    """Seeded N(0,1) right-hand sides, column-major n x nrhs (returned as an
    (nrhs, n) array: column c is ``normal(seed + c, n)``)."""
    return np.stack([normal(seed + c, n) for c in range(nrhs)], axis=0)


# ---------------------------------------------------------------------------
# Workload recipes.  kernel kind 0: K(z) = -log|z| / (2 pi) (2D Laplace);
# kind 1: K(z) = 1 / (4 pi |z|) (3D Laplace).  Matrix A = diag * I + w * K
# with K_ii := 0 (second-kind form), w = 1/N.
# ---------------------------------------------------------------------------

def cell_self_integral(kind: int, h: float) -> float:
    """Diagonal entry of the first-kind discretisations of Sec. 4 (Examples
    1 and 2): piecewise-constant collocation on a grid of side h gives
    K_ij = h^d K(x_i - x_j) off the diagonal and K_ii = the integral of K
    over the cell [-h/2, h/2]^d around the collocation point.  Closed forms
    (a = h/2), by scaling the integral over the unit square / cube:
      2D, K = -log|z| / (2 pi):
        int_[0,1]^2 log(x^2 + y^2) = log 2 + pi/2 - 3, so
        int_[-a,a]^2 log|z| = 2 a^2 (2 log a + log 2 + pi/2 - 3);
      3D, K = 1 / (4 pi |z|):
        int_[0,1]^3 1/|z| = (3/2) log((sqrt 3 + 1)/(sqrt 3 - 1)) - pi/4, so
        int_[-a,a]^3 1/|z| = 8 a^2 times that.
    The paper approximates these integrals adaptively; the closed forms are
    the values that quadrature converges to."""
    a = 0.5 * h
    if kind == 0:
        return -(2.0 * a * a * (2.0 * math.log(a) + math.log(2.0) + 0.5 * math.pi - 3.0)) / (2.0 * math.pi)
    if kind == 1:
        c = 1.5 * math.log((math.sqrt(3.0) + 1.0) / (math.sqrt(3.0) - 1.0)) - 0.25 * math.pi
        return 8.0 * a * a * c / (4.0 * math.pi)
    raise ValueError(kind)


def workload(name: str) -> dict:
    """Named synthetic workloads.  Returns a dict with points, kernel, eps,
    leaf size, rhs seeds.  Points are float64, shape (n, dim)."""
    if name == "laplace2d_grid64":            # 64x64 grid, N = 4096
        pts = grid_points(64, 2)
        return dict(name=name, pts=pts, dim=2, kind=0, eps=1e-6, leaf=64, rhs_seeds=[1])
    if name == "laplace2d_grid64_first_kind":  # Example 1 as in the paper: first kind, N = 4096
        pts = grid_points(64, 2)
        h = 1.0 / 64
        return dict(name=name, pts=pts, dim=2, kind=0, eps=1e-6, leaf=64, rhs_seeds=[1],
                    diag=cell_self_integral(0, h), weight=h * h)
    if name == "laplace3d_grid16_first_kind":  # Example 2 as in the paper: first kind, N = 4096
        pts = grid_points(16, 3)
        h = 1.0 / 16
        return dict(name=name, pts=pts, dim=3, kind=1, eps=1e-3, leaf=64, rhs_seeds=[1],
                    diag=cell_self_integral(1, h), weight=h ** 3)
    if name == "laplace2d_grid256":           # 256x256 grid, N = 65536 (profiling size)
        pts = grid_points(256, 2)
        return dict(name=name, pts=pts, dim=2, kind=0, eps=1e-6, leaf=64, rhs_seeds=[1, 2, 3, 4])
    if name == "laplace2d_grid512":           # 512x512 grid, N = 262144
        pts = grid_points(512, 2)
        return dict(name=name, pts=pts, dim=2, kind=0, eps=1e-6, leaf=64, rhs_seeds=[1, 2, 3, 4])
    if name == "laplace3d_grid32":            # 32^3 grid, N = 32768
        pts = grid_points(32, 3)
        return dict(name=name, pts=pts, dim=3, kind=1, eps=1e-3, leaf=64, rhs_seeds=[1])
    if name == "laplace3d_grid64":            # 64^3 grid, N = 262144
        pts = grid_points(64, 3)
        return dict(name=name, pts=pts, dim=3, kind=1, eps=1e-6, leaf=64, rhs_seeds=[1])
    raise KeyError(name)


def batched_sizes(nprob: int = 256) -> np.ndarray:
    """Problem sizes of the batched 2D workload: N_p = 1024 + floor(u * 15361),
    u uniform number p of the stream seeded 1000 + p (first draw)."""
    return np.array([1024 + int(uniform(1000 + p, 1)[0] * 15361) for p in range(nprob)],
                    dtype=np.int64)


def batched_problem(p: int, n: int) -> np.ndarray:
    """Points of problem p of the batched workload: iid uniform in the unit
    square from the stream seeded 1000 + p, skipping the first draw (used for
    the size)."""
    u = uniform(1000 + p, 1 + 2 * n)[1:]
    return u.reshape(n, 2)

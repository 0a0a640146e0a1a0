"""Seeded synthetic workloads for the finite cell Stokes smoother.

This module only draws numbers: background grids, obstacle lists and random
vectors.  It holds none of the method's arithmetic, so both the CUDA library
tests and the CPU oracle tests can use it.

The paper's experiments use a 2D channel with a cylindrical obstacle
(Sec. 4, eq. cf_inflow).  The workloads here stand in for it and for the
porous-medium style 3D problems with seeded obstacles:

* ``channel_2d``  -- unit square, one circular hole, parabolic inflow at x=0,
  no-slip walls at y=0,1, do-nothing outflow at x=1, body force
  (sin(pi x), cos(pi y)).
* ``porous_3d``   -- unit cube, non-overlapping spheres, no-slip on the y and
  z faces, do-nothing x faces, unit body force in x.
* ``batch_2d``    -- uneven 2D problems with 1..8 rotated elliptical holes.

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014): state +=
0x9E3779B97F4A7C15, then the two xor-shift-multiply rounds; a uniform double
is (z >> 11) * 2^-53.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


class SplitMix64:
    """Scalar SplitMix64 stream."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * _M1) & _MASK
        z = ((z ^ (z >> 27)) * _M2) & _MASK
        return z ^ (z >> 31)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return a + (b - a) * u

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1)) if hi > lo else lo


def uniform_array(n: int, seed: int, a: float = -1.0, b: float = 1.0) -> np.ndarray:
    """n uniform doubles in [a, b): element i is SplitMix64 output i+1 of seed."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + i * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return a + (b - a) * u


# Obstacle record: [type, cx, cy, cz, r0, r1, r2, cos(theta), sin(theta)]
#   type 0: circle (2D) or sphere (3D) with radius r0
#   type 1: ellipse (2D) with semi-axes r0 (along the rotated x axis) and r1
SHAPE_FIELDS = 9


@dataclasses.dataclass
class Problem:
    """One finite cell Stokes problem on a uniform background grid."""

    name: str
    dim: int
    n: Tuple[int, ...]               # cells per direction on the finest level
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    shapes: np.ndarray               # [nshape, 9]
    alpha: float                     # fictitious-domain scaling
    qdepth: int                      # cut-cell quadrature depth
    nlevels: int                     # multigrid levels L
    eta: float = 1e-3                # viscosity
    beta: float = 100.0              # Nitsche lambda = beta * eta / h_min
    omega: float = 0.8               # smoother damping
    nu_pre: int = 2
    nu_post: int = 2
    preset: int = 0                  # 0 channel, 1 porous, 2 no strong data
    force_kind: int = 0
    force: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    ubar: float = 0.3                # inflow mean (channel preset)
    rtol: float = 1e-8
    restart: int = 30
    amr_uniform: int = -1            # >= 0: adaptive quadtree (2D) or octree (3D), cells refined uniformly
                                     # to this level and cut cells to the finest (n = lattice of the finest level)

    def level_n(self, level: int) -> Tuple[int, ...]:
        """Cells per direction on level ``level`` (1 = coarsest, L = finest)."""
        f = 2 ** (self.nlevels - level)
        return tuple(k // f for k in self.n)

    def ndof(self, level: int | None = None) -> int:
        n = self.level_n(self.nlevels if level is None else level)
        nodes = 1
        for k in n:
            nodes *= k + 1
        return nodes * (self.dim + 1)


def _spheres(rng: SplitMix64, count: int, rmin: float, rmax: float, dim: int,
             max_tries: int = 200000) -> np.ndarray:
    """Non-overlapping balls inside the unit box by rejection sampling.

    Draw order per attempt: radius, then centre coordinates x, y(, z)."""
    out: List[List[float]] = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("sphere packing did not finish; lower the volume fraction")
        r = rng.uniform(rmin, rmax)
        c = [rng.uniform(r, 1.0 - r) for _ in range(dim)]
        ok = True
        for s in out:
            d2 = sum((c[k] - s[1 + k]) ** 2 for k in range(dim))
            if d2 < (r + s[4]) ** 2:
                ok = False
                break
        if ok:
            cc = c + [0.0] * (3 - dim)
            out.append([0.0, cc[0], cc[1], cc[2], r, r, r, 1.0, 0.0])
    return np.array(out, dtype=np.float64).reshape(-1, SHAPE_FIELDS)


def radius_scale(count: int, target_fraction: float = 0.30, rmin: float = 0.04,
                 rmax: float = 0.12) -> float:
    """Scale for U[rmin, rmax] radii so the expected solid fraction of ``count``
    balls stays at ``target_fraction`` (random sequential packing jams near
    0.38, so larger fractions cannot be drawn)."""
    e_r3 = (rmax ** 4 - rmin ** 4) / (4.0 * (rmax - rmin))
    frac = count * (4.0 / 3.0) * math.pi * e_r3
    return min(1.0, (target_fraction / frac) ** (1.0 / 3.0))


def channel_2d(seed: int = 0, n: int = 32, nlevels: int = 3, alpha: float = 1e-8,
               qdepth: int = 4, radius: float = 0.2) -> Problem:
    """2D channel on the unit square with one circular hole (centre drawn in
    [0.35, 0.65]^2), parabolic inflow, alpha = 1e-8, quadtree depth 4."""
    rng = SplitMix64(seed)
    cx, cy = rng.uniform(0.35, 0.65), rng.uniform(0.35, 0.65)
    shapes = np.array([[0.0, cx, cy, 0.0, radius, radius, radius, 1.0, 0.0]])
    return Problem(name=f"channel2d_n{n}_s{seed}", dim=2, n=(n, n), lo=(0.0, 0.0), hi=(1.0, 1.0),
                   shapes=shapes, alpha=alpha, qdepth=qdepth, nlevels=nlevels, preset=0,
                   force_kind=1, force=(1.0, 1.0, 0.0))


def channel_3d(seed: int = 0, n: int = 16, nlevels: int = 3, alpha: float = 1e-8,
               qdepth: int = 3, radius: float = 0.2) -> Problem:
    """3D duct on the unit cube with one spherical obstacle (centre drawn in
    [0.35, 0.65]^3), inflow at x = 0 with the product of the parabolas in y
    and z, no-slip on the y and z faces, a unit body force in x."""
    rng = SplitMix64(seed)
    c = [rng.uniform(0.35, 0.65) for _ in range(3)]
    shapes = np.array([[0.0, c[0], c[1], c[2], radius, radius, radius, 1.0, 0.0]])
    return Problem(name=f"channel3d_n{n}_s{seed}", dim=3, n=(n, n, n), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                   shapes=shapes, alpha=alpha, qdepth=qdepth, nlevels=nlevels, preset=0, force_kind=0,
                   force=(1.0, 0.0, 0.0))


def porous_3d(seed: int = 0, n: int = 64, nspheres: int = 40, nlevels: int = 5,
              alpha: float = 1e-8, qdepth: int = 3, scale: float | None = None) -> Problem:
    """3D porous medium: ``nspheres`` non-overlapping spheres with radii
    U[0.04, 0.12] (scaled to keep a drawable volume fraction), no-slip on the
    y/z faces and on the spheres, unit body force in x."""
    rng = SplitMix64(seed)
    s = radius_scale(nspheres) if scale is None else scale
    shapes = _spheres(rng, nspheres, 0.04 * s, 0.12 * s, 3)
    return Problem(name=f"porous3d_n{n}_k{nspheres}_s{seed}", dim=3, n=(n, n, n),
                   lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), shapes=shapes, alpha=alpha,
                   qdepth=qdepth, nlevels=nlevels, preset=1, force_kind=0,
                   force=(1.0, 0.0, 0.0))


def ellipses_2d(rng: SplitMix64, count: int) -> np.ndarray:
    """``count`` rotated ellipses, centres U[0.25, 0.75]^2 (overlap allowed),
    semi-axes U[0.03, 0.2], angle U[0, pi).  Draw order: cx, cy, a, b, angle."""
    rows = []
    for _ in range(count):
        cx, cy = rng.uniform(0.25, 0.75), rng.uniform(0.25, 0.75)
        a, b = rng.uniform(0.03, 0.2), rng.uniform(0.03, 0.2)
        th = rng.uniform(0.0, math.pi)
        rows.append([1.0, cx, cy, 0.0, a, b, 0.0, math.cos(th), math.sin(th)])
    return np.array(rows, dtype=np.float64).reshape(-1, SHAPE_FIELDS)


def batch_2d(seed: int, sizes=(16, 32, 64, 128), alphas=(1e-6, 1e-8, 1e-10)) -> Problem:
    """One problem of the uneven 2D batch: grid n from ``sizes``, 1..8
    ellipses, alpha from ``alphas``; channel boundary conditions."""
    rng = SplitMix64(0x5EED0000 + seed)
    n = sizes[rng.randint(0, len(sizes) - 1)]
    count = rng.randint(1, 8)
    alpha = alphas[rng.randint(0, len(alphas) - 1)]
    shapes = ellipses_2d(rng, count)
    nlev = 1
    m = n
    while m % 2 == 0 and m // 2 >= 4:
        m //= 2
        nlev += 1
    return Problem(name=f"batch2d_{seed}_n{n}", dim=2, n=(n, n), lo=(0.0, 0.0), hi=(1.0, 1.0),
                   shapes=shapes, alpha=alpha, qdepth=4, nlevels=nlev, preset=0,
                   force_kind=1, force=(1.0, 1.0, 0.0))


def channel_replay_2d(seed: int = 0, nx: int = 1024, ny: int = 256, nlevels: int = 6,
                      alpha: float = 1e-10) -> Problem:
    """Stand-in for the paper's channel flow benchmark (Sec. 4): a 2.2 x 0.41
    channel on an nx x ny background grid (1024 x 256 is the size of the
    paper's coarse grid Omega^1 in Table tab:grid), a cylinder of diameter 0.1
    near the inflow (centre drawn in [0.15, 0.25] x [0.15, 0.26]: the exact
    benchmark position is not given in the paper), parabolic inflow with
    ubar = 0.3, eta = 1e-3, alpha = 1e-10, no body force, V(6,6) cycles."""
    rng = SplitMix64(0xC4A77E1 + seed)
    cx, cy = rng.uniform(0.15, 0.25), rng.uniform(0.15, 0.26)
    shapes = np.array([[0.0, cx, cy, 0.0, 0.05, 0.05, 0.05, 1.0, 0.0]])
    return Problem(name=f"channel_replay_{nx}x{ny}_s{seed}", dim=2, n=(nx, ny), lo=(0.0, 0.0),
                   hi=(2.2, 0.41), shapes=shapes, alpha=alpha, qdepth=4, nlevels=nlevels,
                   nu_pre=6, nu_post=6, preset=0, force_kind=0, force=(0.0, 0.0, 0.0))


def roofline_2d(n: int = 4096, nlevels: int = 9) -> Problem:
    """2D case shaped like the paper's 53M-DoF grid: n^2 cells, one circle of
    radius 0.2 at the centre, alpha = 1e-10."""
    shapes = np.array([[0.0, 0.5, 0.5, 0.0, 0.2, 0.2, 0.2, 1.0, 0.0]])
    return Problem(name=f"roofline2d_n{n}", dim=2, n=(n, n), lo=(0.0, 0.0), hi=(1.0, 1.0),
                   shapes=shapes, alpha=1e-10, qdepth=4, nlevels=nlevels, preset=0,
                   force_kind=1, force=(1.0, 1.0, 0.0))


def random_vector(problem: Problem, seed: int, level: int | None = None) -> np.ndarray:
    """Uniform(-1, 1) vector of the level's DoF count."""
    return uniform_array(problem.ndof(level), seed)


def serving_stream(seed: int = 0, count: int = 2000, rate: float = 50.0,
                   sizes=(16, 32, 48, 64, 96), min_spheres: int = 5, max_spheres: int = 200):
    """Poisson arrivals (exponential gaps, mean 1/rate) of 3D porous-medium
    solves: grid n from ``sizes``, sphere count uniform in [min, max] with the
    radius law of ``radius_scale``.  Returns a list of (arrival_s, Problem).
    Draw order per request: gap, size, count, then the geometry seed."""
    rng = SplitMix64(0x5E4E0000 + seed)
    t = 0.0
    out = []
    for k in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        n = sizes[rng.randint(0, len(sizes) - 1)]
        ns = rng.randint(min_spheres, max_spheres)
        gseed = rng.next_u64() & 0xFFFFFFFF
        nlev = 1
        m = n
        while m % 2 == 0 and m // 2 >= 4:
            m //= 2
            nlev += 1
        p = porous_3d(gseed, n=n, nspheres=ns, nlevels=nlev)
        p.name = f"serve{k}_n{n}_k{ns}"
        out.append((t, p))
    return out

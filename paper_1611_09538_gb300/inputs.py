"""Seeded synthetic charge systems shaped like the paper's workloads.

This module only draws positions and charges; it holds none of the method's
arithmetic, so both the CUDA path and the FP64 oracle consume the same bytes
without sharing any numerics.

Workloads (positions in the box [0,Lx)x[0,Ly)x[0,Lz), z periodic):
  * uniform charges with alternating signs (Section 6, Examples 6.1-6.3),
  * uniform charges with U[-1,1] values shifted to zero net charge,
  * Gaussian blobs (clustered systems, a stress case for cell lists),
  * a charged wall facing an oppositely charged cloud (stand-in for Example 6.6),
  * batches of independent systems with log-uniform N and random Lz.
Every generator uses numpy's PCG64 (``default_rng(seed)``) in float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class System:
    """One charge system plus the SE1P parameters it is evaluated with."""

    x: np.ndarray  # [N,3] float64, x,y in [0,L) (free), z in [0,Lz) (periodic)
    q: np.ndarray  # [N] float64, sum(q) == 0 up to rounding
    L: tuple  # (Lx, Ly, Lz)
    params: dict = field(default_factory=dict)
    name: str = ""


def uniform_alternating(n: int, L=(1.0, 1.0, 1.0), seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """N uniform positions, charges +1,-1,+1,... (neutral for even N)."""
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3)) * np.asarray(L, dtype=np.float64)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    if n % 2 == 1:  # keep odd-N systems neutral: last charge absorbs the surplus
        q[-1] = 0.0
    return x, q


def uniform_shifted(n: int, L=(1.0, 1.0, 1.0), seed: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """N uniform positions, charges U[-1,1] minus their mean (zero net charge)."""
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3)) * np.asarray(L, dtype=np.float64)
    q = rng.uniform(-1.0, 1.0, n)
    q -= q.mean()
    return x, q


def clustered(n: int, L=(1.0, 1.0, 2.0), centres: int = 8, sigma: float = 0.05,
              seed: int = 3) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian blobs: centres ~ U([0.2,0.8]^2 x [0,Lz)), points ~ N(c, sigma^2 I).

    x,y samples falling outside [0,L) are redrawn; z is wrapped periodically.
    Charges alternate +-1 (neutral for even N).
    """
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = L
    c = np.column_stack([rng.uniform(0.2 * Lx, 0.8 * Lx, centres),
                         rng.uniform(0.2 * Ly, 0.8 * Ly, centres),
                         rng.uniform(0.0, Lz, centres)])
    which = rng.integers(0, centres, n)
    x = c[which] + sigma * rng.standard_normal((n, 3))
    for ax, Lax in ((0, Lx), (1, Ly)):
        bad = (x[:, ax] < 0) | (x[:, ax] >= Lax)
        while bad.any():
            x[bad, ax] = c[which[bad], ax] + sigma * rng.standard_normal(int(bad.sum()))
            bad = (x[:, ax] < 0) | (x[:, ax] >= Lax)
    x[:, 2] = np.mod(x[:, 2], Lz)
    x[:, 2][x[:, 2] >= Lz] = 0.0
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    if n % 2 == 1:
        q[-1] = 0.0
    return x, q


def cloud_wall_like(n: int, L: float, seed: int = 5) -> tuple[np.ndarray, np.ndarray]:
    """A charged wall facing a cloud of opposite charge, in the cube [0,L)^3 (z periodic).

    Stand-in for the cloud-wall system of Section 6 (Example 6.6), whose generator the paper
    does not give: a strongly polar arrangement with a large dipole along the free axis x.
    Charges +1 (first half): x ~ L/2 + N(0, (0.01 L)^2), y, z uniform.  Charges -1 (second
    half): a Gaussian cloud around (L/4, L/2, L/2) with sigma = L/10.  x, y samples outside
    [0, L) are redrawn; z is wrapped.  Neutral (for odd n one wall charge is 0)."""
    rng = np.random.default_rng(seed)
    n_wall = n - n // 2
    x = np.empty((n, 3))
    x[:n_wall, 0] = L / 2 + 0.01 * L * rng.standard_normal(n_wall)
    x[:n_wall, 1:] = rng.random((n_wall, 2)) * L
    c = np.array([L / 4, L / 2, L / 2])
    x[n_wall:] = c + 0.1 * L * rng.standard_normal((n - n_wall, 3))
    for ax in (0, 1):
        while True:
            bad = np.flatnonzero((x[:, ax] < 0) | (x[:, ax] >= L))
            if bad.size == 0:
                break
            wall, cloud = bad[bad < n_wall], bad[bad >= n_wall]
            if ax == 0:
                x[wall, 0] = L / 2 + 0.01 * L * rng.standard_normal(wall.size)
            else:
                x[wall, 1] = rng.random(wall.size) * L
            x[cloud, ax] = c[ax] + 0.1 * L * rng.standard_normal(cloud.size)
    x[:, 2] = np.mod(x[:, 2], L)
    x[:, 2][x[:, 2] >= L] = 0.0
    q = np.where(np.arange(n) < n_wall, 1.0, -1.0)
    if n % 2 == 1:  # odd n: the wall holds one charge more; keep the system neutral
        q[n_wall - 1] = 0.0
    return x, q


def batch_systems(count: int = 64, n_lo: int = 1000, n_hi: int = 50000, lz_lo: float = 1.0,
                  lz_hi: float = 4.0, seed: int = 4) -> list[System]:
    """Independent uniform neutral systems, N log-uniform in [n_lo, n_hi], L=[1,1,Lz]."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        n = 2 * int(round(math.exp(rng.uniform(math.log(n_lo / 2), math.log(n_hi / 2)))))
        lz = float(rng.uniform(lz_lo, lz_hi))
        x, q = uniform_alternating(n, (1.0, 1.0, lz), seed=seed + 1000 + i)
        out.append(System(x, q, (1.0, 1.0, lz), name=f"batch{i}"))
    return out


# ---------------------------------------------------------------------------
# Named workloads.  Parameters follow the paper's recipe (Section 4.3):
# M/2 = k_inf, P even, s_l and n_l for the local pad set, s0 >= 1+sqrt(2).
# Integer FFT sizes are given explicitly so that every consumer uses the same
# grids without deriving them from each other.
# ---------------------------------------------------------------------------

def parity_p0() -> System:
    """N=1000 uniform, xi=8, M=40^3, P=24, s_l=4, n_l=6 (Example 6.3-like accuracy)."""
    x, q = uniform_alternating(1000, seed=0)
    return System(x, q, (1.0, 1.0, 1.0), dict(xi=8.0, M=(40, 40, 40), P=24, Mt=64, n0=192,
                                                nI=256, nl=6, rc=0.3), "P0")


def config_c1() -> System:
    """N=1000 uniform, xi=8, M=32^3, P=16, rc=0.3."""
    x, q = uniform_alternating(1000, seed=0)
    return System(x, q, (1.0, 1.0, 1.0), dict(xi=8.0, M=(32, 32, 32), P=16, Mt=48, n0=144,
                                                nI=144, nl=3, rc=0.3), "C1")


def config_c2(n: int = 100_000) -> System:
    """N=100k uniform in [0,1)^3, q~U[-1,1]-mean, xi=20, M=64^3, P=24, s_l=2, n_l=4, rc=0.15."""
    x, q = uniform_shifted(n, seed=1)
    return System(x, q, (1.0, 1.0, 1.0), dict(xi=20.0, M=(64, 64, 64), P=24, Mt=96, n0=288,
                                                nI=192, nl=4, rc=0.15), "C2")


def config_c3(n: int = 1_000_000) -> System:
    """N=1M uniform in [0,1)x[0,1)x[0,8), +-1, xi=40, M=64x64x512, P=24, rc=0.09."""
    x, q = uniform_alternating(n, (1.0, 1.0, 8.0), seed=2)
    return System(x, q, (1.0, 1.0, 8.0), dict(xi=40.0, M=(64, 64, 512), P=24, Mt=96, n0=288,
                                                nI=192, nl=4, rc=0.09), "C3")


def config_c3_resolved(n: int = 1_000_000) -> System:
    """The C3 charges on the grid that resolves xi = 40: M = 128 x 128 x 1024 (h = 1/128,
    eta = 0.83 < 1).  The printed grid (h = 1/64) gives eta = 3.3, where the scaling grows
    with k and amplifies FP32 rounding ~1e6-fold (Eq. 3.3)."""
    s = config_c3(n)
    s.params = dict(xi=40.0, M=(128, 128, 1024), P=24, Mt=160, n0=480, nI=320, nl=4, rc=0.09)
    s.name = "C3 resolved"
    return s


def config_c4(n: int = 200_000) -> System:
    """N=200k in 8 Gaussian blobs (sigma=0.05) in L=[1,1,2], +-1.

    The lowest z mode is k3 = pi (L3 = 2), so the I slabs use s_l = 4 (nI = 384):
    the quadrature error of Section 4.2 behaves like exp(-|k3| s_l Lt)."""
    x, q = clustered(n, seed=3)
    return System(x, q, (1.0, 1.0, 2.0), dict(xi=20.0, M=(64, 64, 128), P=24, Mt=96, n0=288,
                                                nI=384, nl=4, rc=0.15), "C4")

"""Seeded synthetic particle sets shaped like the paper's three test problems.

This module only draws random inputs; it contains none of the merging
arithmetic, so both the CUDA path and the CPU oracle can consume its output.

Units: positions are in grid-cell units (cell size L = 1, cell ``c`` spans
[c, c+1) on each axis, linear id ``c = ix + nx*(iy + ny*iz)``), momenta in
units of m*c, weights are dimensionless.  Particles are emitted cell-major
(ascending cell id); ``shuffle=True`` applies one seeded global permutation.

Workloads (all seeded with ``numpy.random.default_rng(seed)``, PCG64):

* ``counter_beams``  - stand-in for the counter-propagating plasma blocks of
  Sec. 4.1: 1D grid of 64 cells x 200 particles, 1D position + 3D momentum,
  two drifting beams (gamma*beta = +-0.3/sqrt(1-0.09)) with Gaussian spread
  0.02 on every momentum component, unit weights, tol_x = tol_p = 0.1, seed 0.
* ``two_stream``  - stand-in for the two-stream instability of Sec. 4.2:
  1D grid of 4096 cells, N_c = round(1000 (1 + 0.01 sin(2 pi (c + 1/2)/256))),
  two beams at +-0.2/sqrt(1-0.04) with spread 0.01, unit weights, tol 0.05,
  seed 1.
* ``shower``  - stand-in for the magnetic shower of Sec. 4.3: 2D grid
  512 x 512, N_c = min(20000, floor(LogNormal(ln 50, 1.5))), |p| log-uniform
  on [1, 1e4], directions uniform on the 10-degree cap about +x, weights
  LogNormal(0, 1), tol 0.05 (the tolerance is not given for this workload;
  the two-stream value is reused), seed 2.
* ``two_stream_f32``  - the ``two_stream`` particles rounded to float32.
* ``hot_6d``  - 3D grid 128^3, N_c ~ Poisson(64) with a seeded 1 % of cells
  holding 5000 particles, Maxwell-Juettner momenta at T = 0.1 m c^2 drawn by
  inverse-transform sampling of a tabulated CDF of u^2 exp(-gamma/T), boosted
  to a drift of 0.5c along z with the flipping method of Zenitani (2015,
  Phys. Plasmas 22, 042116), weights U[0.5, 1.5], float32, tol_x = 0.1,
  tol_p = 0.05, seed 4.

Every workload accepts a smaller grid (``cells=`` / ``grid=``) so tests can use
the same distribution at a size a CPU finishes in seconds.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Particles:
    """One call's worth of particles in SoA layout (host numpy arrays)."""

    name: str
    dx: int
    dp: int
    n_cells: int
    cell_size: tuple
    tol_x: float
    tol_p: float
    n_min: int
    cell: np.ndarray  # int32 [n]
    pos: np.ndarray  # [dx, n] float64 or float32
    mom: np.ndarray  # [dp, n]
    w: np.ndarray  # [n]

    @property
    def n(self) -> int:
        return int(self.cell.shape[0])

    @property
    def dtype(self):
        return self.pos.dtype

    def astype(self, dtype) -> "Particles":
        return dataclasses.replace(
            self,
            name=self.name + "_" + np.dtype(dtype).name,
            pos=np.ascontiguousarray(self.pos.astype(dtype)),
            mom=np.ascontiguousarray(self.mom.astype(dtype)),
            w=np.ascontiguousarray(self.w.astype(dtype)),
        )

    def shuffled(self, seed: int) -> "Particles":
        perm = np.random.default_rng(seed).permutation(self.n)
        return dataclasses.replace(
            self,
            name=self.name + "_shuffled",
            cell=np.ascontiguousarray(self.cell[perm]),
            pos=np.ascontiguousarray(self.pos[:, perm]),
            mom=np.ascontiguousarray(self.mom[:, perm]),
            w=np.ascontiguousarray(self.w[perm]),
        )

    def select_cells(self, cells) -> "Particles":
        """The sub-problem made of the given cells only (cell ids kept)."""
        mask = np.isin(self.cell, np.asarray(cells, dtype=np.int64))
        return dataclasses.replace(
            self,
            name=self.name + "_subset",
            cell=np.ascontiguousarray(self.cell[mask]),
            pos=np.ascontiguousarray(self.pos[:, mask]),
            mom=np.ascontiguousarray(self.mom[:, mask]),
            w=np.ascontiguousarray(self.w[mask]),
        )

    def nbytes(self) -> int:
        return self.cell.nbytes + self.pos.nbytes + self.mom.nbytes + self.w.nbytes


def _cell_ids(counts: np.ndarray) -> np.ndarray:
    return np.repeat(np.arange(counts.shape[0], dtype=np.int32), counts)


def _positions_in_cells(rng, cell: np.ndarray, grid: tuple, dtype) -> np.ndarray:
    dx = len(grid)
    n = cell.shape[0]
    pos = np.empty((dx, n), dtype=dtype)
    rem = cell.astype(np.int64)
    for a in range(dx):
        idx = rem % grid[a]
        rem = rem // grid[a]
        pos[a] = (idx + rng.random(n)).astype(dtype)
    return pos


def counter_beams(cells: int = 64, per_cell: int = 200, seed: int = 0) -> Particles:
    rng = np.random.default_rng(seed)
    counts = np.full(cells, per_cell, dtype=np.int64)
    cell = _cell_ids(counts)
    n = cell.shape[0]
    pos = _positions_in_cells(rng, cell, (cells,), np.float64)
    u_d = 0.3 / math.sqrt(1.0 - 0.09)
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    mom = rng.normal(0.0, 0.02, size=(3, n))
    mom[0] += sign * u_d
    w = np.ones(n)
    return Particles("counter_beams", 1, 3, cells, (1.0, 1.0, 1.0), 0.1, 0.1, 0,
                     cell, pos, np.ascontiguousarray(mom), w)


def two_stream(cells: int = 4096, seed: int = 1) -> Particles:
    rng = np.random.default_rng(seed)
    c = np.arange(cells)
    counts = np.rint(1000.0 * (1.0 + 0.01 * np.sin(2.0 * math.pi * (c + 0.5) / 256.0)))
    counts = counts.astype(np.int64)
    cell = _cell_ids(counts)
    n = cell.shape[0]
    pos = _positions_in_cells(rng, cell, (cells,), np.float64)
    u_d = 0.2 / math.sqrt(1.0 - 0.04)
    # alternate beams inside each cell
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    local = np.arange(n) - np.repeat(starts, counts)
    sign = np.where(local % 2 == 0, 1.0, -1.0)
    mom = rng.normal(0.0, 0.01, size=(3, n))
    mom[0] += sign * u_d
    w = np.ones(n)
    return Particles("two_stream", 1, 3, cells, (1.0, 1.0, 1.0), 0.05, 0.05, 0,
                     cell, pos, np.ascontiguousarray(mom), w)


def two_stream_f32(cells: int = 4096, seed: int = 1) -> Particles:
    p = two_stream(cells, seed).astype(np.float32)
    p.name = "two_stream_f32"
    return p


def shower(grid: tuple = (512, 512), seed: int = 2, cap: int = 20000) -> Particles:
    rng = np.random.default_rng(seed)
    n_cells = grid[0] * grid[1]
    counts = np.floor(rng.lognormal(math.log(50.0), 1.5, size=n_cells))
    counts = np.minimum(counts, cap).astype(np.int64)
    cell = _cell_ids(counts)
    n = cell.shape[0]
    pos = _positions_in_cells(rng, cell, grid, np.float64)
    pmag = 10.0 ** rng.uniform(0.0, 4.0, size=n)
    cos_t = rng.uniform(math.cos(math.radians(10.0)), 1.0, size=n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    mom = np.empty((3, n))
    mom[0] = pmag * cos_t
    mom[1] = pmag * sin_t * np.cos(phi)
    mom[2] = pmag * sin_t * np.sin(phi)
    w = rng.lognormal(0.0, 1.0, size=n)
    return Particles("shower", 2, 3, n_cells, (1.0, 1.0, 1.0), 0.05, 0.05, 0,
                     cell, pos, mom, w)


def _juettner_table(T: float, m: int = 1 << 16):
    """Tabulated CDF of the rest-frame Maxwell-Juettner speed density."""
    u_max = 40.0 * T + 40.0 * math.sqrt(T)
    u = np.linspace(0.0, u_max, m)
    f = u * u * np.exp(-(np.sqrt(1.0 + u * u) - 1.0) / T)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(u))])
    cdf /= cdf[-1]
    return u, cdf


def _juettner_boosted(rng, n: int, T: float, beta: float, dtype) -> np.ndarray:
    u_tab, cdf = _juettner_table(T)
    u = np.interp(rng.random(n), cdf, u_tab)
    # isotropic direction
    mu = rng.uniform(-1.0, 1.0, size=n)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    ux = u * s * np.cos(phi)
    uy = u * s * np.sin(phi)
    uz = u * mu
    # flipping method: flip u_z when -beta v_z > X, then boost along z
    gam = np.sqrt(1.0 + u * u)
    flip = -beta * (uz / gam) > rng.random(n)
    uz = np.where(flip, -uz, uz)
    Gam = 1.0 / math.sqrt(1.0 - beta * beta)
    uz = Gam * (uz + beta * gam)
    mom = np.empty((3, n), dtype=dtype)
    mom[0], mom[1], mom[2] = ux, uy, uz
    return mom


def hot_6d(grid: tuple = (128, 128, 128), seed: int = 4, hot_count: int = 5000,
           hot_frac: float = 0.01, mean: float = 64.0) -> Particles:
    rng = np.random.default_rng(seed)
    n_cells = grid[0] * grid[1] * grid[2]
    counts = rng.poisson(mean, size=n_cells).astype(np.int64)
    n_hot = int(round(hot_frac * n_cells))
    if n_hot:
        counts[rng.choice(n_cells, size=n_hot, replace=False)] = hot_count
    cell = _cell_ids(counts)
    n = cell.shape[0]
    pos = _positions_in_cells(rng, cell, grid, np.float32)
    mom = np.empty((3, n), dtype=np.float32)
    chunk = 1 << 24
    for b in range(0, n, chunk):
        e = min(n, b + chunk)
        mom[:, b:e] = _juettner_boosted(rng, e - b, 0.1, 0.5, np.float32)
    w = rng.uniform(0.5, 1.5, size=n).astype(np.float32)
    return Particles("hot_6d", 3, 3, n_cells, (1.0, 1.0, 1.0), 0.1, 0.05, 0,
                     cell, pos, mom, w)


WORKLOADS = {
    "counter_beams": counter_beams,
    "two_stream": two_stream,
    "shower": shower,
    "two_stream_f32": two_stream_f32,
    "hot_6d": hot_6d,
}


def random_cell(rng, m: int, dx: int = 1, dp: int = 3, dtype=np.float64,
                drift=(0.3, 0.0, 0.0), spread: float = 0.05,
                weights: str = "uniform") -> Particles:
    """A single cell (id 0) of ``m`` particles: small random cases for tests."""
    pos = rng.random((dx, m))
    mom = rng.normal(0.0, spread, size=(dp, m))
    for a in range(dp):
        mom[a] += drift[a] if a < len(drift) else 0.0
    if weights == "uniform":
        w = np.ones(m)
    else:
        w = rng.lognormal(0.0, 1.0, size=m)
    return Particles("random_cell", dx, dp, 1, (1.0, 1.0, 1.0), 0.1, 0.1, 0,
                     np.zeros(m, dtype=np.int32), pos.astype(dtype),
                     mom.astype(dtype), w.astype(dtype))

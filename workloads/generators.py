"""Seeded synthetic point sets shaped like the paper's low-dimensional workloads.

This module draws random numbers and lays out float32 point arrays. It holds
none of the clustering arithmetic (no distance test, no grid, no tree): both
the CPU oracle and the CUDA path take its output as plain input.

The paper's own datasets (GPS traces, cosmology particles; Table 1) are not
available; every family below is a stand-in with the same dimension, size and
kind of structure:

* ``blobs``     -- isotropic Gaussian blobs plus uniform noise (small cases).
* ``roads``     -- 2D GPS-trace-like points jittered along random polylines.
* ``halos``     -- 3D cosmology-like particles: NFW-profile halos with a
                   power-law size distribution plus a uniform background.
* ``batch``     -- thousands of blob instances with lognormal sizes.
* ``serve_schedule`` -- Poisson arrivals of jobs, each a window of one of
                   the ``serve_pools`` (shuffled point sets of the above).

All generators use ``numpy.random.Generator(PCG64(seed))`` and return
C-contiguous ``float32`` arrays of shape ``(n, d)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "blobs", "roads", "halos", "halo_eps", "batch_instances", "serve_pools", "serve_schedule",
    "uniform", "Instance", "ServeJob", "SERVE_POOL_N", "SERVE_FAMILIES",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, d: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``n`` points uniform in ``[lo, hi]^d``."""
    r = _rng(seed)
    return np.ascontiguousarray(r.uniform(lo, hi, size=(n, d)).astype(np.float32))


def blobs(n: int, d: int, seed: int, n_blobs: int = 8, sigma: float = 0.02,
          blob_frac: float = 0.9) -> np.ndarray:
    """Gaussian blobs plus uniform noise in the unit cube.

    ``round(blob_frac * n)`` points are split multinomially over ``n_blobs``
    equal-weight blobs with centres uniform in ``[0,1]^d`` and standard
    deviation ``sigma`` per axis (no clipping); the rest are uniform in
    ``[0,1]^d``. The result is shuffled.
    """
    r = _rng(seed)
    n_blob = int(round(blob_frac * n))
    n_noise = n - n_blob
    centres = r.uniform(0.0, 1.0, size=(n_blobs, d))
    counts = r.multinomial(n_blob, [1.0 / n_blobs] * n_blobs)
    parts = []
    for c, k in zip(centres, counts):
        parts.append(c + sigma * r.standard_normal(size=(int(k), d)))
    parts.append(r.uniform(0.0, 1.0, size=(n_noise, d)))
    pts = np.concatenate(parts, axis=0)
    pts = pts[r.permutation(n)]
    return np.ascontiguousarray(pts.astype(np.float32))


def roads(n: int, seed: int, n_roads: int = 2000, n_segments: int = 10,
          seg_len: tuple[float, float] = (0.002, 0.008), jitter: float = 1e-4,
          road_frac: float = 0.95) -> np.ndarray:
    """2D GPS-trace-like points along random polylines in ``[0,1]^2``.

    Each road starts uniform in ``[0.05,0.95]^2`` and takes ``n_segments``
    steps with a uniform heading and a length uniform in ``seg_len``; the
    vertices are clamped to the unit square. ``road_frac`` of the points are
    placed on the roads (segment chosen in proportion to its length, position
    uniform along it) with ``N(0, jitter^2)`` noise on each axis; the rest are
    uniform in the unit square.
    """
    r = _rng(seed)
    n_road = int(round(road_frac * n))
    n_noise = n - n_road
    start = r.uniform(0.05, 0.95, size=(n_roads, 1, 2))
    heading = r.uniform(0.0, 2.0 * math.pi, size=(n_roads, n_segments))
    length = r.uniform(seg_len[0], seg_len[1], size=(n_roads, n_segments))
    steps = np.stack([np.cos(heading) * length, np.sin(heading) * length], axis=-1)
    verts = np.concatenate([start, start + np.cumsum(steps, axis=1)], axis=1)
    verts = np.clip(verts, 0.0, 1.0)
    a = verts[:, :-1, :].reshape(-1, 2)
    b = verts[:, 1:, :].reshape(-1, 2)
    seglen = np.linalg.norm(b - a, axis=1)
    p = seglen / seglen.sum()
    counts = r.multinomial(n_road, p)
    seg_of = np.repeat(np.arange(a.shape[0]), counts)
    t = r.uniform(0.0, 1.0, size=(n_road, 1))
    on = a[seg_of] + t * (b[seg_of] - a[seg_of])
    on += jitter * r.standard_normal(size=on.shape)
    noise = r.uniform(0.0, 1.0, size=(n_noise, 2))
    pts = np.concatenate([on, noise], axis=0)
    pts = pts[r.permutation(n)]
    return np.ascontiguousarray(pts.astype(np.float32))


def _nfw_mass(x: np.ndarray) -> np.ndarray:
    return np.log1p(x) - x / (1.0 + x)


def _nfw_inverse(u: np.ndarray, c: float, iters: int = 32) -> np.ndarray:
    """Radius in units of ``r_s`` whose enclosed NFW mass fraction (truncated
    at concentration ``c``) equals ``u``; float64 bisection on ``[0, c]``."""
    target = u * _nfw_mass(np.asarray(c, dtype=np.float64))
    lo = np.zeros_like(u)
    hi = np.full_like(u, c)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        below = _nfw_mass(mid) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def halo_eps(n: int) -> float:
    """0.2 times the mean inter-particle spacing of ``n`` points in the unit
    cube, rounded to float32 (the linking length used with ``halos``)."""
    return float(np.float32(0.2 * n ** (-1.0 / 3.0)))


def halos(n: int, seed: int, n_halos: int = 50000, size_range: tuple[float, float] = (10.0, 1e5),
          r_s: float = 0.002, conc: float = 10.0, halo_frac: float = 0.7,
          chunk: int = 1 << 22) -> np.ndarray:
    """3D cosmology-like particles: NFW halos plus a uniform background.

    Halo sizes are drawn from ``p(s) ~ s^-2`` on ``size_range`` and rescaled
    (largest remainder) so they sum to ``round(halo_frac * n)``. Centres are
    uniform in ``[0.02, 0.98]^3``; each particle's radius follows the NFW
    enclosed-mass profile with scale radius ``r_s`` truncated at ``conc * r_s``
    (so every halo stays inside the unit cube); directions are isotropic. The
    remaining particles are uniform in ``[0,1]^3``. The result is shuffled.
    """
    r = _rng(seed)
    n_halo_pts = int(round(halo_frac * n))
    n_bg = n - n_halo_pts
    smin, smax = size_range
    u = r.uniform(0.0, 1.0, size=n_halos)
    sizes = 1.0 / (1.0 / smin - u * (1.0 / smin - 1.0 / smax))
    scaled = sizes * (n_halo_pts / sizes.sum())
    base = np.floor(scaled).astype(np.int64)
    rem = n_halo_pts - int(base.sum())
    if rem > 0:
        order = np.argsort(-(scaled - base), kind="stable")
        base[order[:rem]] += 1
    centres = r.uniform(0.02, 0.98, size=(n_halos, 3))
    halo_of = np.repeat(np.arange(n_halos), base)
    out = np.empty((n, 3), dtype=np.float32)
    for s in range(0, n_halo_pts, chunk):
        e = min(n_halo_pts, s + chunk)
        k = e - s
        rad = r_s * _nfw_inverse(r.uniform(0.0, 1.0, size=k), conc)
        v = r.standard_normal(size=(k, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        out[s:e] = (centres[halo_of[s:e]] + rad[:, None] * v).astype(np.float32)
    out[n_halo_pts:] = r.uniform(0.0, 1.0, size=(n_bg, 3)).astype(np.float32)
    perm = r.permutation(n)
    return np.ascontiguousarray(out[perm])


@dataclass
class Instance:
    """One clustering problem of a batch."""
    points: np.ndarray
    eps: float
    min_pts: int

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def dim(self) -> int:
        return int(self.points.shape[1])


def batch_instances(count: int, seed: int, median: float = 20000.0, sigma: float = 1.2,
                    clip: tuple[int, int] = (1000, 500000), eps_range: tuple[float, float] = (0.01, 0.05),
                    min_pts_choices: tuple[int, ...] = (2, 5, 10), size_scale: float = 1.0) -> list[Instance]:
    """Independent blob instances with lognormal sizes.

    Sizes are ``lognormal(ln median, sigma)`` clipped to ``clip`` (then
    multiplied by ``size_scale``, at least 1); the dimension is uniform in
    {2, 3}; each instance is ``blobs`` in that dimension with 8 blobs;
    ``eps`` is uniform in ``eps_range`` (rounded to float32) and ``min_pts``
    uniform over ``min_pts_choices``.
    """
    r = _rng(seed)
    sizes = np.clip(r.lognormal(math.log(median), sigma, size=count), clip[0], clip[1])
    sizes = np.maximum(1, np.round(sizes * size_scale)).astype(np.int64)
    dims = r.choice([2, 3], size=count)
    epss = r.uniform(eps_range[0], eps_range[1], size=count).astype(np.float32)
    mps = r.choice(np.asarray(min_pts_choices), size=count)
    seeds = r.integers(0, 2**62, size=count)
    out = []
    for i in range(count):
        pts = blobs(int(sizes[i]), int(dims[i]), int(seeds[i]))
        out.append(Instance(pts, float(epss[i]), int(mps[i])))
    return out


@dataclass
class ServeJob:
    """One request of a serving schedule: ``n`` rows of pool ``pool`` starting
    at row ``offset``, clustered with ``eps``, ``min_pts`` and ``algo``."""
    arrival_s: float
    family: str
    pool: str
    offset: int
    n: int
    eps: float
    min_pts: int
    algo: int


SERVE_POOL_N = 8_000_000
SERVE_FAMILIES = ("blobs3", "roads", "halos", "batch")


def serve_pools(n: int, seed: int) -> dict[str, np.ndarray]:
    """The shuffled point pools the jobs of a serving schedule read from:
    3D and 2D blobs, roads and halos, ``n`` points each (the halo count
    scaled from 50,000 halos per 2^24 points). As every pool is shuffled, a
    window of ``k`` consecutive rows is a uniform random subsample."""
    r = _rng(seed)
    s = r.integers(0, 2**62, size=4)
    return {
        "blobs3": blobs(n, 3, int(s[0])),
        "blobs2": blobs(n, 2, int(s[1])),
        "roads": roads(n, int(s[2])),
        "halos": halos(n, int(s[3]), n_halos=max(10, int(round(50000 * n / 2**24)))),
    }


def serve_schedule(n_jobs: int, rate_per_s: float, seed: int, pool_n: int = SERVE_POOL_N,
                   size_range: tuple[int, int] = (10_000, 8_000_000),
                   families: tuple[str, ...] = SERVE_FAMILIES) -> list[ServeJob]:
    """Poisson arrivals of jobs drawn from the workload families.

    Inter-arrival times are exponential with mean ``1/rate_per_s``; sizes
    are log-uniform on ``size_range`` (capped at ``pool_n``); the family is
    uniform over ``families``; each job reads a random window of its pool.

    * ``blobs3``: 3D blobs, eps 0.03, minPts 5, DenseBox.
    * ``roads``: eps rescaled with the size so that the point density per
      neighbourhood is kept (``2e-4 * (4194304 / n)^(1/2)``), minPts 10,
      FDbscan.
    * ``halos``: eps ``halo_eps(n)``, minPts 10, DenseBox.
    * ``batch``: one instance of a batch -- blobs in 2D or 3D (uniform), eps
      uniform in [0.01, 0.05], minPts uniform in {2, 5, 10}, DenseBox.
    """
    r = _rng(seed)
    t = np.cumsum(r.exponential(1.0 / rate_per_s, size=n_jobs))
    sizes = np.exp(r.uniform(math.log(size_range[0]), math.log(size_range[1]), size=n_jobs)).astype(np.int64)
    sizes = np.minimum(sizes, pool_n)
    fam = r.choice(len(families), size=n_jobs)
    u = r.uniform(0.0, 1.0, size=(n_jobs, 4))
    jobs = []
    for i in range(n_jobs):
        f = families[int(fam[i])]
        n = int(sizes[i])
        off = int(u[i, 0] * (pool_n - n + 1))
        if f == "blobs3":
            jobs.append(ServeJob(float(t[i]), f, "blobs3", off, n, float(np.float32(0.03)), 5, 1))
        elif f == "roads":
            eps = float(np.float32(2e-4 * (4194304 / n) ** 0.5))
            jobs.append(ServeJob(float(t[i]), f, "roads", off, n, eps, 10, 0))
        elif f == "halos":
            jobs.append(ServeJob(float(t[i]), f, "halos", off, n, halo_eps(n), 10, 1))
        else:
            pool = "blobs2" if u[i, 1] < 0.5 else "blobs3"
            eps = float(np.float32(0.01 + 0.04 * u[i, 2]))
            mp = (2, 5, 10)[min(2, int(u[i, 3] * 3))]
            jobs.append(ServeJob(float(t[i]), f, pool, off, n, eps, mp, 1))
    return jobs

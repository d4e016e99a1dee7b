"""Seeded synthetic inputs for the photonic band-structure path.

This module holds no arithmetic of the method itself: it only produces the
permittivity samples, Bloch vectors and random starting blocks that both the
CUDA path and the CPU oracle consume. Every generator is deterministic given
its arguments (NumPy ``default_rng`` for anything random).

Conventions shared by both sides:

* a permittivity field is a float64 array of shape ``(m, n)``; entry ``[j, i]``
  is the sample at the centre ``((i+1/2) a/n, (j+1/2) b/m)`` of cell ``(i, j)``
  (flat index ``j*n + i``);
* a block of ``p`` complex columns of length ``D`` is a complex128 array of
  shape ``(p, D)``: row ``c`` is column ``c`` (column-major ``D x p``).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "cell_centres", "const_eps", "rod_eps", "disks_eps", "gxmg_path",
    "random_block", "serving_jobs",
]


def cell_centres(n: int, m: int, a: float = 1.0, b: float = 1.0):
    """Cell-centre coordinates ``(X1, X2)``, each of shape ``(m, n)``."""
    x1 = (np.arange(n) + 0.5) * (a / n)
    x2 = (np.arange(m) + 0.5) * (b / m)
    return np.meshgrid(x1, x2, indexing="xy")


def const_eps(n: int, m: int, value: float = 1.0) -> np.ndarray:
    """Homogeneous medium: every cell sample equals ``value``."""
    return np.full((m, n), float(value))


def _periodic_dist(X1, X2, c1, c2, a, b):
    d1 = np.abs(X1 - c1)
    d1 = np.minimum(d1, a - d1)
    d2 = np.abs(X2 - c2)
    d2 = np.minimum(d2, b - d2)
    return np.sqrt(d1 * d1 + d2 * d2)


def rod_eps(n: int, m: int, a: float = 1.0, b: float = 1.0, radius: float = 0.2,
            eps_rod: float = 8.9, eps_bg: float = 1.0,
            centre: tuple[float, float] | None = None) -> np.ndarray:
    """Square-lattice rod crystal sampled at cell centres.

    A cell takes ``eps_rod`` when its centre lies within periodic distance
    ``radius * a`` of the rod centre (default the cell-of-lattice centre
    ``(a/2, b/2)``), else ``eps_bg``.
    """
    X1, X2 = cell_centres(n, m, a, b)
    c1, c2 = centre if centre is not None else (0.5 * a, 0.5 * b)
    r = radius * a
    return np.where(_periodic_dist(X1, X2, c1, c2, a, b) <= r, eps_rod, eps_bg).astype(np.float64)


def disks_eps(n: int, m: int, seed: int = 0, ndisks: int = 16, rmin: float = 0.05,
              rmax: float = 0.15, epsmin: float = 2.0, epsmax: float = 13.0,
              eps_bg: float = 1.0, a: float = 1.0, b: float = 1.0,
              max_tries: int = 100000) -> np.ndarray:
    """Random field of non-overlapping disks (periodic distance), background ``eps_bg``.

    Centres U[0,a)x[0,b), radii U(rmin, rmax)*a, permittivities U(epsmin, epsmax);
    a candidate is rejected when it overlaps an accepted disk
    (``d <= r1 + r2`` under periodic distance).
    """
    rng = np.random.default_rng(seed)
    disks = []
    tries = 0
    while len(disks) < ndisks:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("disks_eps: could not place the requested disks")
        c = (rng.uniform(0, a), rng.uniform(0, b))
        r = rng.uniform(rmin, rmax) * a
        e = rng.uniform(epsmin, epsmax)
        ok = True
        for (d1, d2, rr, _) in disks:
            dx = abs(c[0] - d1); dx = min(dx, a - dx)
            dy = abs(c[1] - d2); dy = min(dy, b - dy)
            if np.hypot(dx, dy) <= r + rr:
                ok = False
                break
        if ok:
            disks.append((c[0], c[1], r, e))
    X1, X2 = cell_centres(n, m, a, b)
    out = np.full((m, n), float(eps_bg))
    for (c1, c2, r, e) in disks:
        out[_periodic_dist(X1, X2, c1, c2, a, b) <= r] = e
    return out


def gxmg_path(nk: int, a: float = 1.0, b: float = 1.0) -> np.ndarray:
    """Bloch vectors along Gamma-X-M-Gamma, ``(nk, 2)`` float64.

    ``nk - 1`` must be a multiple of 3: each leg gets ``(nk-1)/3`` equal steps,
    Gamma=(0,0), X=(pi/a,0), M=(pi/a,pi/b); Gamma appears at both ends.
    """
    if nk < 4 or (nk - 1) % 3:
        raise ValueError("nk - 1 must be a positive multiple of 3")
    s = (nk - 1) // 3
    G = np.array([0.0, 0.0]); X = np.array([np.pi / a, 0.0]); M = np.array([np.pi / a, np.pi / b])
    pts = []
    for (P, Q) in ((G, X), (X, M), (M, G)):
        for t in range(s):
            pts.append(P + (Q - P) * (t / s))
    pts.append(G.copy())
    return np.array(pts)


def random_block(D: int, p: int, seed: int = 0) -> np.ndarray:
    """Random complex block, shape ``(p, D)``: ``re + 1j*im``, both standard normal.

    Drawn as ``default_rng(seed).standard_normal((2, D, p))`` so that the
    ``D x p`` column-major matrix is ``X[0] + 1j*X[1]``.
    """
    x = np.random.default_rng(seed).standard_normal((2, D, p))
    return np.ascontiguousarray((x[0] + 1j * x[1]).T)


def serving_jobs(njobs: int = 200, seed: int = 0, rate_per_s: float = 1.0,
                 grids=(128, 256, 512, 1024, 2048)):
    """Poisson-arrival band-structure jobs (rod crystals), as a list of dicts."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for jid in range(njobs):
        t += rng.exponential(1.0 / rate_per_s)
        bands = int(rng.integers(6, 13))
        nk_legs = int(rng.integers(3, 22))
        jobs.append(dict(job=jid, arrival_s=t, radius=float(rng.uniform(0.1, 0.45)),
                         eps_rod=float(rng.uniform(2, 13)), grid=int(rng.choice(grids)),
                         nk=3 * nk_legs + 1, bands=bands, block=bands + 2))
    return jobs

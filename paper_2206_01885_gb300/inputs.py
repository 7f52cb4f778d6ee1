"""Seeded synthetic inputs for the data-driven H^2 construction.

This module is the only code shared by the CUDA path's callers (tests, bench)
and the CPU oracle's callers.  It draws random numbers and nothing else: no
tree, no admissibility test, no kernel evaluation, no reduction.  Every array
is float64 and every generator is numpy's PCG64 seeded explicitly, so that the
same call returns the same bits on x86 and on Arm.

Workloads (the paper's section 6.1.1 datasets, plus the shapes used to size the
benchmark):
  * ``uniform_cube``      i.i.d. uniform points in [0,1]^d ("cube" dataset)
  * ``sphere_surface``    uniform points on the unit sphere surface
  * ``three_spheres``     points on three intersecting unit spheres whose centres
                          form an equilateral triangle of side 1 ("3-sphere")
  * ``gaussian_mixture``  16 isotropic Gaussians in [0,1]^2, std log-uniform in
                          [0.01, 0.1], samples outside the square redrawn
  * ``standard_normal``   right-hand sides z ~ N(0, 1) (section 6 error metric)
  * ``sample_rows``       row indices without replacement for the sampled check
  * ``unit_cells``        uniform points over a caller-given list of unit cells,
                          used for the artificial separated sets Z1, Z2 of the
                          r-from-epsilon calibration (section 4.2)
"""
from __future__ import annotations

import itertools

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(n: int, d: int = 3, seed: int = 1) -> np.ndarray:
    """n points i.i.d. uniform in [0,1]^d, shape (n, d), row-major float64."""
    return _rng(seed).random((n, d))


def sphere_surface(n: int, seed: int = 5, d: int = 3) -> np.ndarray:
    """n points uniform on the unit sphere surface (normalised Gaussians)."""
    g = _rng(seed).standard_normal((n, d))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def three_spheres(n: int, seed: int = 6) -> np.ndarray:
    """n points on three unit spheres with centres on an equilateral triangle of
    side 1 in the z=0 plane; roughly n/3 points per sphere."""
    rng = _rng(seed)
    centres = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, np.sqrt(3.0) / 2.0, 0.0]])
    which = rng.integers(0, 3, size=n)
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g + centres[which]


def gaussian_mixture(n: int, seed: int = 3, ncomp: int = 16, d: int = 2) -> np.ndarray:
    """n points from an equal-weight mixture of ``ncomp`` isotropic Gaussians with
    means uniform in [0,1]^d and standard deviations log-uniform in [0.01, 0.1];
    samples falling outside [0,1]^d are rejected and redrawn."""
    rng = _rng(seed)
    means = rng.random((ncomp, d))
    stds = np.exp(rng.uniform(np.log(0.01), np.log(0.1), size=ncomp))
    out = np.empty((n, d))
    filled = 0
    while filled < n:
        m = n - filled
        comp = rng.integers(0, ncomp, size=m)
        pts = means[comp] + stds[comp, None] * rng.standard_normal((m, d))
        ok = np.all((pts >= 0.0) & (pts <= 1.0), axis=1)
        pts = pts[ok]
        out[filled:filled + len(pts)] = pts
        filled += len(pts)
    return out


def standard_normal(n: int, seed: int = 11, nrhs: int = 1) -> np.ndarray:
    """Right-hand side(s) z ~ N(0,1); shape (n,) for one, (n, nrhs) otherwise."""
    z = _rng(seed).standard_normal((n, nrhs))
    return z[:, 0].copy() if nrhs == 1 else z


def sample_rows(n: int, nrows: int, seed: int = 12) -> np.ndarray:
    """``min(nrows, n)`` distinct row indices, sorted, int64."""
    nrows = min(nrows, n)
    return np.sort(_rng(seed).choice(n, size=nrows, replace=False)).astype(np.int64)


def cells_with_offsets(d: int, max_inf: int, min_sq: int) -> np.ndarray:
    """Integer offsets v with max|v_k| <= max_inf and |v|^2 >= min_sq, sorted
    lexicographically.  The caller states which ``min_sq`` makes a unit cell at
    offset v well separated from the unit cell at the origin."""
    rng_ = range(-max_inf, max_inf + 1)
    cells = [v for v in itertools.product(rng_, repeat=d) if sum(c * c for c in v) >= min_sq]
    return np.array(cells, dtype=np.float64)


def unit_cells(n: int, cells: np.ndarray, seed: int) -> np.ndarray:
    """n points, each in a cell drawn uniformly from ``cells`` (offsets of unit
    cells [v, v+1)^d), uniform inside its cell."""
    rng = _rng(seed)
    cells = np.asarray(cells, dtype=np.float64).reshape(-1, cells.shape[-1] if np.ndim(cells) > 1 else 1)
    pick = rng.integers(0, len(cells), size=n)
    return cells[pick] + rng.random((n, cells.shape[1]))


def calibration_sets(d: int, min_sq: int, n1: int = 512, n2: int = 4096,
                     seed1: int = 7, seed2: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """The artificial sets of the r-from-epsilon calibration: Z1 uniform in the
    unit cell at the origin, Z2 uniform over the unit cells at offsets v with
    max|v_k| <= 3 and |v|^2 >= ``min_sq``."""
    z1 = unit_cells(n1, np.zeros((1, d)), seed1)
    z2 = unit_cells(n2, cells_with_offsets(d, 3, min_sq), seed2)
    return z1, z2


# Named workloads: (points, kernel name, kernel parameters, leaf size, tolerance)
def workload(name: str):
    """Return (points, kernel, kparams, leaf_size, eps) for a named workload."""
    if name == "cube8k":
        return uniform_cube(8000, 3, seed=1), "coulomb", (), 200, 1e-6
    if name == "cube1m":
        return uniform_cube(1 << 20, 3, seed=2), "coulomb", (), 256, 1e-8
    if name == "gmix2m":
        return gaussian_mixture(1 << 21, seed=3), "gaussian", (0.2,), 128, 1e-6
    if name == "sphere8m":
        return sphere_surface(1 << 23, seed=5), "coulomb", (), 256, 1e-6
    raise KeyError(name)


def batched_problems(count: int, nmin: int, nmax: int, seed: int = 4):
    """Independent problems of uneven sizes (the batched configuration): for
    each, n log-uniform in [nmin, nmax], the point set ("cube" or "sphere",
    50/50) and a kernel index in {0, 1, 2}, each drawn uniformly.  Returns a
    list of (n, kind, kernel_index, point_seed)."""
    rng = _rng(seed)
    out = []
    for a in range(count):
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        kind = "cube" if rng.random() < 0.5 else "sphere"
        out.append((n, kind, int(rng.integers(0, 3)), seed * 1000 + a))
    return out

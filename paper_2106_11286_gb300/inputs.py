"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the Metropolis method's arithmetic: it only builds
neighbour lists of test geometries and draws seeded states and masks with
numpy.  Both the CUDA path and the CPU oracle take what it returns as input,
so it imports neither of them.

Geometries (all neighbour lists are symmetric CSR in natural site order):

* ``bcc_nanoparticle`` -- a sphere cut from a bcc crystal with an open
  surface, the "complex structures ... with any crystal lattice" use case of
  arXiv 2106.11286 (abstract, Sec. on lattice independence), plus a seeded
  vacancy mask.
* ``open_chain``, ``dimers``, ``isolated_sites`` -- small graphs whose
  thermodynamics has a closed form, used to pin the oracle.
"""
from __future__ import annotations

import numpy as np


def random_unit_spins(n: int, seed: int) -> np.ndarray:
    """n x 3 FP64 unit vectors, isotropic (normalised Gaussian triples)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def aligned_spins(n: int, axis) -> np.ndarray:
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    return np.tile(a, (n, 1))


def vacancy_mask(n: int, fraction: float, seed: int) -> np.ndarray:
    """uint8 mask, 0 = vacancy, drawn independently per site with numpy."""
    rng = np.random.default_rng(seed)
    return (rng.random(n) >= fraction).astype(np.uint8)


def _csr_from_lists(rows: list[list[int]]):
    row_ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([j for r in rows for j in r], dtype=np.int32)
    return row_ptr, col


def open_chain(n: int):
    """Open 1-D chain 0-1-...-(n-1)."""
    rows = [[j for j in (i - 1, i + 1) if 0 <= j < n] for i in range(n)]
    return _csr_from_lists(rows)


def dimers(n_pairs: int):
    """n_pairs disconnected two-site molecules (2k, 2k+1)."""
    rows = []
    for k in range(n_pairs):
        rows.append([2 * k + 1])
        rows.append([2 * k])
    return _csr_from_lists(rows)


def isolated_sites(n: int):
    """n sites with no bonds."""
    return np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)


# bcc neighbour offsets: a corner (basis 0) of cell c touches the centres of
# the 8 cells c + {-1,0}^3; a centre (basis 1) touches the corners c + {0,1}^3.
_BCC_OFFS = {
    0: [(dx, dy, dz) for dz in (-1, 0) for dy in (-1, 0) for dx in (-1, 0)],
    1: [(dx, dy, dz) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)],
}


def bcc_nanoparticle(radius: float, box: int, vacancy_fraction: float = 0.0, seed: int = 0,
                     return_positions: bool = False):
    """Sphere of radius ``radius`` (lattice constants) cut from a box^3-cell bcc crystal.

    Sites: corners at integer cell coordinates, centres at +1/2; a site is kept
    when its distance to the box centre (box/2, box/2, box/2) is <= radius.
    Sites are numbered in increasing full-crystal natural index
    ((cz*box + cy)*box + cx)*2 + b.  Bonds to sites outside the sphere are
    dropped (open surface).  Returns (row_ptr int64, col int32, mask uint8)
    and optionally the positions.
    """
    box = int(box)
    c0 = box / 2.0
    r2 = float(radius) ** 2
    ar = np.arange(box, dtype=np.float64)
    # full-crystal index map: -1 outside the sphere
    full = np.full((box, box, box, 2), -1, dtype=np.int64)
    inside = np.zeros((box, box, box, 2), dtype=bool)
    for b in (0, 1):
        p = ar + 0.5 * b - c0
        d2 = p[:, None, None] ** 2 + p[None, :, None] ** 2 + p[None, None, :] ** 2  # [z,y,x]
        inside[..., b] = d2 <= r2
    n = int(inside.sum())
    full[inside] = np.arange(n, dtype=np.int64)
    zz, yy, xx, bb = np.nonzero(inside)  # C order == natural order
    cols = np.full((n, 8), -1, dtype=np.int64)
    for b in (0, 1):
        sel = bb == b
        for k, (dx, dy, dz) in enumerate(_BCC_OFFS[b]):
            nx, ny, nz = xx[sel] + dx, yy[sel] + dy, zz[sel] + dz
            ok = (nx >= 0) & (nx < box) & (ny >= 0) & (ny < box) & (nz >= 0) & (nz < box)
            j = np.full(int(sel.sum()), -1, dtype=np.int64)
            j[ok] = full[nz[ok], ny[ok], nx[ok], 1 - b]
            cols[sel, k] = j
    del full
    valid = cols >= 0
    deg = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    col = cols[valid].astype(np.int32)  # row-major: keeps each row's offset order
    mask = vacancy_mask(n, vacancy_fraction, seed) if vacancy_fraction > 0 else np.ones(n, dtype=np.uint8)
    if return_positions:
        pos = np.stack([xx + 0.5 * bb, yy + 0.5 * bb, zz + 0.5 * bb], axis=1).astype(np.float64)
        return row_ptr, col, mask, pos
    return row_ptr, col, mask

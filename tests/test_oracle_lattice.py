"""Pins of the oracle's lattices and colourings by brute-force geometry.

Neighbour lists are checked against an O(n^2) search over explicit site
positions (minimum-image distance equal to the nearest-neighbour distance),
which shares nothing with the builders' index arithmetic.  Colourings are
checked to be proper (no bond inside a colour class, the independence that
makes a colour pass exact), with the class counts the crystal structure fixes.
"""
import itertools

import numpy as np
import pytest

from paper_2106_11286_gb300 import inputs

BASIS = {
    "sc": [(0, 0, 0)],
    "bcc": [(0, 0, 0), (0.5, 0.5, 0.5)],
    "fcc": [(0, 0, 0), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)],
}
NN2 = {"sc": 1.0, "bcc": 0.75, "fcc": 0.5}
Z = {"sc": 6, "bcc": 8, "fcc": 12}


def positions(kind, dims):
    Lx, Ly, Lz = dims
    pos = []
    for cz, cy, cx in itertools.product(range(Lz), range(Ly), range(Lx)):
        for b in BASIS[kind]:
            pos.append((cx + b[0], cy + b[1], cz + b[2]))
    return np.array(pos, dtype=np.float64)


def brute_neighbours(kind, dims, periodic):
    pos = positions(kind, dims)
    L = np.array(dims, dtype=float)
    d = pos[None, :, :] - pos[:, None, :]
    if periodic:
        d -= L * np.round(d / L)
    d2 = (d ** 2).sum(-1)
    return [set(np.nonzero(np.isclose(row, NN2[kind]))[0].tolist()) for row in d2], d, pos


CASES = [("sc", (4, 4, 6), True), ("sc", (3, 4, 5), False), ("bcc", (3, 4, 5), True),
         ("bcc", (3, 3, 4), False), ("fcc", (3, 3, 4), True), ("fcc", (2, 3, 3), False)]


@pytest.mark.parametrize("kind,dims,periodic", CASES)
def test_neighbours_match_geometry(orc, kind, dims, periodic):
    row_ptr, col = orc.neighbours(kind, dims, periodic)
    want, d, _ = brute_neighbours(kind, dims, periodic)
    n = len(want)
    assert len(row_ptr) == n + 1
    for i in range(n):
        got = col[row_ptr[i]:row_ptr[i + 1]].tolist()
        assert len(got) == len(set(got))
        assert set(got) == want[i], (kind, i)
        # documented fixed order
        offs = [tuple(d[i, j]) for j in got]
        if kind == "sc":
            order = {(-1, 0, 0): 0, (1, 0, 0): 1, (0, -1, 0): 2, (0, 1, 0): 3, (0, 0, -1): 4, (0, 0, 1): 5}
            keys = [order[tuple(int(round(c)) for c in o)] for o in offs]
        else:
            keys = [(o[2], o[1], o[0]) for o in offs]
        assert keys == sorted(keys)
    if periodic:
        assert (np.diff(row_ptr) == Z[kind]).all()
        assert len(col) == Z[kind] * n          # z N / 2 bonds, each listed twice


@pytest.mark.parametrize("kind,dims,periodic", CASES)
def test_neighbour_list_symmetric(orc, kind, dims, periodic):
    row_ptr, col = orc.neighbours(kind, dims, periodic)
    n = len(row_ptr) - 1
    pairs = {(i, int(j)) for i in range(n) for j in col[row_ptr[i]:row_ptr[i + 1]]}
    assert all((j, i) in pairs for i, j in pairs)


def proper(row_ptr, col, colour, mask=None):
    n = len(row_ptr) - 1
    for i in range(n):
        if mask is not None and not mask[i]:
            continue
        for j in col[row_ptr[i]:row_ptr[i + 1]]:
            if mask is not None and not mask[j]:
                continue
            if colour[i] == colour[j]:
                return False
    return True


@pytest.mark.parametrize("kind,dims,ncol", [("sc", (4, 6, 8), 2), ("bcc", (3, 5, 4), 2), ("fcc", (3, 3, 5), 4)])
def test_structured_colouring_proper(orc, kind, dims, ncol):
    g = orc.lattice(kind, dims, periodic=True)
    assert g.n_colours == ncol
    assert set(np.unique(g.colour).tolist()) == set(range(ncol))
    assert proper(g.row_ptr, g.col, g.colour)
    # equal class sizes
    counts = np.bincount(g.colour)
    assert (counts == g.n // ncol).all()


def test_sc_odd_periodic_not_two_colourable(orc):
    g = orc.lattice("sc", (5, 4, 4), periodic=True)
    assert not proper(g.row_ptr, g.col, g.colour)
    colour, nc = orc.colour_greedy(g.row_ptr, g.col)
    assert proper(g.row_ptr, g.col, colour) and nc >= 3  # greedy is not optimal


def test_greedy_colouring_bcc_sphere(orc):
    row_ptr, col, mask = inputs.bcc_nanoparticle(radius=4.0, box=10, vacancy_fraction=0.05, seed=3)
    colour, nc = orc.colour_greedy(row_ptr, col, mask)
    assert nc == 2
    assert proper(row_ptr, col, colour, mask)
    assert (colour[mask == 0] == -1).all()


def test_greedy_colouring_sc_open_and_fcc(orc):
    row_ptr, col = orc.neighbours("sc", (5, 3, 4), False)
    colour, nc = orc.colour_greedy(row_ptr, col)
    assert nc == 2 and proper(row_ptr, col, colour)
    row_ptr, col = orc.neighbours("fcc", (3, 3, 3), True)
    colour, nc = orc.colour_greedy(row_ptr, col)
    assert proper(row_ptr, col, colour) and nc >= 4


def test_nanoparticle_geometry():
    row_ptr, col, mask, pos = inputs.bcc_nanoparticle(radius=3.5, box=9, return_positions=True)
    n = len(pos)
    d = pos[None] - pos[:, None]
    d2 = (d ** 2).sum(-1)
    for i in range(n):
        want = set(np.nonzero(np.isclose(d2[i], 0.75))[0].tolist())
        assert set(col[row_ptr[i]:row_ptr[i + 1]].tolist()) == want
    c = 4.5
    assert (((pos - c) ** 2).sum(1) <= 3.5 ** 2 + 1e-12).all()
    assert mask.all()

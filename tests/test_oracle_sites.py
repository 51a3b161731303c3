"""The oracle's single-site form of Metropolis steps (ii)-(iii), used for
sampled parity checks on lattices too large for a whole oracle sweep.

Applied site by site, colour class by colour class, with the local field of
step (i) summed from the neighbour table in stored order, it must reproduce
the oracle's sweep bit for bit in every random-number schedule; the sc
neighbour list of single sites must equal the rows of the sc neighbour table.
"""
import numpy as np
import pytest

from paper_2106_11286_gb300 import inputs

PARAMS = dict(J=1.0, K=0.3, e=(0.2, -0.5, 1.0))


def _sweep_by_sites(orc, g, S, *, beta, seed, sweep_index, mode):
    S = S.copy()
    for c in range(g.n_colours):
        sites = np.nonzero(g.colour == c)[0]
        ranks = np.arange(len(sites))
        h = np.zeros((len(sites), 3))
        for t, i in enumerate(sites):   # step (i), neighbour order as stored
            for j in g.col[g.row_ptr[i]:g.row_ptr[i + 1]]:
                h[t] += S[j]
        sub = S[sites].copy()
        orc.sites_update(sites, ranks, np.full(len(sites), c), h, sub, beta=beta, seed=seed,
                         sweep_index=sweep_index, mode=mode, **PARAMS)
        S[sites] = sub
    return S


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("kind,dims", [("sc", (6, 4, 4)), ("bcc", (3, 3, 2)), ("fcc", (2, 2, 3))])
def test_site_updates_reproduce_the_sweep(orc, kind, dims, mode):
    g = orc.lattice(kind, dims)
    S0 = inputs.random_unit_spins(g.n, 31)
    if mode == 2:
        S0 = S0.astype(np.float16).astype(np.float64)
    want = S0.copy()
    orc.sweep(g, want, beta=0.8, seed=9, sweep_index=5, mode=mode, **PARAMS)
    got = _sweep_by_sites(orc, g, S0, beta=0.8, seed=9, sweep_index=5, mode=mode)
    assert np.array_equal(got, want)
    assert not np.array_equal(got, S0)


@pytest.mark.parametrize("dims,periodic", [((6, 4, 8), True), ((5, 3, 4), False), ((2, 2, 2), True)])
def test_sc_site_neighbours_match_the_table(orc, dims, periodic):
    g = orc.lattice("sc", dims, periodic)
    nb = orc.sc_site_neighbours(dims, periodic, np.arange(g.n))
    for i in range(g.n):
        row = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        assert list(nb[i][nb[i] >= 0]) == list(row)


@pytest.mark.parametrize("dims", [(6, 4, 8), (2, 6, 4), (8, 3, 5)])
def test_sc_sites_colour_rank_matches_counting(orc, dims):
    colour = orc.colour_structured("sc", dims)
    n = len(colour)
    want_rank = np.empty(n, dtype=np.int64)
    for c in (0, 1):   # rank = how many sites of the same colour come first
        want_rank[colour == c] = np.arange(int((colour == c).sum()))
    got_colour, got_rank = orc.sc_sites_colour_rank(dims, np.arange(n))
    assert np.array_equal(got_colour, colour)
    assert np.array_equal(got_rank, want_rank)


def test_init_sites_match_init_spins(orc):
    g = orc.lattice("sc", (6, 4, 8))
    S = orc.init_spins(g, seed=12, replica=3)
    idx = np.array([0, 7, 100, g.n - 1])
    assert np.array_equal(orc.init_sites(idx, seed=12, replica=3), S[idx])
    # beyond 2^32 the index's high half enters the counter: no repeat of the low half
    far = orc.init_sites(np.array([5, 5 + 2 ** 32]), seed=12, replica=3)
    assert not np.array_equal(far[0], far[1])
    assert np.allclose(np.linalg.norm(far, axis=1), 1.0, atol=1e-15)

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


@pytest.mark.parametrize("mode", [0, 1])
def test_band_flag_is_two_sided(orc, mode):
    """With J = K = 0 every dH is exactly 0, so every move is accepted through
    the dH <= 0 branch; a decision is still as close to the boundary
    P = exp(-beta dH) as |ln P|, and the flag must say so exactly when
    |ln P| < band (a one-sided flag would never set one here)."""
    m = 4000
    sites = np.arange(m, dtype=np.int64)
    ranks = np.arange(m, dtype=np.int64)
    colours = np.zeros(m, dtype=np.int32)
    h = inputs.random_unit_spins(m, 3)
    S = inputs.random_unit_spins(m, 4)
    band = 0.3
    acc, flag = orc.sites_update(sites, ranks, colours, h, S, J=0.0, K=0.0, e=(0, 0, 1), beta=1.0, seed=6,
                                 sweep_index=2, mode=mode, band=band)
    assert acc.all()
    P = np.array([orc.trial_uniforms(mode, seed=6, replica=0, site=int(i), rank=int(i), sweep_index=2,
                                     colour=0)[2] for i in sites])
    want = (P > 0) & (np.abs(np.log(np.where(P > 0, P, 1.0))) < band)
    assert np.array_equal(flag, want)
    assert 0.1 < want.mean() < 0.5   # 1 - exp(-0.3) = 0.26 of the draws


def test_band_flag_both_sides_of_zero(orc):
    """On a lattice the flag marks accepted decisions with dH on either side of
    0 whenever |beta dH + ln P| < band; with a wide band both signs occur."""
    dims = (8, 8, 8)
    S = inputs.random_unit_spins(8 * 8 * 8, 5)
    sites = np.arange(len(S))
    colour, rank = orc.sc_sites_colour_rank(dims, sites)
    h = S[orc.sc_site_neighbours(dims, True, sites)].sum(axis=1)
    new = S.copy()
    acc, flag = orc.sites_update(sites, rank, colour, h, new, beta=2.0, seed=3, sweep_index=1, mode=1,
                                 band=0.5, **PARAMS)
    # dH of the accepted moves, from Eq. 1's single-site energy of old and new spin
    ev = np.asarray(PARAMS["e"]) / np.linalg.norm(PARAMS["e"])

    def e_site(s):
        return -PARAMS["J"] * (s * h).sum(1) - PARAMS["K"] * (s @ ev) ** 2
    dH = e_site(new) - e_site(S)
    assert np.any(flag & acc & (dH <= 0)) and np.any(flag & acc & (dH > 0))


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_parallel_sweep_is_bit_identical(orc, mode, threads):
    rp, col, mask = inputs.bcc_nanoparticle(radius=4, box=10, vacancy_fraction=0.05, seed=2)
    cases = [(orc.lattice("sc", (8, 6, 4)), None), (orc.lattice("fcc", (3, 3, 2)), None),
             (orc.csr_graph(rp, col, mask), None)]
    for g, _ in cases:
        S0 = orc.init_spins(g, seed=4)
        if mode == 2:
            S0 = S0.astype(np.float16).astype(np.float64)
        a, b = S0.copy(), S0.copy()
        fa = np.zeros(g.n, dtype=np.uint8)
        fb = np.zeros(g.n, dtype=np.uint8)
        ra = orc.sweep(g, a, beta=1.1, seed=8, sweep_index=4, mode=mode, band=1e-2, band_site=fa, **PARAMS)
        rb = orc.sweep_parallel(g, b, beta=1.1, seed=8, sweep_index=4, mode=mode, band=1e-2, band_site=fb,
                                threads=threads, **PARAMS)
        assert np.array_equal(a, b)
        assert np.array_equal(fa, fb)
        assert ra[0] == rb[0] and ra[2] == rb[2]
        assert rb[1] == pytest.approx(ra[1], rel=1e-12, abs=1e-12)

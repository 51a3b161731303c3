"""Lattices beyond 2^31 sites on one GPU, checked through sampled sites.

* hs_get_sites returns exactly the spins a whole copy holds (lattice, slab).
* sc 2048^3 (8,589,934,592 spins; FP32 state 103 GB, FP16 52 GB), periodic,
  J = 1, K = 0.05, e = z, T = 1.2: the library's initial spins at sampled
  natural indices up to 2^33 equal the oracle's draw of those indices, and
  one sweep (register stencil) at 20,000 sampled sites of each colour
  follows the oracle's single-site form of steps (ii)-(iii) -- colour 0
  from the start state's neighbours, colour 1 from the neighbours the GPU's
  colour-0 pass left -- under the bars of the small-lattice parity tests.
"""
import numpy as np
import pytest

from paper_2106_11286_gb300 import hs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_get_sites_matches_whole_copies(precision):
    dims = (16, 12, 10)
    rng = np.random.default_rng(1)
    with hs.Lattice("sc", dims=dims, precision=precision, seed=4) as lat:
        lat.init()
        lat.sweep(0.8, 2)
        S = lat.get_spins()
        idx = rng.integers(0, len(S), 500)
        assert np.array_equal(lat.get_sites(idx), S[idx])
    with hs.Slab(dims, 4, 3, precision=precision, seed=4) as slab:
        slab.init()
        S = slab.get_spins()
        idx = 4 * 16 * 12 + rng.integers(0, len(S), 300)
        assert np.array_equal(slab.get_sites(idx), S[idx - 4 * 16 * 12])
        with pytest.raises(hs.HSError):
            slab.get_sites([0])   # not owned


DIMS = (2048, 2048, 2048)
PARAMS = dict(J=1.0, K=0.05, e=(0.0, 0.0, 1.0))
BAND = {"fp32": 1e-4, "fp16": 3e-2}
TOL = {"fp32": 2e-6, "fp16": 1e-3}
MODE = {"fp32": 1, "fp16": 2}
STORE = {"fp32": np.float32, "fp16": np.float16}


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_2048_sampled_sites(orc, precision):
    n = DIMS[0] * DIMS[1] * DIMS[2]
    beta, seed, sweep_index = 1 / 1.2, 9, 1
    rng = np.random.default_rng(2048)
    sites = np.unique(np.concatenate([rng.integers(0, n, 40000), [0, n - 1, 2 ** 32 - 1, 2 ** 32, 2 ** 32 + 1]]))
    colour, rank = orc.sc_sites_colour_rank(DIMS, sites)
    nb = orc.sc_site_neighbours(DIMS, True, sites)
    with hs.Lattice("sc", dims=DIMS, precision=precision, seed=seed, **PARAMS) as lat:
        lat.init()
        lat.set_sweep_counter(sweep_index)
        S0 = lat.get_sites(sites)
        N0 = lat.get_sites(nb.ravel()).reshape(len(sites), 6, 3)
        lat.sweep(beta, 1)
        S1 = lat.get_sites(sites)
        N1 = lat.get_sites(nb.ravel()).reshape(len(sites), 6, 3)
    # initial spins: the oracle's draw of each natural index, rounded to storage
    want0 = orc.init_sites(sites, seed=seed).astype(STORE[precision]).astype(np.float64)
    assert np.abs(S0 - want0).max() <= TOL[precision]
    for c in (0, 1):
        sel = colour == c
        src = N0 if c == 0 else N1   # the neighbours are of the other colour
        h = np.zeros((int(sel.sum()), 3))
        for k in range(6):           # step (i), order -x, +x, -y, +y, -z, +z
            h += src[sel, k]
        want = S0[sel].copy()
        acc, band = orc.sites_update(sites[sel], rank[sel], colour[sel], h, want, beta=beta, seed=seed,
                                     sweep_index=sweep_index, mode=MODE[precision], band=BAND[precision], **PARAMS)
        got = S1[sel]
        acc_gpu = np.any(got != S0[sel], axis=1)
        assert 0.1 < acc.mean() < 0.9
        assert int(np.sum((acc_gpu != acc) & ~band)) == 0, (precision, c)
        both = acc & acc_gpu
        assert np.abs(got[both] - want[both]).max() <= TOL[precision]
        rej = ~acc & ~acc_gpu
        assert np.array_equal(got[rej], S0[sel][rej])

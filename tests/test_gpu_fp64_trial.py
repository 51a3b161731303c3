"""The FP64 trial orientation's sine and cosine (table lookup + angle
addition + Taylor series, not the CUDA library's sincospi) against the
oracle's C library sin/cos: after one FP64 sweep from the same state, every
accepted spin (the trial itself) equals the oracle's within 2e-15, over
hundreds of thousands of trials -- a few units in the last place, where the
parity bar allows 1e-12.  |S| = 1 holds to 1e-15.
"""
import numpy as np
import pytest

from helpers import oracle_graph
from paper_2106_11286_gb300 import hs, inputs

pytestmark = pytest.mark.gpu

PARAMS = dict(J=1.0, K=0.1, e=(0.0, 0.0, 1.0))


@pytest.mark.parametrize("kind,dims", [("sc", (64, 64, 64)), ("bcc", (24, 24, 24))])
def test_fp64_trials_match_the_oracle_to_ulps(orc, kind, dims):
    g = oracle_graph(orc, kind, dims)
    S0 = inputs.random_unit_spins(g.n, 21)
    with hs.Lattice(kind, dims=dims, precision="fp64", seed=13, **PARAMS) as lat:
        lat.set_spins(S0)
        lat.set_sweep_counter(4)
        lat.sweep(0.3, 1)  # hot: most moves accepted
        got = lat.get_spins()
    want = S0.copy()
    band = np.zeros(g.n, dtype=np.uint8)
    orc.sweep(g, want, beta=0.3, seed=13, sweep_index=4, mode=0, band=1e-9, band_site=band, **PARAMS)
    acc_g = np.any(got != S0, axis=1)
    acc_o = np.any(want != S0, axis=1)
    same = acc_g == acc_o
    assert (~same).sum() <= band.sum()
    both = same & acc_o
    assert both.sum() > 0.5 * g.n
    assert np.abs(got[both] - want[both]).max() < 2e-15
    assert np.abs(np.linalg.norm(got, axis=1) - 1).max() < 1e-15

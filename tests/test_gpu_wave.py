"""The wavefront kernel (many colour passes in one persistent launch, passes
following each other plane by plane) against the register stencil and the
oracle: spins bit-identical to the stencil after many sweeps in every tested
configuration (unit size, passes per group, lag, partial last group, several
launches), accepted moves equal, E and M sums equal to FP32 rounding, and one
sweep element by element against the oracle.
"""
import numpy as np
import pytest

from helpers import check_sweep_parity, oracle_graph
from paper_2106_11286_gb300 import hs, inputs

pytestmark = pytest.mark.gpu

PARAMS = dict(J=1.0, K=0.1, e=(0.2, -0.3, 1.0))


def _run(dims, precision, sweeps, launch, seed=3, beta=0.9):
    with hs.Lattice("sc", dims=dims, precision=precision, seed=seed, **PARAMS) as lat:
        if launch is not None:
            lat.set_launch(**launch)
        lat.init()
        lat.accumulate(True)
        lat.sweep(beta, sweeps)
        mom, count = lat.read_accumulator()
        return lat.get_spins(), mom, count, lat.measure()["accept_rate"], lat.launch


@pytest.mark.parametrize("precision,dims", [("fp32", (16, 16, 16)), ("fp32", (24, 8, 12)), ("fp32", (64, 32, 6)),
                                            ("fp16", (32, 16, 10))])
@pytest.mark.parametrize("cfg", [dict(), dict(tile_y=1), dict(tile_y=4, chunk_z=3, ring=3),
                                 dict(chunk_z=1), dict(chunk_z=5, ring=7), dict(tile_y=1, chunk_z=32, ring=4)])
def test_wave_matches_stencil(precision, dims, cfg):
    sweeps = 7  # 14 passes: full groups and a partial last one for most chunk sizes
    want, mom_w, cnt_w, acc_w, _ = _run(dims, precision, sweeps, dict(kernel="stencil"))
    got, mom_g, cnt_g, acc_g, launch = _run(dims, precision, sweeps, dict(kernel="wave", **cfg))
    assert launch["kernel"] == hs.KERNELS["wave"]
    assert np.array_equal(got, want)
    assert cnt_g == cnt_w == sweeps
    assert acc_g == acc_w
    np.testing.assert_allclose(mom_g, mom_w, rtol=2e-5, atol=1e-6 * np.prod(dims))


def test_wave_several_launches_and_single_passes():
    dims = (16, 16, 8)
    want, _, _, _, _ = _run(dims, "fp32", 300, dict(kernel="stencil"))
    got, _, cnt, _, _ = _run(dims, "fp32", 300, dict(kernel="wave"))  # 600 passes: two launches
    assert cnt == 300
    assert np.array_equal(got, want)
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=3, **PARAMS) as a, \
            hs.Lattice("sc", dims=dims, precision="fp32", seed=3, **PARAMS) as b:
        a.set_launch(kernel="wave")
        for lat in (a, b):
            lat.init()
            hs.hs_sweep_pass(lat.h, 1.0, 0)
            hs.hs_sweep_pass(lat.h, 1.0, 1)
        assert np.array_equal(a.get_spins(), b.get_spins())


def test_wave_one_sweep_against_oracle(orc):
    dims = (16, 16, 16)
    g = oracle_graph(orc, "sc", dims)
    S0 = inputs.random_unit_spins(g.n, 8).astype(np.float32).astype(np.float64)
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=4, **PARAMS) as lat:
        lat.set_launch(kernel="wave")
        lat.set_spins(S0)
        lat.set_sweep_counter(5)
        lat.sweep(1.0, 1)
        got = lat.get_spins()
    want = S0.copy()
    band = np.zeros(g.n, dtype=np.uint8)
    orc.sweep(g, want, beta=1.0, seed=4, sweep_index=5, mode=1, band=1e-4, band_site=band, **PARAMS)
    assert check_sweep_parity(g, S0, got, want, band, 2e-6) <= max(2, g.n // 200)


def test_wave_launch_rules():
    with hs.Lattice("sc", dims=(16, 16, 16), precision="fp64", seed=1, **PARAMS) as lat:
        with pytest.raises(hs.HSError):
            lat.set_launch(kernel="wave")
    with hs.Lattice("sc", dims=(16, 16, 16), precision="fp32", seed=1, **PARAMS) as lat:
        for bad in (dict(tile_y=9), dict(ring=2), dict(chunk_z=33), dict(vec_width=2)):
            with pytest.raises(hs.HSError):
                lat.set_launch(kernel="wave", **bad)
        lat.set_launch(kernel="wave")
        lat.set_anisotropy_tensor(np.eye(3))  # back to the automatic launch, which takes the term
        assert lat.launch["kernel"] == hs.KERNELS["stencil"]
        with pytest.raises(hs.HSError):
            lat.set_launch(kernel="wave")
    with hs.Slab((16, 16, 16), 0, 8, precision="fp32") as s:
        with pytest.raises(hs.HSError):
            s.set_launch(kernel="wave")

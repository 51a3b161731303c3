"""The on-site anisotropy tensor term -sum_i S_i^T A S_i on the GPU against the
oracle (same bar as the plain parity tests: FP64 decisions identical outside
the 1e-9 band and spins within 1e-12; FP32 / FP16 decisions may differ only
inside their rounding bands), for the register stencil and the neighbour
table, plus the fused per-sweep energy, hs_measure and the launch rules.
"""
import numpy as np
import pytest

from helpers import check_sweep_parity, make_gpu, oracle_graph
from paper_2106_11286_gb300 import hs
from test_gpu_parity import BAND, CASES, MODE, TOL, _run_one_sweep

pytestmark = pytest.mark.gpu

# a tensor with large off-diagonal entries and a trace part
A_TENSOR = np.array([[0.15, 0.30, -0.10],
                     [0.30, -0.20, 0.25],
                     [-0.10, 0.25, 0.05]])
PARAMS_T = dict(J=1.0, K=0.1, e=(0.0, 0.0, 1.0), A=A_TENSOR)
PARAMS_O = dict(J=1.0, K=0.1, e=(0.0, 0.0, 1.0))


@pytest.mark.parametrize("name", ["sc16", "sc_12x8x6", "sc_10x6x4", "sc_2x4x6", "sc_open_5x4x3", "sc_masked",
                                  "bcc_4", "fcc_3", "bcc_sphere"])
def test_fp64_tensor_sweep(orc, name):
    g, S0, S_gpu, S_orc, band, meas, acc = _run_one_sweep(orc, CASES[name], "fp64", beta=1.0, seed=4,
                                                         sweep_index=6, params=PARAMS_T)
    mism = check_sweep_parity(g, S0, S_gpu, S_orc, band, TOL["fp64"])
    assert mism == int(band.sum() > 0) * mism
    assert 0 < acc < g.n_present
    want = orc.measure(g, S_orc, **PARAMS_T)
    assert meas["E"] == pytest.approx(want["E"], rel=1e-10, abs=1e-9)
    # the term matters: without it the oracle's energy is another number
    assert abs(orc.energy(g, S_orc, **PARAMS_O) - want["E"]) > 1e-3 * g.n_present


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("name", ["sc16", "sc_12x8x6", "sc_10x6x4", "fcc_3", "bcc_sphere"])
def test_reduced_precision_tensor_sweep(orc, name, precision):
    g, S0, S_gpu, S_orc, band, meas, acc = _run_one_sweep(orc, CASES[name], precision, beta=1.0, seed=5,
                                                         sweep_index=9, params=PARAMS_T)
    mism = check_sweep_parity(g, S0, S_gpu, S_orc, band, TOL[precision])
    assert mism <= max(2, g.n_present // 200)
    want = orc.measure(g, S_gpu, **PARAMS_T)
    assert meas["E"] == pytest.approx(want["E"], rel=1e-9, abs=1e-8)


@pytest.mark.parametrize("precision,rel", [("fp64", 1e-10), ("fp32", 2e-5), ("fp16", 2e-5)])
@pytest.mark.parametrize("kind,dims", [("sc", (16, 16, 16)), ("fcc", (4, 4, 4))])
def test_fused_energy_with_tensor(orc, precision, rel, kind, dims):
    """E accumulated inside the colour passes equals the full recompute of
    the state the sweep left."""
    g = oracle_graph(orc, kind, dims)
    with make_gpu(kind, dims, precision=precision, seed=3, **PARAMS_T) as lat:
        lat.init()
        lat.accumulate(True)
        lat.sweep(0.8, 3)
        mom, count = lat.read_accumulator()
        S = lat.get_spins()
        last = hs.hs_read_sums(lat.h)
    assert count == 3
    want = orc.energy(g, S, **PARAMS_T)
    assert last[0] == pytest.approx(want, rel=rel, abs=rel * g.n)


def test_fp64_tensor_multi_sweep(orc):
    g = oracle_graph(orc, "sc", (16, 16, 16))
    with make_gpu("sc", (16, 16, 16), precision="fp64", seed=2, **PARAMS_T) as lat:
        lat.init()
        S = lat.get_spins()
        bands = 0
        for s in range(8):
            _, _, nb = orc.sweep(g, S, beta=1.2, seed=2, sweep_index=s, band=1e-9, **PARAMS_T)
            bands += nb
        lat.sweep(1.2, 8)
        got = lat.get_spins()
    assert bands == 0
    np.testing.assert_allclose(got, S, atol=1e-12, rtol=0)


def test_tensor_launch_rules():
    with hs.Lattice("sc", dims=(16, 16, 16), precision="fp32", seed=1, **PARAMS_O) as lat:
        auto = lat.launch
        lat.set_anisotropy_tensor(A_TENSOR)
        np.testing.assert_array_equal(hs.hs_get_anisotropy_tensor(lat.h),
                                      [0.15, -0.20, 0.05, 0.30, -0.10, 0.25])
        L = lat.launch
        assert L["kernel"] == hs.KERNELS["stencil"] and L["prefetch"] == 2
        for bad in (dict(kernel="pipe"), dict(kernel="march"), dict(kernel=2), dict(kernel=6),
                    dict(kernel="stencil", prefetch=3)):
            with pytest.raises(hs.HSError):
                lat.set_launch(**bad)
        with pytest.raises(hs.HSError):
            hs.hs_batch_create([lat.h])
        with pytest.raises(hs.HSError):
            hs.hs_set_anisotropy_tensor(lat.h, [0, 0, 0, np.inf, 0, 0])
        lat.set_anisotropy_tensor(None)
        assert not hs.hs_get_anisotropy_tensor(lat.h).any()
        assert lat.launch == auto
    with pytest.raises(ValueError):
        hs.tensor_entries(np.arange(9.0).reshape(3, 3))


def test_tensor_slab_matches_whole(orc):
    """A z-slab carries the term too: two slabs with halo exchange equal the
    whole lattice."""
    from paper_2106_11286_gb300 import inputs, shards
    dims = (8, 6, 8)
    S0 = inputs.random_unit_spins(8 * 6 * 8, 3).astype(np.float32).astype(np.float64)
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=6, **PARAMS_T) as whole:
        whole.set_spins(S0)
        whole.sweep(1.0, 2)
        want = whole.get_spins()
    with shards.ShardedLattice(dims, 2, precision="fp32", seed=6, **PARAMS_O) as sh:
        for s in sh.slabs:
            s.set_anisotropy_tensor(A_TENSOR)
        sh.set_spins(S0)
        sh.sweep(1.0, 2)
        assert np.array_equal(sh.get_spins(), want)

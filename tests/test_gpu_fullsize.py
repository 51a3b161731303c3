"""Full-size parity: the sc 256^3 throughput workload (16,777,216 spins,
periodic, J = 1, K = 0.05, e = z, T = 1.2), one sweep on the GPU against the
oracle's sweep of the whole lattice, element by element.

The GPU runs in the launch configuration the autotuner picks for this
lattice (the configuration the throughput measurement times) and in each sc
kernel kind; every one must reproduce the oracle's sweep from the same state,
sweep counter and keys under the bar of the small-lattice parity tests.
"""
import numpy as np
import pytest

from helpers import check_sweep_parity, storage_round
from paper_2106_11286_gb300 import hs, inputs

pytestmark = pytest.mark.gpu

DIMS = (256, 256, 256)
PARAMS = dict(J=1.0, K=0.05, e=(0.0, 0.0, 1.0))
BETA = 1.0 / 1.2
SEED = 2
SWEEP = 7
MODE = {"fp64": 0, "fp32": 1}
BAND = {"fp64": 1e-9, "fp32": 1e-4}
TOL = {"fp64": 1e-12, "fp32": 2e-6}


@pytest.fixture(scope="module")
def graph(orc):
    return orc.lattice("sc", DIMS)


@pytest.fixture(scope="module")
def reference(orc, graph):
    """Oracle sweep of the full lattice, per precision's random-number schedule."""
    out = {}
    S0 = inputs.random_unit_spins(graph.n, 21)
    for precision in ("fp32", "fp64"):
        start = storage_round(S0, precision)
        S = start.copy()
        band = np.zeros(graph.n, dtype=np.uint8)
        acc, _, _ = orc.sweep(graph, S, beta=BETA, seed=SEED, sweep_index=SWEEP, mode=MODE[precision],
                              band=BAND[precision], band_site=band, **PARAMS)
        out[precision] = (start, S, band, acc)
    return out


def _gpu_sweep(precision, start, launch):
    with hs.Lattice("sc", dims=DIMS, precision=precision, seed=SEED, **PARAMS) as lat:
        if launch == "autotuned":
            lat.init()
            lat.autotune(BETA, 2)
        elif launch is not None:
            lat.set_launch(**launch)
        lat.set_spins(start)
        lat.set_sweep_counter(SWEEP)
        lat.sweep(BETA, 1)
        return lat.get_spins(), lat.measure(), lat.launch


FP32_LAUNCHES = {
    "autotuned": "autotuned",
    "stencil": dict(kernel="stencil", vec_width=4),
    "stencil_prefetch": dict(kernel="stencil", vec_width=4, prefetch=1),
    "pipe": dict(kernel="pipe", vec_width=4),
    "march": dict(kernel="march", vec_width=4),
    "staged": dict(kernel="staged", vec_width=4),
}


@pytest.mark.parametrize("name", list(FP32_LAUNCHES))
def test_fp32_full_lattice_sweep(orc, graph, reference, name):
    start, want, band, acc = reference["fp32"]
    got, meas, launch = _gpu_sweep("fp32", start, FP32_LAUNCHES[name])
    if name != "autotuned":
        assert launch["kernel"] == hs.KERNELS[FP32_LAUNCHES[name]["kernel"]]
    mism = check_sweep_parity(graph, start, got, want, band, TOL["fp32"])
    assert mism <= max(2, graph.n // 100000)
    assert meas["accept_rate"] == pytest.approx(acc / graph.n, abs=(mism + 1) / graph.n)
    ref = orc.measure(graph, got, **PARAMS)
    assert meas["E"] == pytest.approx(ref["E"], rel=1e-9)
    np.testing.assert_allclose(meas["M"], ref["M"], atol=1e-6)


@pytest.mark.parametrize("launch", [None, dict(kernel="pipe", vec_width=2)], ids=["default", "pipe"])
def test_fp64_full_lattice_sweep(orc, graph, reference, launch):
    start, want, band, acc = reference["fp64"]
    got, meas, _ = _gpu_sweep("fp64", start, launch)
    mism = check_sweep_parity(graph, start, got, want, band, TOL["fp64"])
    assert mism == int(band.sum() > 0) * mism
    ref = orc.measure(graph, want, **PARAMS)
    assert meas["E"] == pytest.approx(ref["E"], rel=1e-10)

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
    "stencil_split": dict(kernel="stencil", vec_width=4, prefetch=3),
    "pipe": dict(kernel="pipe", vec_width=4),
    "march": dict(kernel="march", vec_width=4),
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


# ---------------------------------------------------------------- sc 464^3 precision ladder (sampled sites)
# sc 464^3 (99,897,344 spins), periodic, J = 1, K = 0.1, e = z, T = 1.0, the
# library's seeded random start; one sweep in the autotuned launch of each
# precision.  A whole oracle sweep of 10^8 sites is out of reach here, so
# 20,000 sites of each colour are checked one by one: a colour-0 site from the
# start state's neighbours, a colour-1 site from the neighbours the GPU's
# colour-0 pass left (its own inputs), each through the oracle's single-site
# form of steps (ii)-(iii).
DIMS464 = (464, 464, 464)
PARAMS464 = dict(J=1.0, K=0.1, e=(0.0, 0.0, 1.0))
MODE3 = {"fp64": 0, "fp32": 1, "fp16": 2}
BAND3 = {"fp64": 1e-9, "fp32": 1e-4, "fp16": 3e-2}
TOL3 = {"fp64": 1e-12, "fp32": 2e-6, "fp16": 1e-3}


@pytest.fixture(scope="module")
def colour464(orc):
    colour = orc.colour_structured("sc", DIMS464)
    ranks = np.empty(colour.shape, dtype=np.int64)
    for c in (0, 1):   # rank of a site among the sites of its colour, ascending natural index
        sel = colour == c
        ranks[sel] = np.arange(int(sel.sum()))
    return colour, ranks


@pytest.mark.parametrize("precision,launch", [("fp64", None), ("fp32", None), ("fp16", None),
                                             ("fp32", dict(kernel="stencil", vec_width=4, prefetch=3))],
                         ids=["fp64", "fp32", "fp16", "fp32-split"])
def test_464_sampled_sites(orc, colour464, precision, launch):
    colour, ranks = colour464
    beta, seed, sweep_index = 1.0, 5, 3
    with hs.Lattice("sc", dims=DIMS464, precision=precision, seed=seed, **PARAMS464) as lat:
        lat.init()
        if launch is None:
            lat.autotune(beta, 2)
        else:
            lat.set_launch(**launch)
        lat.set_sweep_counter(sweep_index)
        S0 = lat.get_spins()
        lat.sweep(beta, 1)
        S1 = lat.get_spins()
    rng = np.random.default_rng(464)
    for c in (0, 1):
        sites = rng.choice(np.nonzero(colour == c)[0], 20000, replace=False)
        nb = orc.sc_site_neighbours(DIMS464, True, sites)
        src = S0 if c == 0 else S1   # the neighbours are of the other colour
        h = np.zeros((len(sites), 3))
        for k in range(6):            # step (i), order -x, +x, -y, +y, -z, +z
            h += src[nb[:, k]]
        want = S0[sites].copy()
        acc, band = orc.sites_update(sites, ranks[sites], np.full(len(sites), c), h, want, beta=beta, seed=seed,
                                     sweep_index=sweep_index, mode=MODE3[precision], band=BAND3[precision],
                                     **PARAMS464)
        got = S1[sites]
        acc_gpu = np.any(got != S0[sites], axis=1)
        assert 0.1 < acc.mean() < 0.9
        # decisions differ only inside the band, which the oracle flags on
        # either side of dH = 0
        unexplained = int(np.sum((acc_gpu != acc) & ~band))
        assert unexplained == 0, (precision, c, unexplained)
        both = acc & acc_gpu
        assert np.abs(got[both] - want[both]).max() <= TOL3[precision]
        rej = ~acc & ~acc_gpu
        assert np.array_equal(got[rej], S0[sites][rej])


# ---------------------------------------------------------------- bcc nanoparticle (whole lattice)
# Sphere of radius 110 cut from a 232^3-cell bcc crystal, open surface, 1 %
# vacancies (seed 3), CSR neighbour list, J = 1, K = 0.2, e = (1,1,1)/sqrt 3,
# T = 0.9, FP32: one sweep of all 11,039,109 spins in the autotuned launch
# against the oracle's sweep of the same neighbour list.
def test_bcc_nanoparticle_full_sweep(orc):
    rp, col, mask = inputs.bcc_nanoparticle(radius=110, box=232, vacancy_fraction=0.01, seed=3)
    params = dict(J=1.0, K=0.2, e=(1.0, 1.0, 1.0))
    beta, seed, sweep_index = 1 / 0.9, 3, 2
    with hs.Lattice("csr", row_ptr=rp, col_idx=col, site_mask=mask, precision="fp32", seed=seed, **params) as lat:
        lat.init()
        lat.autotune(beta, 2)
        lat.set_sweep_counter(sweep_index)
        S0 = lat.get_spins()
        lat.sweep(beta, 1)
        S1 = lat.get_spins()
        meas = lat.measure()
    g = orc.csr_graph(rp, col, mask)
    assert g.n_present == 11039109
    want = S0.copy()
    band = np.zeros(g.n, dtype=np.uint8)
    acc, _, _ = orc.sweep(g, want, beta=beta, seed=seed, sweep_index=sweep_index, mode=1, band=1e-4,
                          band_site=band, **params)
    mism = check_sweep_parity(g, S0, S1, want, band, 2e-6)
    assert mism <= max(2, g.n_present // 100000)
    ref = orc.measure(g, S1, **params)
    assert meas["E"] == pytest.approx(ref["E"], rel=1e-9)


# ---------------------------------------------------------------- batched replicas (every member)
# 64 sc replicas, L = (16, 24, 32, 48, 64, 96)[r mod 6], periodic, K = 0,
# T_r = 1.30 + 0.30 r / 63, FP32: one sweep of the persistent batched kernel
# from the library's seeded start; every member against the oracle's sweep.
def test_batched_replicas_full_sweep(orc):
    sizes = (16, 24, 32, 48, 64, 96)
    betas = [1.0 / (1.30 + 0.30 * r / 63) for r in range(64)]
    lats = [hs.Lattice("sc", dims=(sizes[r % 6],) * 3, J=1.0, K=0.0, precision="fp32", seed=4, replica=r)
            for r in range(64)]
    try:
        for m in lats:
            m.init()
        S0 = [m.get_spins() for m in lats]
        batch = hs.hs_batch_create([m.h for m in lats])
        try:
            hs.hs_batch_run(batch, betas, 1, 0)
        finally:
            hs.hs_batch_destroy(batch)
        S1 = [m.get_spins() for m in lats]
    finally:
        for m in lats:
            m.close()
    graphs = {L: orc.lattice("sc", (L, L, L)) for L in sizes}
    for r in range(64):
        g = graphs[sizes[r % 6]]
        want = S0[r].copy()
        band = np.zeros(g.n, dtype=np.uint8)
        orc.sweep(g, want, J=1.0, K=0.0, e=(0.0, 0.0, 1.0), beta=betas[r], seed=4, replica=r, sweep_index=0,
                  mode=1, band=1e-4, band_site=band)
        mism = check_sweep_parity(g, S0[r], S1[r], want, band, 2e-6)
        assert mism <= 2, r

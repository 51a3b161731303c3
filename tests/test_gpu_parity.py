"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Bar (FP64 path): accept decisions identical except where the oracle flags
|beta dH + ln P| < 1e-9 (floating-point rounding order can decide those),
accepted spins within 1e-12, rejected spins bit-equal, E and M within 1e-10
relative.  FP32 / FP16 paths: the oracle runs the same random-number schedule
on the storage-rounded state; decisions may differ only inside a band derived
from the FP32 error of beta dH + ln P (1e-4) or of the binary16 trial
rounding (3e-2), spins within 2e-6 (FP32) or one binary16 step (FP16).
"""
import numpy as np
import pytest

from helpers import check_sweep_parity, make_gpu, oracle_graph, storage_round
from paper_2106_11286_gb300 import hs, inputs

pytestmark = pytest.mark.gpu

MODE = {"fp64": 0, "fp32": 1, "fp16": 2}
BAND = {"fp64": 1e-9, "fp32": 1e-4, "fp16": 3e-2}
TOL = {"fp64": 1e-12, "fp32": 2e-6, "fp16": 1e-3}


def _bcc_sphere():
    rp, col, mask = inputs.bcc_nanoparticle(radius=4.3, box=10, vacancy_fraction=0.05, seed=3)
    return dict(kind="csr", row_ptr=rp, col=col, mask=mask)


CASES = {
    "sc16": dict(kind="sc", dims=(16, 16, 16)),
    "sc_12x8x6": dict(kind="sc", dims=(12, 8, 6)),          # Lx/2 = 6: FP32 vector width 2
    "sc_10x6x4": dict(kind="sc", dims=(10, 6, 4)),          # Lx/2 = 5: scalar stencil path
    "sc_2x4x6": dict(kind="sc", dims=(2, 4, 6)),            # L = 2: +x and -x coincide
    "sc_open_5x4x3": dict(kind="sc", dims=(5, 4, 3), periodic=False),
    "sc_masked": dict(kind="sc", dims=(8, 8, 8), mask=inputs.vacancy_mask(512, 0.1, 7)),
    "bcc_4": dict(kind="bcc", dims=(4, 4, 4)),
    "bcc_open_3x4x5": dict(kind="bcc", dims=(3, 4, 5), periodic=False),
    "fcc_3": dict(kind="fcc", dims=(3, 3, 3)),
    "fcc_open_2x3x4": dict(kind="fcc", dims=(2, 3, 4), periodic=False),
    "bcc_sphere": _bcc_sphere(),
}

PARAMS = dict(J=1.0, K=0.1, e=(0.0, 0.0, 1.0))


def _run_one_sweep(orc, case, precision, *, beta, seed, sweep_index, params=PARAMS, state_seed=5):
    g = oracle_graph(orc, case["kind"], case.get("dims"), case.get("periodic", True), case.get("row_ptr"),
                     case.get("col"), case.get("mask"))
    S0 = inputs.random_unit_spins(g.n, state_seed)
    if g.mask is not None:
        S0[g.mask == 0] = 0.0
    S0 = storage_round(S0, precision)
    with make_gpu(case["kind"], case.get("dims"), case.get("periodic", True), case.get("row_ptr"), case.get("col"),
                  case.get("mask"), precision=precision, seed=seed, **params) as lat:
        lat.set_spins(S0)
        assert np.array_equal(lat.get_spins(), S0)
        lat.set_sweep_counter(sweep_index)
        lat.sweep(beta, 1)
        S_gpu = lat.get_spins()
        meas = lat.measure()
    S_orc = S0.copy()
    band = np.zeros(g.n, dtype=np.uint8)
    acc, _, nb = orc.sweep(g, S_orc, beta=beta, seed=seed, sweep_index=sweep_index, mode=MODE[precision],
                           band=BAND[precision], band_site=band, **params)
    return g, S0, S_gpu, S_orc, band, meas, acc


# an easy axis that is not a coordinate axis: the general S.e products (the
# e = (0, 0, 1) cases above take S.e = S_z)
TILTED = dict(J=1.0, K=0.3, e=(0.3, -0.2, 1.0))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("name", ["sc16", "sc_12x8x6", "sc_10x6x4", "sc_masked"])
def test_tilted_easy_axis_single_sweep(orc, name, precision):
    g, S0, S_gpu, S_orc, band, meas, acc = _run_one_sweep(orc, CASES[name], precision, beta=1.0, seed=3,
                                                         sweep_index=7, params=TILTED)
    mism = check_sweep_parity(g, S0, S_gpu, S_orc, band, TOL[precision])
    if precision == "fp64":
        assert mism == int(band.sum() > 0) * mism
    else:
        assert mism <= max(2, g.n_present // 200)
    assert 0 < acc < g.n_present
    want = orc.measure(g, S_gpu, **TILTED)
    assert meas["E"] == pytest.approx(want["E"], rel=1e-9, abs=1e-8)


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_single_sweep(orc, name):
    g, S0, S_gpu, S_orc, band, meas, acc = _run_one_sweep(orc, CASES[name], "fp64", beta=1.0, seed=1,
                                                         sweep_index=3)
    mism = check_sweep_parity(g, S0, S_gpu, S_orc, band, TOL["fp64"])
    assert mism == int(band.sum() > 0) * mism  # mismatches only where the band fired
    assert 0 < acc < g.n_present
    assert meas["accept_rate"] == pytest.approx(acc / g.n_present, abs=mism / g.n_present + 1e-12)
    want = orc.measure(g, S_orc, **PARAMS)
    assert meas["n_sites"] == g.n_present
    assert meas["E"] == pytest.approx(want["E"], rel=1e-10, abs=1e-9)
    np.testing.assert_allclose(meas["M"], want["M"], atol=1e-12)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("name", ["sc16", "sc_12x8x6", "sc_10x6x4", "sc_masked", "fcc_3", "bcc_sphere"])
def test_reduced_precision_single_sweep(orc, name, precision):
    g, S0, S_gpu, S_orc, band, meas, acc = _run_one_sweep(orc, CASES[name], precision, beta=1.0, seed=2,
                                                         sweep_index=11)
    if precision == "fp16":
        # the stored state is binary16 on the GPU; compare the oracle's trial
        # rounded the same way (it rounds the FP64 trial, the GPU the FP32 one)
        assert np.array_equal(S_gpu.astype(np.float16).astype(np.float64), S_gpu)
    mism = check_sweep_parity(g, S0, S_gpu, S_orc, band, TOL[precision])
    assert mism <= max(2, g.n_present // 200)
    want = orc.measure(g, S_gpu, **PARAMS)
    assert meas["E"] == pytest.approx(want["E"], rel=1e-9, abs=1e-8)


def test_fp64_multi_sweep_and_resume(orc):
    """Ten sweeps from the library's own random start; then a checkpointed
    copy (spins + sweep counter) continues bit for bit."""
    case = CASES["sc16"]
    g = oracle_graph(orc, "sc", case["dims"])
    beta = 1.0
    with make_gpu("sc", case["dims"], precision="fp64", seed=1, **PARAMS) as lat:
        lat.init()
        S_init = lat.get_spins()
        S_orc = orc.init_spins(g, seed=1)
        np.testing.assert_allclose(S_init, S_orc, atol=1e-15, rtol=0)
        S_orc = S_init.copy()
        bands = 0
        for s in range(10):
            _, _, nb = orc.sweep(g, S_orc, beta=beta, seed=1, sweep_index=s, band=1e-9, **PARAMS)
            bands += nb
        lat.sweep(beta, 10)
        S10 = lat.get_spins()
        assert bands == 0
        np.testing.assert_allclose(S10, S_orc, atol=1e-12, rtol=0)
        assert lat.info.sweep == 10
        lat.sweep(beta, 7)
        S17 = lat.get_spins()
    with make_gpu("sc", case["dims"], precision="fp64", seed=1, **PARAMS) as lat2:
        lat2.set_spins(S10)
        lat2.set_sweep_counter(10)
        lat2.sweep(beta, 7)
        assert np.array_equal(lat2.get_spins(), S17)


@pytest.mark.parametrize("kind,dims,mask", [("sc", (8, 6, 4), None), ("fcc", (2, 2, 3), None),
                                            ("bcc", (3, 3, 3), inputs.vacancy_mask(54, 0.2, 1))])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_init_matches_oracle(orc, kind, dims, mask, precision):
    g = orc.lattice(kind, dims, True, mask)
    want = storage_round(orc.init_spins(g, seed=9, replica=4), precision)
    with hs.Lattice(kind, dims=dims, site_mask=mask, precision=precision, seed=9, replica=4) as lat:
        lat.init()
        got = lat.get_spins()
    tol = {"fp64": 1e-15, "fp32": 0.0, "fp16": 0.0}[precision]
    if precision == "fp64":
        np.testing.assert_allclose(got, want, atol=tol, rtol=0)
    else:  # FP64 init rounded once: equal unless the FP64 values straddle a rounding boundary
        diff = np.abs(got - want)
        ulp = 2.0 ** -23 if precision == "fp32" else 2.0 ** -10
        assert (diff <= ulp).all() and (diff > 0).mean() < 1e-3


@pytest.mark.parametrize("params", [PARAMS, TILTED], ids=["z_axis", "tilted_axis"])
def test_accumulator_matches_oracle(orc, params):
    """Fused per-sweep moments (E split at the later colour, FP64 totals)
    equal the oracle's full recompute after each sweep."""
    dims = (8, 8, 8)
    g = orc.lattice("sc", dims)
    beta = 0.8
    with make_gpu("sc", dims, precision="fp64", seed=4, **params) as lat:
        lat.init()
        S = lat.get_spins()
        lat.accumulate(True)
        lat.reset_accumulator()
        lat.sweep(beta, 5)
        mom, count = lat.read_accumulator()
    assert count == 5
    want = np.zeros(9)
    for s in range(5):
        orc.sweep(g, S, beta=beta, seed=4, sweep_index=s, **params)
        m = orc.measure(g, S, **params)
        want += [m["E"], m["E"] ** 2, m["absM"], m["M2"], m["M4"], *m["M"], m["absMe"]]
    np.testing.assert_allclose(mom, want, rtol=1e-10, atol=1e-10)


def test_ring_fold_over_many_sweeps(orc):
    """More sweeps than one ring fold takes (64): the fused moments equal the
    oracle's per-sweep recompute, and the same chain cut into calls at other
    points (so the folds group other sweeps) gives bit-identical moments."""
    dims = (8, 8, 8)
    g = orc.lattice("sc", dims)
    beta, n = 0.8, 139
    with make_gpu("sc", dims, precision="fp64", seed=4, **PARAMS) as lat:
        lat.init()
        S = lat.get_spins()
        lat.accumulate(True)
        lat.reset_accumulator()
        lat.sweep(beta, n)
        mom, count = lat.read_accumulator()
        last = hs.hs_read_sums(lat.h)
    with make_gpu("sc", dims, precision="fp64", seed=4, **PARAMS) as lat:
        lat.init()
        lat.accumulate(True)
        lat.reset_accumulator()
        for k in (1, 63, 64, 11):
            lat.sweep(beta, k)
        mom2, count2 = lat.read_accumulator()
        last2 = hs.hs_read_sums(lat.h)
    assert count == count2 == n
    np.testing.assert_array_equal(mom2, mom)
    np.testing.assert_array_equal(last2, last)
    want = np.zeros(9)
    for s in range(n):
        orc.sweep(g, S, beta=beta, seed=4, sweep_index=s, **PARAMS)
        m = orc.measure(g, S, **PARAMS)
        want += [m["E"], m["E"] ** 2, m["absM"], m["M2"], m["M4"], *m["M"], m["absMe"]]
    np.testing.assert_allclose(mom, want, rtol=1e-9, atol=1e-9)
    assert last[0] == pytest.approx(m["E"], rel=1e-10, abs=1e-9)


def test_table_path_accumulator(orc):
    case = CASES["bcc_sphere"]
    g = oracle_graph(orc, "csr", row_ptr=case["row_ptr"], col=case["col"], mask=case["mask"])
    with make_gpu("csr", row_ptr=case["row_ptr"], col=case["col"], mask=case["mask"], precision="fp64", seed=8,
                  J=1.0, K=0.2, e=(1, 1, 1)) as lat:
        assert lat.info.n_colours == g.n_colours == 2
        lat.init()
        S = lat.get_spins()
        lat.accumulate(True)
        lat.sweep(1.1, 3)
        mom, count = lat.read_accumulator()
    want = np.zeros(9)
    for s in range(3):
        orc.sweep(g, S, J=1.0, K=0.2, e=(1, 1, 1), beta=1.1, seed=8, sweep_index=s)
        m = orc.measure(g, S, J=1.0, K=0.2, e=(1, 1, 1))
        want += [m["E"], m["E"] ** 2, m["absM"], m["M2"], m["M4"], *m["M"], m["absMe"]]
    assert count == 3
    np.testing.assert_allclose(mom, want, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("kind,dims", [("sc", (10, 6, 4)), ("bcc", (3, 3, 2))])
def test_set_spins_from_page_locked_memory(precision, kind, dims):
    """Page-locked host input stores the same state as pageable input."""
    import torch
    with make_gpu(kind, dims, precision=precision, seed=1, **PARAMS) as lat:
        S = inputs.random_unit_spins(lat.info.n_sites, 5)
        lat.set_spins(S)
        want = lat.get_spins()
        pinned = torch.from_numpy(S.copy()).pin_memory()
        assert pinned.is_pinned()
        lat.init()
        assert not np.array_equal(lat.get_spins(), want)
        hs.hs_set_spins(lat.h, pinned.numpy())
        got = lat.get_spins()
    np.testing.assert_array_equal(got, want)


def test_edge_cases():
    # every site a vacancy: nothing to do, nothing fails
    with hs.Lattice("bcc", dims=(2, 2, 2), site_mask=np.zeros(16, np.uint8)) as lat:
        lat.sweep(1.0, 3)
        m = lat.measure()
        assert m["n_sites"] == 0 and m["E"] == 0.0
        assert (lat.get_spins() == 0).all()
    # zero sweeps, isolated sites (no bonds, width 0 table)
    rp, col = inputs.isolated_sites(37)
    with hs.Lattice("csr", row_ptr=rp, col_idx=col, K=0.5, precision="fp32", seed=1) as lat:
        lat.sweep(2.0, 0)
        lat.init()
        lat.sweep(2.0, 4)
        assert np.abs(np.linalg.norm(lat.get_spins(), axis=1) - 1).max() < 1e-6
    with hs.Lattice("sc", dims=(4, 4, 4)) as lat:
        with pytest.raises(hs.HSError):
            lat.sweep(-1.0, 1)
        with pytest.raises(hs.HSError):
            lat.sweep(float("nan"), 1)
    with pytest.raises(hs.HSError) as ei:
        hs.Lattice("sc", dims=(5, 4, 4))
    assert ei.value.code == -4


def test_beta_zero_accepts_everything_and_infinite_beta_nothing():
    with hs.Lattice("sc", dims=(16, 16, 16), K=0.1, precision="fp32", seed=3) as lat:
        lat.init()
        lat.sweep(0.0, 2)
        assert lat.measure()["accept_rate"] == 1.0
    with hs.Lattice("fcc", dims=(3, 3, 3), K=0.3, precision="fp64", seed=3) as lat:
        lat.init(hs.HS_INIT_ALIGNED)
        E0 = lat.measure()["E"]
        assert E0 == pytest.approx(-108 * (6 + 0.3), rel=1e-14)   # -N (J z / 2 + K)
        lat.sweep(1e12, 3)
        m = lat.measure()
        assert m["accept_rate"] == 0.0 and m["E"] == E0


def _launch_configs(precision, dims):
    widths = {"fp64": (1, 2), "fp32": (1, 2, 4), "fp16": (1, 2, 4, 8)}[precision]
    es = {"fp64": 8, "fp32": 4, "fp16": 2}[precision]
    lh = dims[0] // 2
    out = []
    for v in widths:
        if lh % v:
            continue
        out += [dict(kernel="stencil", vec_width=v, blocks_per_sm=1), dict(kernel="stencil", vec_width=v),
                dict(kernel="stencil", vec_width=v, prefetch=3),
                dict(kernel="stencil", vec_width=v, prefetch=1), dict(kernel="stencil", vec_width=v, prefetch=1,
                                                                       blocks_per_sm=1),
                # every pass ascending, and the split prefetch alternating, against the automatic orders
                dict(kernel="stencil", vec_width=v, order=1), dict(kernel="stencil", vec_width=v, prefetch=3, order=2),
                dict(kernel="stencil", vec_width=v, prefetch=1, order=1)]
        if 4 <= v * es <= 16:
            out += [dict(kernel="pipe", vec_width=v), dict(kernel="pipe", vec_width=v, blocks_per_sm=1)]
        for ty in (1, 2, 4):
            if dims[1] % ty == 0:
                out += [dict(kernel="march", vec_width=v, tile_y=ty), dict(kernel="march", vec_width=v, tile_y=ty,
                                                                           blocks_per_sm=1)]
    return out


@pytest.mark.parametrize("precision,dims", [("fp32", (16, 8, 6)), ("fp16", (32, 8, 4)), ("fp64", (8, 12, 8)),
                                            ("fp32", (8, 4, 2)),
                                            # rows of 36 vectors: split prefetch on rows wider than a warp
                                            ("fp32", (288, 16, 4)), ("fp16", (288, 8, 6))])
def test_launch_configuration_does_not_change_results(precision, dims):
    """A site's random numbers and arithmetic depend only on its natural index,
    so every kernel, vector width, CTA count, slab, prefetch mode and order
    of the work items gives bit-identical chains; the autotuner restores the
    state it perturbs."""
    outs = []
    cfgs = _launch_configs(precision, dims)
    assert all(any(c["kernel"] == k for c in cfgs) for k in ("stencil", "pipe", "march"))
    for cfg in cfgs:
        with hs.Lattice("sc", dims=dims, K=0.1, precision=precision, seed=6) as lat:
            lat.set_launch(**cfg)
            got = lat.launch
            assert got["vec_width"] == cfg["vec_width"] and got["kernel"] == hs.KERNELS[cfg["kernel"]]
            if cfg["kernel"] == "stencil":
                assert got["order"] == cfg.get("order", 1 if cfg.get("prefetch") == 3 else 2)
            lat.init()
            lat.accumulate(True)
            lat.sweep(0.9, 6)
            outs.append((lat.get_spins(), lat.read_accumulator()[0]))
    for (S, mom), cfg in zip(outs[1:], cfgs[1:]):
        assert np.array_equal(S, outs[0][0]), cfg
        # spins are bit-identical; FP32 per-thread partial sums group differently
        np.testing.assert_allclose(mom, outs[0][1], rtol=1e-12 if precision == "fp64" else 2e-6)
    with hs.Lattice("sc", dims=dims, K=0.1, precision=precision, seed=6) as lat:
        lat.init()
        lat.accumulate(True)
        lat.sweep(0.9, 2)
        lat.autotune(0.9, 2)
        assert lat.info.sweep == 2
        lat.sweep(0.9, 4)
        assert np.array_equal(lat.get_spins(), outs[0][0])
        assert lat.read_accumulator()[1] == 6


@pytest.mark.parametrize("precision", ["fp32", "fp16", "fp64"])
@pytest.mark.parametrize("kind,dims", [("bcc", (6, 5, 4)), ("fcc", (4, 3, 4)), ("sc_masked", (8, 8, 6))])
def test_table_launch_configuration_does_not_change_results(precision, kind, dims):
    """The neighbour-table kernel: CTAs per SM and the L2 prefetch of the next
    site's row give bit-identical chains."""
    mask = inputs.vacancy_mask(int(np.prod(dims)), 0.1, 4) if kind == "sc_masked" else None
    lattice = "sc" if kind == "sc_masked" else kind
    outs = []
    cfgs = [dict(kernel="table", blocks_per_sm=b, prefetch=pf) for b in (1, 0) for pf in (1, 2)]
    for cfg in cfgs:
        with hs.Lattice(lattice, dims=dims, site_mask=mask, K=0.1, precision=precision, seed=8) as lat:
            lat.set_launch(**cfg)
            assert lat.launch["prefetch"] == cfg["prefetch"]
            lat.init()
            lat.sweep(0.9, 5)
            outs.append(lat.get_spins())
    for S, cfg in zip(outs[1:], cfgs[1:]):
        assert np.array_equal(S, outs[0]), cfg

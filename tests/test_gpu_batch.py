"""Batched replicas (one persistent kernel for many lattices of uneven size,
in one precision: FP64, FP32 or FP16).

* The batch reproduces, member by member, what hs_sweep does on each lattice
  alone: identical spins, moments within the FP32 partial-sum tolerance.
* Physics: for K = 0 the Binder cumulant U4 = 1 - <M^4> / (3 <M^2>^2) of
  Eq. 2's magnetisation crosses between sizes at T_c; the sc Heisenberg value
  is T_c / J = 1.443 (the paper quotes 1.445).  The crossing of L = 32 and
  L = 48 must lie within max(3 sigma, 0.01) of 1.443, sigma from a jackknife
  over measurement blocks.
"""
import numpy as np
import pytest

from paper_2106_11286_gb300 import hs

pytestmark = pytest.mark.gpu


def _members(dims_list, betas, K=0.1, seed=11, precision="fp32", axes=None):
    axes = axes or [(0, 0, 1)] * len(dims_list)
    return [hs.Lattice("sc", dims=d, J=1.0, K=K, e=axes[r], precision=precision, seed=seed, replica=r)
            for r, d in enumerate(dims_list)]


RTOL = {"fp64": 1e-12, "fp32": 2e-6, "fp16": 2e-6}   # moments: FP64 sums taken in another order


# every member along z (FP32 batches then run their S.e = S_z kernels), or one
# member with another axis (the whole batch takes the general products)
@pytest.mark.parametrize("axes", ["z", "mixed"])
@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16"])
def test_batch_matches_individual_sweeps(precision, axes):
    dims = [(16, 16, 16), (24, 24, 24), (8, 8, 8), (32, 16, 8), (40, 8, 12)]
    betas = [0.6, 0.8, 1.0, 1.2, 0.9]
    ax = [(0, 0, 1)] * 5 if axes == "z" else [(0, 0, 1), (0.3, -0.2, 1.0), (0, 0, 1), (0, 0, 1), (1, 0, 0)]
    a = _members(dims, betas, precision=precision, axes=ax)
    b = _members(dims, betas, precision=precision, axes=ax)
    for x, y in zip(a, b):
        x.init()
        y.init()
        x.accumulate(True)
    batch = hs.hs_batch_create([m.h for m in a])
    try:
        for n_equil, n_sweeps in ((3, 5), (3, 5), (0, 4)):   # second call reuses the captured graph
            for m in a:
                m.reset_accumulator()
            hs.hs_batch_run(batch, betas, n_sweeps, n_equil)
            rates = []
            for m, beta in zip(b, betas):
                m.accumulate(False)
                m.sweep(beta, n_equil)
                r_eq = m.measure()["accept_rate"] if n_equil else 0.0
                m.accumulate(True)
                m.reset_accumulator()
                m.sweep(beta, n_sweeps)
                r_sw = m.measure()["accept_rate"]
                rates.append((r_eq * n_equil + r_sw * n_sweeps) / (n_equil + n_sweeps))
            for x, y, rate in zip(a, b, rates):
                assert np.array_equal(x.get_spins(), y.get_spins())
                mx, cx = x.read_accumulator()
                my, cy = y.read_accumulator()
                assert cx == cy == n_sweeps
                np.testing.assert_allclose(mx, my, rtol=RTOL[precision], atol=1e-9)
                assert x.info.sweep == y.info.sweep
                # a batch run's acceptance rate covers all of its sweeps
                assert x.measure()["accept_rate"] == pytest.approx(rate, abs=1e-12)
    finally:
        hs.hs_batch_destroy(batch)
        for m in a + b:
            m.close()


def test_batch_autotune_keeps_the_chains():
    """The batch autotuner times every work split and restores every member:
    afterwards the batch continues exactly as an untuned one; every split
    gives the same spins."""
    dims = [(16, 16, 16), (24, 24, 24), (8, 8, 8), (32, 16, 8), (48, 48, 48)]
    betas = [0.6, 0.8, 1.0, 1.2, 0.9]
    a = _members(dims, betas)
    b = _members(dims, betas)
    for m in a + b:
        m.init()
        m.accumulate(True)
    ba = hs.hs_batch_create([m.h for m in a])
    bb = hs.hs_batch_create([m.h for m in b])
    try:
        assert hs.hs_batch_get_layout(bb) == {"ctas_per_sm": 2, "align_rows": 2, "prefetch": 0, "schedule": 0}
        hs.hs_batch_run(ba, betas, 2, 1)
        hs.hs_batch_run(bb, betas, 2, 1)
        before = [m.get_spins() for m in a]
        layout = hs.hs_batch_autotune(ba, betas, 2)
        assert layout["ctas_per_sm"] in (1, 2) and layout["align_rows"] in (0, 1, 2)
        for m, s in zip(a, before):
            assert np.array_equal(m.get_spins(), s)
            assert m.info.sweep == 3
        hs.hs_batch_run(ba, betas, 4, 0)
        hs.hs_batch_run(bb, betas, 4, 0)
        for x, y in zip(a, b):
            assert np.array_equal(x.get_spins(), y.get_spins())
            mx, cx = x.read_accumulator()
            my, cy = y.read_accumulator()
            assert cx == cy == 6
            np.testing.assert_allclose(mx, my, rtol=2e-6, atol=1e-9)
    finally:
        hs.hs_batch_destroy(ba)
        hs.hs_batch_destroy(bb)
        for m in a + b:
            m.close()


@pytest.mark.parametrize("ctas,align,prefetch,schedule", [(1, 0, 1, 0), (2, 1, 1, 0), (2, 0, 1, 0), (1, 1, 0, 0),
                                                           (2, 0, 0, 1), (2, 1, 1, 1), (1, 0, 0, 1), (2, 0, 0, 0),
                                                           (2, 2, 1, 0), (2, 2, 0, 1), (1, 2, 0, 0)])
def test_batch_layouts_give_identical_chains(ctas, align, prefetch, schedule):
    """Every work split (contiguous ranges, or interleaved blocks sweeping a
    member side by side), load schedule (split prefetch included) and colour schedule
    (persistent, or a launch per pass) gives the spins of the default layout
    bit for bit, and the same moments up to the order of the FP64 segment
    sums."""
    dims = [(16, 16, 16), (24, 24, 24), (8, 8, 8), (32, 16, 8), (48, 48, 48), (96, 96, 96)]
    betas = [0.6, 0.8, 1.0, 1.2, 0.9, 0.7]
    a = _members(dims, betas)
    b = _members(dims, betas)
    for m in a + b:
        m.init()
        m.accumulate(True)
    ba = hs.hs_batch_create([m.h for m in a])
    bb = hs.hs_batch_create([m.h for m in b])
    try:
        hs.hs_batch_set_layout(bb, ctas, align, prefetch, schedule)
        assert hs.hs_batch_get_layout(bb) == {"ctas_per_sm": ctas, "align_rows": align, "prefetch": prefetch,
                                              "schedule": schedule}
        hs.hs_batch_run(ba, betas, 3, 2)
        hs.hs_batch_run(bb, betas, 3, 2)
        for x, y in zip(a, b):
            assert np.array_equal(x.get_spins(), y.get_spins())
            mx, cx = x.read_accumulator()
            my, cy = y.read_accumulator()
            assert cx == cy == 3
            np.testing.assert_allclose(mx, my, rtol=2e-6, atol=1e-9)
        with pytest.raises(hs.HSError):
            hs.hs_batch_set_layout(bb, 0, 0, 0)
        with pytest.raises(hs.HSError):
            hs.hs_batch_set_layout(bb, 1, 0, 2)
        with pytest.raises(hs.HSError):
            hs.hs_batch_set_layout(bb, 1, 0, 0, 2)   # 48^3 and 96^3 do not fit in a CTA's shared memory
        with pytest.raises(hs.HSError):
            hs.hs_batch_set_layout(bb, 1, 0, 0, 3)
        with pytest.raises(hs.HSError):
            hs.hs_batch_set_layout(bb, 1, 3, 0, 0)
    finally:
        hs.hs_batch_destroy(ba)
        hs.hs_batch_destroy(bb)
        for m in a + b:
            m.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16"])
def test_resident_schedule_gives_identical_chains(precision):
    """Schedule 2: every member (here up to 24^3, 166 KB of FP32 planes; up
    to 16^3, 98 KB, in FP64) in one CTA's shared memory for the whole run.
    Member by member the spins equal hs_sweep on each lattice alone and the
    persistent batch's, bit for bit, over repeated runs with and without
    equilibration; moments and acceptance rates agree up to the order of the
    FP64 sums."""
    big = (12, 12, 12) if precision == "fp64" else (24, 24, 24)
    dims = [(16, 16, 16), big, (8, 8, 8), (16, 8, 24), (24, 16, 8), (8, 24, 16)]
    betas = [0.6, 0.8, 1.0, 1.2, 0.9, 0.7]
    a = _members(dims, betas, precision=precision)
    b = _members(dims, betas, precision=precision)
    c = _members(dims, betas, precision=precision)
    for m in a + b + c:
        m.init()
        m.accumulate(True)
    ba = hs.hs_batch_create([m.h for m in a])
    bb = hs.hs_batch_create([m.h for m in b])
    try:
        hs.hs_batch_set_layout(ba, 2, 2, 0, 2)
        assert hs.hs_batch_get_layout(ba)["schedule"] == 2
        for n_equil, n_sweeps in ((3, 5), (0, 4), (2, 0)):
            for m in a + b + c:
                m.reset_accumulator()
            hs.hs_batch_run(ba, betas, n_sweeps, n_equil)
            hs.hs_batch_run(bb, betas, n_sweeps, n_equil)
            for m, beta in zip(c, betas):
                m.accumulate(False)
                m.sweep(beta, n_equil)
                m.accumulate(True)
                m.sweep(beta, n_sweeps)
            for x, y, z in zip(a, b, c):
                assert np.array_equal(x.get_spins(), y.get_spins())
                assert np.array_equal(x.get_spins(), z.get_spins())
                mx, cx = x.read_accumulator()
                my, cy = y.read_accumulator()
                mz, cz = z.read_accumulator()
                assert cx == cy == cz == n_sweeps
                np.testing.assert_allclose(mx, my, rtol=RTOL[precision], atol=1e-9)
                np.testing.assert_allclose(mx, mz, rtol=RTOL[precision], atol=1e-9)
                assert x.info.sweep == y.info.sweep == z.info.sweep
                assert x.measure()["accept_rate"] == pytest.approx(y.measure()["accept_rate"], abs=1e-12)
        layout = hs.hs_batch_autotune(ba, betas, 2)   # the resident schedule is one of its candidates
        assert layout["schedule"] in (0, 1, 2)
        hs.hs_batch_run(ba, betas, 3, 0)
        hs.hs_batch_run(bb, betas, 3, 0)
        for x, y in zip(a, b):
            assert np.array_equal(x.get_spins(), y.get_spins())
    finally:
        hs.hs_batch_destroy(ba)
        hs.hs_batch_destroy(bb)
        for m in a + b + c:
            m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp16"])
@pytest.mark.parametrize("ctas,align,prefetch,schedule", [(2, 2, 0, 0), (1, 0, 1, 0), (2, 1, 1, 1), (2, 2, 0, 1)])
def test_batch_layouts_other_precisions(precision, ctas, align, prefetch, schedule):
    """FP64 and FP16 batches: each work split, load and colour schedule gives
    the spins of hs_sweep on each member alone, bit for bit."""
    dims = [(16, 16, 16), (24, 24, 24), (8, 8, 8), (32, 16, 8), (48, 48, 48)]
    betas = [0.6, 0.8, 1.0, 1.2, 0.9]
    a = _members(dims, betas, precision=precision)
    c = _members(dims, betas, precision=precision)
    for m in a + c:
        m.init()
        m.accumulate(True)
    ba = hs.hs_batch_create([m.h for m in a])
    try:
        hs.hs_batch_set_layout(ba, ctas, align, prefetch, schedule)
        hs.hs_batch_run(ba, betas, 3, 2)
        for m, beta in zip(c, betas):
            m.accumulate(False)
            m.sweep(beta, 2)
            m.accumulate(True)
            m.sweep(beta, 3)
        for x, z in zip(a, c):
            assert np.array_equal(x.get_spins(), z.get_spins())
            mx, cx = x.read_accumulator()
            mz, cz = z.read_accumulator()
            assert cx == cz == 3
            np.testing.assert_allclose(mx, mz, rtol=RTOL[precision], atol=1e-9)
    finally:
        hs.hs_batch_destroy(ba)
        for m in a + c:
            m.close()


def test_batch_rejects_unsupported_members():
    with hs.Lattice("sc", dims=(8, 8, 8), precision="fp64") as x, \
            hs.Lattice("sc", dims=(8, 8, 8), precision="fp32") as y:
        with pytest.raises(hs.HSError):
            hs.hs_batch_create([x.h, y.h])                        # two precisions
    for precision in ("fp32", "fp16"):
        with hs.Lattice("sc", dims=(12, 8, 8), precision=precision) as x:   # Lx/2 = 6 not divisible by 4
            with pytest.raises(hs.HSError):
                hs.hs_batch_create([x.h])
    with hs.Lattice("sc", dims=(6, 8, 8), precision="fp64") as x:   # Lx/2 = 3 not divisible by 2
        with pytest.raises(hs.HSError):
            hs.hs_batch_create([x.h])
    with hs.Lattice("sc", dims=(8, 8, 8), precision="fp32", site_mask=np.ones(512, dtype=np.uint8)) as x:
        with pytest.raises(hs.HSError):
            hs.hs_batch_create([x.h])                              # the neighbour-table layout


def _crossing(Ts, u_small, u_large):
    d = u_large - u_small
    idx = np.nonzero((d[:-1] > 0) & (d[1:] <= 0))[0]
    if len(idx) == 0:
        return np.nan
    k = idx[0]
    return Ts[k] + (Ts[k + 1] - Ts[k]) * d[k] / (d[k] - d[k + 1])


def test_binder_crossing_locates_tc():
    sizes = (32, 48)
    Ts = np.linspace(1.41, 1.47, 7)
    lats = []
    for L in sizes:
        for i, T in enumerate(Ts):
            lats.append(hs.Lattice("sc", dims=(L, L, L), J=1.0, K=0.0, precision="fp32", seed=2024,
                                   replica=1000 * L + i))
    betas = [1.0 / T for L in sizes for T in Ts]
    for m in lats:
        m.init()
    batch = hs.hs_batch_create([m.h for m in lats])
    n_blocks, block = 24, 2500
    m2 = np.zeros((n_blocks, len(lats)))
    m4 = np.zeros((n_blocks, len(lats)))
    try:
        hs.hs_batch_run(batch, betas, 0, 5000)       # equilibrate
        for k in range(n_blocks):
            for m in lats:
                m.reset_accumulator()
            hs.hs_batch_run(batch, betas, block, 0)
            for j, m in enumerate(lats):
                mom, cnt = m.read_accumulator()
                assert cnt == block
                m2[k, j] = mom[3] / cnt
                m4[k, j] = mom[4] / cnt
    finally:
        hs.hs_batch_destroy(batch)
        for m in lats:
            m.close()
    nT = len(Ts)

    def estimate(rows):
        a2 = m2[rows].mean(0)
        a4 = m4[rows].mean(0)
        u = 1.0 - a4 / (3.0 * a2 ** 2)
        return _crossing(Ts, u[:nT], u[nT:])
    t_all = estimate(np.arange(n_blocks))
    jack = np.array([estimate(np.delete(np.arange(n_blocks), k)) for k in range(n_blocks)])
    assert np.isfinite(t_all) and np.isfinite(jack).all()
    sigma = np.sqrt((n_blocks - 1) / n_blocks * ((jack - jack.mean()) ** 2).sum())
    assert abs(t_all - 1.443) < max(3 * sigma, 0.01), (t_all, sigma)

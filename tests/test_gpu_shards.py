"""z-slab domain decomposition on one GPU (the exchange a multi-device run
performs), against the whole lattice.

* A lattice cut into 1 .. 16 slabs (down to one plane each), halos exchanged
  between colour passes, reproduces the whole lattice's chain bit for bit in
  every precision; the slabs' fused sums add up to the whole lattice's E, M
  and accepted moves.
* Slabs initialise with the whole lattice's global indices.
* The sc 256^3 workload in four slabs matches the whole lattice after a
  sweep.
* A one-rank torch.distributed slab (its own periodic neighbour) matches.
* Boundary-first passes (boundary planes, then the interior while the halo
  copies run on a communication stream) give the same chain and sums, for
  slabs of one plane up to sixteen, with any number of CTAs left free for
  the communication, and with whole and split passes mixed in one sweep.
"""
import os
import socket

import numpy as np
import pytest

from helpers import storage_round
from paper_2106_11286_gb300 import hs, inputs, shards

pytestmark = pytest.mark.gpu

PARAMS = dict(J=1.0, K=0.3, e=(0.3, -0.2, 1.0))


def _whole_and_sharded(dims, n_slabs, precision, seed=5, sweeps=3, beta=0.9, start=7, overlap=False):
    n = dims[0] * dims[1] * dims[2]
    S0 = storage_round(inputs.random_unit_spins(n, 17), precision)
    with hs.Lattice("sc", dims=dims, precision=precision, seed=seed, **PARAMS) as whole:
        whole.set_spins(S0)
        whole.set_sweep_counter(start)
        whole.accumulate(True)   # the fused sums (a slab always measures them)
        whole.sweep(beta, sweeps)
        want, want_sums = whole.get_spins(), hs.hs_read_sums(whole.h)
    with shards.ShardedLattice(dims, n_slabs, precision=precision, seed=seed, overlap=overlap, **PARAMS) as sh:
        sh.set_spins(S0)
        sh.set_sweep_counter(start)
        sh.sweep(beta, sweeps)
        got, obs = sh.get_spins(), sh.last_observables()
    return S0, want, want_sums, got, obs


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("n_slabs", [1, 2, 4, 8, 16])
def test_slabs_reproduce_the_whole_lattice(precision, n_slabs, overlap):
    dims = (16, 12, 16)   # 16 .. 1 planes per slab: an interior of 14 .. 2 planes, or none
    S0, want, want_sums, got, obs = _whole_and_sharded(dims, n_slabs, precision, overlap=overlap)
    assert not np.array_equal(want, S0)
    assert np.array_equal(got, want)
    assert want_sums[0] != 0.0
    n = dims[0] * dims[1] * dims[2]
    # FP64 sums in another grouping; FP32 / FP16 per-thread partials also group differently
    rel, atol = (1e-12, 1e-9) if precision == "fp64" else (2e-6, 1e-4)
    assert obs["E"] == pytest.approx(want_sums[0], rel=rel, abs=atol)
    np.testing.assert_allclose(obs["M"] * n, want_sums[1:4], rtol=rel, atol=atol)
    assert obs["accepted"] == want_sums[4]


def test_slab_init_uses_global_indices():
    dims = (8, 6, 12)
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=3, replica=2) as whole:
        whole.init()
        want = whole.get_spins()
    with shards.ShardedLattice(dims, 3, precision="fp32", seed=3, replica=2) as sh:
        sh.init()
        assert np.array_equal(sh.get_spins(), want)


def test_256_workload_in_four_slabs():
    dims = (256, 256, 256)
    p = dict(J=1.0, K=0.05, e=(0.0, 0.0, 1.0))
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=2, **p) as whole:
        whole.init()
        S0 = whole.get_spins()
        whole.sweep(1 / 1.2, 1)
        want = whole.get_spins()
    with shards.ShardedLattice(dims, 4, precision="fp32", seed=2, **p) as sh:
        sh.set_spins(S0)
        sh.sweep(1 / 1.2, 1)
        assert np.array_equal(sh.get_spins(), want)


def test_slab_api_limits():
    with hs.Slab((8, 8, 8), 2, 4, precision="fp32") as s:
        assert s.info.n_present == 8 * 8 * 4
        with pytest.raises(hs.HSError):
            s.sweep(1.0, 1)
        with pytest.raises(hs.HSError):
            s.measure()
        with pytest.raises(hs.HSError):
            s.set_launch(kernel="pipe")
        with pytest.raises(hs.HSError):
            hs.hs_batch_create([s.h])
        with pytest.raises(hs.HSError):
            hs.hs_slab_plane(s.h, 0, 0, 4)
    with pytest.raises(hs.HSError):
        hs.Slab((8, 8, 8), 6, 4)   # planes beyond Lz


@pytest.mark.parametrize("overlap", [False, True])
def test_one_rank_distributed_slab(overlap):
    import torch
    import torch.distributed as dist
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    dims = (16, 8, 8)
    n = dims[0] * dims[1] * dims[2]
    S0 = storage_round(inputs.random_unit_spins(n, 4), "fp32")
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=8, **PARAMS) as whole:
        whole.set_spins(S0)
        whole.accumulate(True)   # the fused sums (a slab always measures them)
        whole.sweep(1.0, 2)
        want, want_sums = whole.get_spins(), hs.hs_read_sums(whole.h)
    assert want_sums[0] != 0.0
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        ds = shards.DistributedSlab(dims, precision="fp32", seed=8, overlap=overlap, **PARAMS)
        ds.slab.set_spins(S0)
        ds.exchange(0)
        ds.exchange(1)
        ds.sweep(1.0, 2)
        assert np.array_equal(ds.slab.get_spins(), want)
        obs = ds.last_observables()
        assert obs["E"] == pytest.approx(want_sums[0], rel=2e-6)
        ds.close()
    finally:
        dist.destroy_process_group()
        torch.cuda.synchronize()


def _sums_close(obs, want_sums, n):
    assert obs["E"] == pytest.approx(want_sums[0], rel=2e-6, abs=1e-4)
    np.testing.assert_allclose(obs["M"] * n, want_sums[1:4], rtol=2e-6, atol=1e-4)
    assert obs["accepted"] == want_sums[4]


@pytest.mark.parametrize("reserve", [0, 5, -1])
def test_boundary_first_with_ctas_left_free(reserve):
    """Interior launches of fewer CTAs (down to one) than the pass's stride
    of partial sums: the sets' unwritten tails read zero, so the sums hold."""
    dims = (64, 64, 32)
    n = dims[0] * dims[1] * dims[2]
    S0 = storage_round(inputs.random_unit_spins(n, 9), "fp32")
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=4, **PARAMS) as whole:
        whole.set_spins(S0)
        whole.accumulate(True)
        whole.sweep(0.8, 2)
        want, want_sums = whole.get_spins(), hs.hs_read_sums(whole.h)
    with shards.ShardedLattice(dims, 2, precision="fp32", seed=4, overlap=True, **PARAMS) as sh:
        for s in sh.slabs:
            r = reserve
            if r < 0:   # all but one CTA
                r = _pass_ctas(s) - 1
            s.reserve_ctas(r)
        sh.set_spins(S0)
        sh.sweep(0.8, 2)
        assert np.array_equal(sh.get_spins(), want)
        _sums_close(sh.last_observables(), want_sums, n)


def _pass_ctas(slab):
    """The largest reserve a slab takes + 1 (its pass's CTA count), found
    through the reserve's own range check."""
    lo, hi = 0, 1 << 16
    while lo < hi:   # largest r with reserve_ctas(r) accepted
        mid = (lo + hi + 1) // 2
        try:
            slab.reserve_ctas(mid)
            lo = mid
        except hs.HSError:
            hi = mid - 1
    slab.reserve_ctas(0)
    return lo + 1


def test_whole_and_split_passes_mixed():
    """Sweeps that alternate whole passes and boundary / interior parts, and
    one sweep with a whole colour-0 pass and a split colour-1 pass: only the
    partial sets written in a sweep enter its sums."""
    dims = (16, 12, 12)
    n = dims[0] * dims[1] * dims[2]
    S0 = storage_round(inputs.random_unit_spins(n, 3), "fp32")
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=6, **PARAMS) as whole, \
            shards.ShardedLattice(dims, 2, precision="fp32", seed=6, **PARAMS) as sh:
        whole.set_spins(S0)
        whole.accumulate(True)
        sh.set_spins(S0)
        for mode in ("whole", "split", "whole", "mixed", "split"):
            whole.sweep(1.1, 1)
            want, want_sums = whole.get_spins(), hs.hs_read_sums(whole.h)
            for c in (0, 1):
                split = mode == "split" or (mode == "mixed" and c == 1)
                for s in sh.slabs:
                    if split:
                        s.sweep_part(1.1, c, hs.HS_PART_BOUNDARY)
                        s.sweep_part(1.1, c, hs.HS_PART_INTERIOR)
                    else:
                        s.sweep_part(1.1, c, hs.HS_PART_WHOLE)
                sh.exchange(c)
            assert np.array_equal(sh.get_spins(), want), mode
            _sums_close(sh.last_observables(), want_sums, n)


def test_pass_part_rules():
    with hs.Slab((8, 8, 8), 0, 4, precision="fp32") as s:
        with pytest.raises(hs.HSError):
            s.sweep_part(1.0, 0, hs.HS_PART_INTERIOR)     # no boundary part before it
        s.sweep_part(1.0, 0, hs.HS_PART_BOUNDARY)
        with pytest.raises(hs.HSError):
            s.sweep_part(1.0, 0, hs.HS_PART_BOUNDARY)     # the interior part is due
        with pytest.raises(hs.HSError):
            s.sweep_part(1.0, 1, hs.HS_PART_INTERIOR)     # of the other colour
        with pytest.raises(hs.HSError):
            s.reserve_ctas(0)                             # mid-sweep
        with pytest.raises(hs.HSError):
            s.set_launch(prefetch=3)                      # mid-sweep
        s.sweep_part(1.0, 0, hs.HS_PART_INTERIOR)
        with pytest.raises(hs.HSError):
            s.sweep_part(1.0, 1, 3)                       # no such part
        s.sweep_part(1.0, 1, hs.HS_PART_WHOLE)
        assert s.info.sweep == 1
        s.reserve_ctas(0)
        with pytest.raises(hs.HSError):
            s.reserve_ctas(-1)
        with pytest.raises(hs.HSError):
            s.reserve_ctas(1 << 20)
    with hs.Lattice("sc", dims=(8, 8, 8), precision="fp32") as lat:
        with pytest.raises(hs.HSError):
            hs.hs_sweep_pass_part(lat.h, 1.0, 0, hs.HS_PART_BOUNDARY)
        with pytest.raises(hs.HSError):
            hs.hs_slab_reserve_ctas(lat.h, 0)
        with pytest.raises(hs.HSError):
            hs.hs_slab_set_comm_stream(lat.h, None)


def test_whole_part_is_the_pass():
    dims = (16, 8, 8)
    out = []
    for part in (False, True):
        with hs.Lattice("sc", dims=dims, precision="fp32", seed=2, **PARAMS) as lat:
            lat.init()
            for c in (0, 1):
                if part:
                    hs.hs_sweep_pass_part(lat.h, 0.7, c, hs.HS_PART_WHOLE)
                else:
                    hs.hs_sweep_pass(lat.h, 0.7, c)
            out.append((lat.get_spins(), hs.hs_read_sums(lat.h), lat.info.sweep))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2] == 1


@pytest.mark.parametrize("overlap", [False, True])
def test_distributed_slab_without_a_process_group(overlap):
    """No torch.distributed group: one slab, its own periodic neighbour, no
    collective (the one-process form of the strong-scaling run)."""
    import torch.distributed as dist
    assert not dist.is_initialized()
    dims = (16, 8, 8)
    n = dims[0] * dims[1] * dims[2]
    S0 = storage_round(inputs.random_unit_spins(n, 6), "fp32")
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=3, **PARAMS) as whole:
        whole.set_spins(S0)
        whole.accumulate(True)
        whole.sweep(0.9, 3)
        want, want_mom = whole.get_spins(), whole.read_accumulator()
    ds = shards.DistributedSlab(dims, precision="fp32", seed=3, overlap=overlap, **PARAMS)
    try:
        assert (ds.rank, ds.world) == (0, 1)
        ds.set_spins(S0)
        ds.accumulate(True)
        ds.sweep(0.9, 3)
        assert np.array_equal(ds.get_spins(), want)
        mom, cnt = ds.read_accumulator()
        assert cnt == want_mom[1] == 3
        np.testing.assert_allclose(mom, want_mom[0], rtol=2e-6, atol=1e-9)
        _sums_close(ds.last_observables(), hs.hs_read_sums(ds.slab.h), n)
    finally:
        ds.close()

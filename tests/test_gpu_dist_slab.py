"""The multi-process z-slab path itself: two processes, one slab each, on the
one GPU of the test machine, with DistributedSlab's world > 1 branch --
packed boundary planes (hs_slab_pack / hs_slab_unpack) exchanged between the
ranks after every colour pass, the five fused sums allreduced every sweep and
the whole lattice's moments accumulated on the device (hs_accumulate_sums).
The transport is "host" (gloo through pinned host buffers): NCCL cannot pair
two ranks on one device.  Each process launches only its own kernels and
waits for its peer on the host, so no kernel waits on another process.

sc 16 x 8 x 12 periodic, J = 1, K = 0.1, e = (0.3, -0.2, 1): after three
sweeps the slabs, concatenated in rank order, equal the whole lattice's spins
bit for bit, and every rank's accumulator holds the whole lattice's moments
(FP64 sums added in another order; FP32 per-thread partials grouped
differently).  The same holds with the boundary-first schedule (overlap:
boundary planes updated first, the exchange on a communication stream with
the interior update queued before the host waits for the messages).
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

from paper_2106_11286_gb300 import hs, inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (16, 8, 12)
PARAMS = dict(J=1.0, K=0.1, e=(0.3, -0.2, 1.0))
SWEEPS = 3


def _worker(rank, world, port, precision, overlap, S0, q):
    sys.path.insert(0, ROOT)
    try:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
        from paper_2106_11286_gb300 import shards
        ds = shards.DistributedSlab(DIMS, precision=precision, seed=8, transport="host", overlap=overlap,
                                    **PARAMS)
        plane, nz = DIMS[0] * DIMS[1], DIMS[2] // world
        ds.set_spins(S0[rank * nz * plane:(rank + 1) * nz * plane])
        ds.accumulate(True)
        ds.sweep(1.0, SWEEPS)
        mom, cnt = ds.read_accumulator()
        obs = ds.last_observables()
        q.put((rank, ds.get_spins(), mom, cnt, obs["E"]))
        ds.close()
        dist.destroy_process_group()
    except Exception as ex:  # reported to the test, which fails on it
        q.put((rank, repr(ex), None, None, None))


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_two_process_slabs_reproduce_the_whole_lattice(precision, rtol, overlap):
    n = DIMS[0] * DIMS[1] * DIMS[2]
    S0 = inputs.random_unit_spins(n, 21)
    if precision == "fp32":
        S0 = S0.astype(np.float32).astype(np.float64)
    with hs.Lattice("sc", dims=DIMS, precision=precision, seed=8, **PARAMS) as whole:
        whole.set_spins(S0)
        whole.accumulate(True)
        whole.sweep(1.0, SWEEPS)
        want = whole.get_spins()
        want_mom, want_cnt = whole.read_accumulator()
        want_E = hs.hs_read_sums(whole.h)[0]
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, precision, overlap, S0, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = dict()
        for _ in range(2):
            r, spins, mom, cnt, E = q.get(timeout=300)
            assert mom is not None, spins
            got[r] = (spins, mom, cnt, E)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert np.array_equal(np.concatenate([got[0][0], got[1][0]]), want)
    for r in (0, 1):
        spins, mom, cnt, E = got[r]
        assert cnt == want_cnt == SWEEPS
        np.testing.assert_allclose(mom, want_mom, rtol=rtol, atol=1e-9)
        assert E == pytest.approx(want_E, rel=rtol)

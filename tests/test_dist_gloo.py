"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Under torchrun each rank advances its own replica; the whole-job throughput
is the attempts of all ranks over the slowest rank's time.  This checks that
aggregation, and that the replica index (= rank) gives each rank a distinct
Philox stream, without a GPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    from oracle import oracle as orc
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    attempts = 1000.0 * (rank + 1)
    seconds = 0.5 + rank           # rank 1 is the slowest
    tot_a, tot_s = bench.aggregate(attempts, seconds, world)
    # replica = rank: distinct initial states from one seed
    g = orc.lattice("sc", (4, 4, 4))
    S = orc.init_spins(g, seed=2, replica=rank)
    gathered = [torch.zeros(192, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(S.reshape(-1).copy()))
    out[rank] = (tot_a, tot_s, bool((gathered[0] - gathered[1]).abs().max() > 0.1))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        tot_a, tot_s, distinct = res[rank]
        assert tot_a == 3000.0          # sum over ranks
        assert tot_s == 1.5             # max over ranks
        assert distinct

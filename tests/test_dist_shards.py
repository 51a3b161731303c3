"""The z-slab decomposition's exchange on CPU ranks (gloo, world size 2 and
4), with the oracle's single-site form of Metropolis steps (ii)-(iii) as each
rank's compute: every rank owns Lz / W whole z planes plus a halo plane on
each side, updates its sites of one colour, then exchanges that colour's
boundary planes as ``shards.halo_plan`` prescribes.  After three sweeps the
gathered lattice equals the oracle's sweep of the whole lattice bit for bit.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (6, 4, 8)
PARAMS = dict(J=1.0, K=0.3, e=(0.2, -0.5, 1.0))
SWEEPS, BETA, SEED, START = 3, 0.8, 11, 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    from oracle import oracle as orc
    from paper_2106_11286_gb300 import hs, inputs, shards
    Lx, Ly, Lz = DIMS
    plane, nz = Lx * Ly, Lz // world
    n = plane * Lz
    colour = orc.colour_structured("sc", DIMS)
    rank_in_colour = np.empty(n, dtype=np.int64)
    for c in (0, 1):
        sel = colour == c
        rank_in_colour[sel] = np.arange(int(sel.sum()))
    S_all = inputs.random_unit_spins(n, 23)
    # local planes: 0 = halo below, 1 .. nz = own global planes rank nz .., nz + 1 = halo above
    z0 = rank * nz
    loc = np.zeros((nz + 2, plane, 3))
    for j in range(nz + 2):
        loc[j] = S_all.reshape(Lz, plane, 3)[(z0 - 1 + j) % Lz]
    own = np.arange(z0 * plane, (z0 + nz) * plane)

    def local_row(g):   # global natural index -> (local plane, offset in plane)
        zg, off = g // plane, g % plane
        return (zg - z0 + 1) % Lz, off   # local planes hold global planes z0 - 1 .. z0 + nz

    which_plane = {hs.FIRST_OWN: 1, hs.LAST_OWN: nz, hs.HALO_BELOW: 0, hs.HALO_ABOVE: nz + 1}
    for s in range(SWEEPS):
        for c in (0, 1):
            sites = own[colour[own] == c]
            nb = orc.sc_site_neighbours(DIMS, True, sites)
            h = np.zeros((len(sites), 3))
            for k in range(6):
                j, off = local_row(nb[:, k])
                h += loc[j, off]
            js, offs = local_row(sites)
            spins = loc[js, offs].copy()
            orc.sites_update(sites, rank_in_colour[sites], np.full(len(sites), c), h, spins, beta=BETA, seed=SEED,
                             sweep_index=START + s, mode=0, **PARAMS)
            loc[js, offs] = spins
            # exchange colour c's boundary planes (whole planes: the other colour is unchanged)
            reqs = []
            for src, src_which, dst, dst_which in shards.halo_plan(world):
                if src == rank:
                    buf = torch.from_numpy(loc[which_plane[src_which]].copy())
                    reqs.append((dist.isend(buf, dst), None, None))
                if dst == rank:
                    buf = torch.zeros(plane, 3, dtype=torch.float64)
                    reqs.append((dist.irecv(buf, src), buf, which_plane[dst_which]))
            for req, buf, j in reqs:
                req.wait()
                if buf is not None:
                    loc[j] = buf.numpy()
    mine = torch.from_numpy(np.ascontiguousarray(loc[1:nz + 1].reshape(-1, 3)))
    gathered = [torch.zeros(nz * plane, 3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, mine)
    out[rank] = torch.cat(gathered).numpy()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slab_ranks_reproduce_the_whole_sweep(world):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    from paper_2106_11286_gb300 import inputs
    orc.build()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    g = orc.lattice("sc", DIMS)
    want = inputs.random_unit_spins(g.n, 23)
    for s in range(SWEEPS):
        orc.sweep(g, want, beta=BETA, seed=SEED, sweep_index=START + s, mode=0, **PARAMS)
    for r in range(world):
        assert np.array_equal(out[r], want)

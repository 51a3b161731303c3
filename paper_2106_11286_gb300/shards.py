"""Domain decomposition of a periodic sc lattice into z-slabs.

A colour pass updates one colour class; its neighbours are all of the other
colour.  So a lattice cut into slabs of whole z planes advances bit for bit
like the whole lattice if, after each colour pass, every slab sends the
boundary planes of the colour just updated to its neighbours' halos: its
first own plane to the slab below (halo above) and its last own plane to the
slab above (halo below), periodically.  The per-sweep observables combine by
summing each slab's fused FP64 sums (E shares, spin sums, accepted moves):
the scalar allreduce of a multi-device run.

``halo_plan`` is that exchange, written once; ``ShardedLattice`` runs it for
slabs that share one device (plane copies on the device), and
``DistributedSlab`` for one slab per process with torch.distributed
point-to-point sends of device planes.
"""
from __future__ import annotations

import numpy as np

from . import hs


def halo_plan(n_slabs: int):
    """(src slab, src plane, dst slab, dst plane) transfers of one colour's
    boundary planes, slab k owning planes k nz .. (k+1) nz - 1."""
    plan = []
    for k in range(n_slabs):
        plan.append((k, hs.FIRST_OWN, (k - 1) % n_slabs, hs.HALO_ABOVE))
        plan.append((k, hs.LAST_OWN, (k + 1) % n_slabs, hs.HALO_BELOW))
    return plan


def combine_sums(sums, n_sites: int, e_axis) -> dict:
    """Global observables from per-slab sums {E share, sum S, accepted}."""
    tot = np.sum(np.asarray(sums, dtype=np.float64), axis=0)
    M = tot[1:4] / n_sites
    m2 = float(M @ M)
    ev = np.asarray(e_axis, dtype=np.float64)
    ev = ev / np.linalg.norm(ev)
    return {"E": float(tot[0]), "M": M, "absM": m2 ** 0.5, "M2": m2, "M4": m2 * m2, "absMe": abs(float(M @ ev)),
            "accepted": float(tot[4])}


class ShardedLattice:
    """A periodic sc lattice as ``n_slabs`` z-slabs on the current device,
    halos exchanged by device copies between colour passes."""

    def __init__(self, dims, n_slabs: int, *, J=1.0, K=0.0, e=(0.0, 0.0, 1.0), precision="fp32", seed=0,
                 replica=0, stream=None):
        Lx, Ly, Lz = (int(d) for d in dims)
        if n_slabs < 1 or Lz % n_slabs:
            raise ValueError("the slab count must divide Lz")
        self.dims, self.n = (Lx, Ly, Lz), n_slabs
        self.nz = Lz // n_slabs
        self.e = e
        self.slabs = [hs.Slab(self.dims, k * self.nz, self.nz, J=J, K=K, e=e, precision=precision, seed=seed,
                              replica=replica, stream=stream) for k in range(n_slabs)]
        self.plan = halo_plan(n_slabs)

    def close(self):
        for s in self.slabs:
            s.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def exchange(self, colour: int):
        for src, src_which, dst, dst_which in self.plan:
            hs.hs_slab_copy_plane(self.slabs[dst].h, dst_which, self.slabs[src].h, src_which, colour)

    def init(self, mode=hs.HS_INIT_RANDOM):
        for s in self.slabs:
            s.init(mode)
        self.exchange(0)
        self.exchange(1)

    def set_spins(self, S):
        plane = self.dims[0] * self.dims[1]
        S = np.asarray(S, dtype=np.float64).reshape(self.dims[2], plane, 3)
        for k, s in enumerate(self.slabs):
            s.set_spins(np.ascontiguousarray(S[k * self.nz:(k + 1) * self.nz].reshape(-1, 3)))
        self.exchange(0)
        self.exchange(1)

    def get_spins(self) -> np.ndarray:
        return np.concatenate([s.get_spins() for s in self.slabs])

    def set_sweep_counter(self, n):
        for s in self.slabs:
            s.set_sweep_counter(n)

    def accumulate(self, on=True):
        for s in self.slabs:
            s.accumulate(on)

    def sweep(self, beta, n=1):
        for _ in range(n):
            for c in (0, 1):
                for s in self.slabs:
                    s.sweep_pass(beta, c)
                self.exchange(c)

    def last_observables(self) -> dict:
        """E, M, |M|, ... of the last sweep, from the slabs' fused sums."""
        n_sites = self.dims[0] * self.dims[1] * self.dims[2]
        return combine_sums([s.read_sums() for s in self.slabs], n_sites, self.e)


class _DevicePlane:
    """A device plane as a CUDA array (no copy), for torch.as_tensor."""

    def __init__(self, ptr: int, nbytes: int, dtype):
        itemsize = np.dtype(dtype).itemsize
        self.__cuda_array_interface__ = {"shape": (nbytes // itemsize,), "typestr": np.dtype(dtype).str,
                                         "data": (ptr, False), "version": 3}


class DistributedSlab:
    """One slab per process (rank r of a torch.distributed group of W ranks
    owns planes r nz .. (r+1) nz - 1): halos move by point-to-point sends of
    the device planes, observables by an allreduce of the five sums."""

    _DTYPES = {"fp64": np.float64, "fp32": np.float32, "fp16": np.float16}

    def __init__(self, dims, *, J=1.0, K=0.0, e=(0.0, 0.0, 1.0), precision="fp32", seed=0, replica=0,
                 stream=None):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        Lx, Ly, Lz = (int(d) for d in dims)
        if Lz % self.world:
            raise ValueError("the rank count must divide Lz")
        self.dims, self.e = (Lx, Ly, Lz), e
        self.nz = Lz // self.world
        self.dtype = self._DTYPES[precision]
        self.slab = hs.Slab(self.dims, self.rank * self.nz, self.nz, J=J, K=K, e=e, precision=precision, seed=seed,
                            replica=replica, stream=stream)
        self.stream = stream

    def _plane(self, colour, component, which):
        import torch
        ptr, nbytes = hs.hs_slab_plane(self.slab.h, colour, component, which)
        return torch.as_tensor(_DevicePlane(ptr, nbytes, self.dtype), device="cuda")

    def exchange(self, colour: int):
        import torch
        if self.world == 1:  # the slab is its own periodic neighbour
            for _, src_which, _, dst_which in halo_plan(1):
                hs.hs_slab_copy_plane(self.slab.h, dst_which, self.slab.h, src_which, colour)
            return
        torch.cuda.synchronize()  # the pass has written the planes the sends read
        reqs = []
        for src, src_which, dst, dst_which in halo_plan(self.world):
            for q in range(3):
                if src == self.rank:
                    reqs.append(self.dist.isend(self._plane(colour, q, src_which), dst))
                if dst == self.rank:
                    reqs.append(self.dist.irecv(self._plane(colour, q, dst_which), src))
        for r in reqs:
            r.wait()
        torch.cuda.synchronize()

    def sweep(self, beta, n=1):
        for _ in range(n):
            for c in (0, 1):
                self.slab.sweep_pass(beta, c)
                self.exchange(c)

    def last_observables(self) -> dict:
        import torch
        sums = torch.as_tensor(self.slab.read_sums(), dtype=torch.float64, device="cuda")
        self.dist.all_reduce(sums)
        n_sites = self.dims[0] * self.dims[1] * self.dims[2]
        return combine_sums([sums.cpu().numpy()], n_sites, self.e)

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


class DistributedSlab:
    """One slab per process (rank r of a torch.distributed group of W ranks
    owns planes r nz .. (r+1) nz - 1).

    After each colour pass the slab packs the colour's first and last own
    planes into one message each (hs_slab_pack: the three component planes
    back to back), exchanges them with its two neighbours and unpacks what it
    receives into its halos.  transport "nccl" sends the device buffers with
    stream-ordered NCCL point-to-point operations, so the host never waits for
    the GPU; "host" stages them through host memory for a CPU backend (gloo),
    which synchronises.  "auto" picks "nccl" when the group's backend is NCCL.
    With accumulation on, every sweep's five fused sums are allreduced and the
    whole lattice's E and M moments are added to this slab's accumulator on
    the device (hs_accumulate_sums), so every rank holds the global moments."""

    _DTYPES = {"fp64": "float64", "fp32": "float32", "fp16": "float16"}

    def __init__(self, dims, *, J=1.0, K=0.0, e=(0.0, 0.0, 1.0), precision="fp32", seed=0, replica=0,
                 stream=None, transport="auto"):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        Lx, Ly, Lz = (int(d) for d in dims)
        if Lz % self.world:
            raise ValueError("the rank count must divide Lz")
        if transport == "auto":
            transport = "nccl" if dist.get_backend() == "nccl" else "host"
        if transport not in ("nccl", "host"):
            raise ValueError("transport must be 'auto', 'nccl' or 'host'")
        self.transport = transport
        self.dims, self.e = (Lx, Ly, Lz), e
        self.n_sites = Lx * Ly * Lz
        self.nz = Lz // self.world
        self.stream = stream
        self.slab = hs.Slab(self.dims, self.rank * self.nz, self.nz, J=J, K=K, e=e, precision=precision, seed=seed,
                            replica=replica, stream=stream)
        self.slab.accumulate(False)   # global moments come from the allreduced sums
        self.accumulating = False
        dtype = getattr(torch, self._DTYPES[precision])
        _, plane_bytes = hs.hs_slab_plane(self.slab.h, 0, 0, hs.FIRST_OWN)
        n = 3 * plane_bytes // torch.empty(0, dtype=dtype).element_size()
        dev = torch.device("cuda", torch.cuda.current_device())
        self.buf = {k: torch.empty(n, dtype=dtype, device=dev) for k in ("send_lo", "send_hi", "recv_lo", "recv_hi")}
        self.sums = torch.zeros(5, dtype=torch.float64, device=dev)
        if transport == "host":
            self.hbuf = {k: torch.empty(n, dtype=dtype).pin_memory() for k in self.buf}
            self.hsums = torch.zeros(5, dtype=torch.float64)

    def _stream_ctx(self):
        return self.torch.cuda.stream(self.stream) if self.stream is not None else _nullcontext()

    def init(self, mode=hs.HS_INIT_RANDOM):
        self.slab.init(mode)
        self.exchange(0)
        self.exchange(1)

    def set_spins(self, S_own):
        """This rank's own planes (Lx Ly nz spins in natural order)."""
        self.slab.set_spins(S_own)
        self.exchange(0)
        self.exchange(1)

    def get_spins(self):
        return self.slab.get_spins()

    def set_sweep_counter(self, n):
        self.slab.set_sweep_counter(n)

    def accumulate(self, on=True):
        self.accumulating = bool(on)

    def reset_accumulator(self):
        self.slab.reset_accumulator()

    def read_accumulator(self):
        """The whole lattice's moments (hs_moment order) and sweep count."""
        return self.slab.read_accumulator()

    def exchange(self, colour: int):
        with self._stream_ctx():
            self._exchange(colour)

    def _exchange(self, colour: int):
        h = self.slab.h
        if self.world == 1:  # the slab is its own periodic neighbour
            for _, src_which, _, dst_which in halo_plan(1):
                hs.hs_slab_copy_plane(h, dst_which, h, src_which, colour)
            return
        lo, hi = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        b = self.buf
        hs.hs_slab_pack(h, colour, hs.FIRST_OWN, b["send_lo"])   # -> the halo above of the slab below
        hs.hs_slab_pack(h, colour, hs.LAST_OWN, b["send_hi"])    # -> the halo below of the slab above
        # posting order: sends (to lo, to hi), receives (from hi, from lo); with two ranks lo == hi, and
        # the peer's first message (its first own plane) is the one for this rank's halo above
        if self.transport == "nccl":
            with self._stream_ctx():
                ops = [self.dist.P2POp(self.dist.isend, b["send_lo"], lo),
                       self.dist.P2POp(self.dist.isend, b["send_hi"], hi),
                       self.dist.P2POp(self.dist.irecv, b["recv_hi"], hi),
                       self.dist.P2POp(self.dist.irecv, b["recv_lo"], lo)]
                for r in self.dist.batch_isend_irecv(ops):
                    r.wait()   # the current stream waits on the transfers; the host does not
        else:
            hb = self.hbuf
            for k in ("send_lo", "send_hi"):
                hb[k].copy_(b[k])
            reqs = [self.dist.isend(hb["send_lo"], lo, tag=0), self.dist.isend(hb["send_hi"], hi, tag=1),
                    self.dist.irecv(hb["recv_hi"], hi, tag=0), self.dist.irecv(hb["recv_lo"], lo, tag=1)]
            for r in reqs:
                r.wait()
            for k in ("recv_hi", "recv_lo"):
                b[k].copy_(hb[k])
        hs.hs_slab_unpack(h, colour, hs.HALO_ABOVE, b["recv_hi"])
        hs.hs_slab_unpack(h, colour, hs.HALO_BELOW, b["recv_lo"])

    def _accumulate_sweep(self):
        h = self.slab.h
        hs.hs_read_sums_device(h, self.sums)
        if self.transport == "nccl":
            with self._stream_ctx():
                self.dist.all_reduce(self.sums)
        else:
            self.hsums.copy_(self.sums)
            self.dist.all_reduce(self.hsums)
            self.sums.copy_(self.hsums)
        hs.hs_accumulate_sums(h, self.sums, self.n_sites)

    def sweep(self, beta, n=1):
        with self._stream_ctx():
            for _ in range(n):
                for c in (0, 1):
                    self.slab.sweep_pass(beta, c)
                    self._exchange(c)
                if self.accumulating:
                    self._accumulate_sweep()

    def last_observables(self) -> dict:
        """E, M, |M|, ... of the last sweep of the whole lattice (host)."""
        sums = self.torch.as_tensor(self.slab.read_sums(), dtype=self.torch.float64)
        if self.transport == "nccl":
            sums = sums.cuda()
        self.dist.all_reduce(sums)
        return combine_sums([sums.cpu().numpy()], self.n_sites, self.e)

    def close(self):
        self.slab.close()


class _nullcontext:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

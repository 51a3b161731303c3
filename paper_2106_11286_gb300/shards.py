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

With ``overlap=True`` both update the boundary planes first
(hs_sweep_pass_part): once a colour's first and last own planes are final,
their exchange runs on a communication stream while the interior planes are
updated on the compute stream, and the next colour pass waits for both.  The
chain is the same bit for bit: a colour pass reads only the other colour, so
the order of its planes does not matter.
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


class _Overlap:
    """The compute stream of a set of slabs (their own), a communication
    stream for their halo copies, and the two events that order them."""

    def __init__(self, stream):
        import torch
        self.compute = stream if stream is not None else torch.cuda.default_stream()
        self.comm = torch.cuda.Stream()
        self.ev_ready, self.ev_done = torch.cuda.Event(), torch.cuda.Event()

    def begin(self):
        """The communication stream waits for the compute stream's work so far."""
        self.ev_ready.record(self.compute)
        self.comm.wait_event(self.ev_ready)

    def end(self):
        """The compute stream waits for the communication stream's work so far."""
        self.ev_done.record(self.comm)
        self.compute.wait_event(self.ev_done)


class ShardedLattice:
    """A periodic sc lattice as ``n_slabs`` z-slabs on the current device,
    halos exchanged by device copies between colour passes (on a separate
    stream, beside the interior update, with ``overlap=True``)."""

    def __init__(self, dims, n_slabs: int, *, J=1.0, K=0.0, e=(0.0, 0.0, 1.0), precision="fp32", seed=0,
                 replica=0, stream=None, overlap=False):
        Lx, Ly, Lz = (int(d) for d in dims)
        if n_slabs < 1 or Lz % n_slabs:
            raise ValueError("the slab count must divide Lz")
        self.dims, self.n = (Lx, Ly, Lz), n_slabs
        self.nz = Lz // n_slabs
        self.e = e
        self.slabs = [hs.Slab(self.dims, k * self.nz, self.nz, J=J, K=K, e=e, precision=precision, seed=seed,
                              replica=replica, stream=stream) for k in range(n_slabs)]
        self.plan = halo_plan(n_slabs)
        self.ov = _Overlap(stream) if overlap else None
        if self.ov is not None:
            for s in self.slabs:
                s.set_comm_stream(self.ov.comm)

    def close(self):
        if self.ov is not None:
            self.ov.comm.synchronize()   # no halo copy in flight when the planes are freed
        for s in self.slabs:
            s.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _copies(self, colour: int):
        for src, src_which, dst, dst_which in self.plan:
            hs.hs_slab_copy_plane(self.slabs[dst].h, dst_which, self.slabs[src].h, src_which, colour)

    def exchange(self, colour: int):
        """The halo copies of one colour, ordered after the work so far and
        before the work that follows."""
        if self.ov is None:
            self._copies(colour)
            return
        self.ov.begin()
        self._copies(colour)
        self.ov.end()

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
                if self.ov is None:
                    for s in self.slabs:
                        s.sweep_pass(beta, c)
                    self._copies(c)
                    continue
                for s in self.slabs:
                    s.sweep_part(beta, c, hs.HS_PART_BOUNDARY)
                self.ov.begin()
                self._copies(c)          # boundary planes -> halos, beside the interior update
                for s in self.slabs:
                    s.sweep_part(beta, c, hs.HS_PART_INTERIOR)
                self.ov.end()

    def last_observables(self) -> dict:
        """E, M, |M|, ... of the last sweep, from the slabs' fused sums."""
        n_sites = self.dims[0] * self.dims[1] * self.dims[2]
        return combine_sums([s.read_sums() for s in self.slabs], n_sites, self.e)


class DistributedSlab:
    """One slab per process (rank r of a torch.distributed group of W ranks
    owns planes r nz .. (r+1) nz - 1; without a process group, one slab
    that is its own periodic neighbour).

    After each colour pass the slab packs the colour's first and last own
    planes into one message each (hs_slab_pack: the three component planes
    back to back), exchanges them with its two neighbours and unpacks what it
    receives into its halos.  transport "nccl" sends the device buffers with
    stream-ordered NCCL point-to-point operations, so the host never waits for
    the GPU; "host" stages them through host memory for a CPU backend (gloo),
    which synchronises.  "auto" picks "nccl" when the group's backend is NCCL.
    With accumulation on, every sweep's five fused sums are allreduced and the
    whole lattice's E and M moments are added to this slab's accumulator on
    the device (hs_accumulate_sums), so every rank holds the global moments.

    overlap=True updates the two boundary planes first and runs the exchange
    (pack, transfer, unpack) on a communication stream while the interior
    planes are updated; with the host transport the interior update is
    queued before the host waits for the boundary messages.  reserve_ctas
    leaves that many CTAs of the interior update unlaunched, so the copy and
    NCCL kernels find free SMs beside it."""

    _DTYPES = {"fp64": "float64", "fp32": "float32", "fp16": "float16"}

    def __init__(self, dims, *, J=1.0, K=0.0, e=(0.0, 0.0, 1.0), precision="fp32", seed=0, replica=0,
                 stream=None, transport="auto", overlap=False, reserve_ctas=0):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        grouped = dist.is_available() and dist.is_initialized()
        # without a process group: one slab, its own periodic neighbour, no collective
        self.rank, self.world = (dist.get_rank(), dist.get_world_size()) if grouped else (0, 1)
        Lx, Ly, Lz = (int(d) for d in dims)
        if Lz % self.world:
            raise ValueError("the rank count must divide Lz")
        if transport == "auto":
            transport = "nccl" if grouped and dist.get_backend() == "nccl" else "host"
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
        self.ov = _Overlap(stream) if overlap else None
        if self.ov is not None:
            self.slab.set_comm_stream(self.ov.comm)
        if reserve_ctas:
            self.slab.reserve_ctas(reserve_ctas)

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
        """The halo exchange of one colour, ordered after the work so far and
        before the work that follows."""
        if self.ov is None:
            with self._stream_ctx():
                self._exchange(colour)
            return
        self.ov.begin()
        with self.torch.cuda.stream(self.ov.comm):
            self._exchange(colour)
        self.ov.end()

    def _exchange(self, colour: int, interior=None):
        """Pack, transfer and unpack one colour's boundary planes on the
        current stream (the slab's communication stream when it has one).
        interior: queued on the compute stream once the host needs the GPU
        no more before it blocks (the host transport's overlap)."""
        h = self.slab.h
        if self.world == 1:  # the slab is its own periodic neighbour
            for _, src_which, _, dst_which in halo_plan(1):
                hs.hs_slab_copy_plane(h, dst_which, h, src_which, colour)
            if interior is not None:
                interior()
            return
        lo, hi = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        b = self.buf
        hs.hs_slab_pack(h, colour, hs.FIRST_OWN, b["send_lo"])   # -> the halo above of the slab below
        hs.hs_slab_pack(h, colour, hs.LAST_OWN, b["send_hi"])    # -> the halo below of the slab above
        # posting order: sends (to lo, to hi), receives (from hi, from lo); with two ranks lo == hi, and
        # the peer's first message (its first own plane) is the one for this rank's halo above
        if self.transport == "nccl":
            if interior is not None:
                interior()
            ops = [self.dist.P2POp(self.dist.isend, b["send_lo"], lo),
                   self.dist.P2POp(self.dist.isend, b["send_hi"], hi),
                   self.dist.P2POp(self.dist.irecv, b["recv_hi"], hi),
                   self.dist.P2POp(self.dist.irecv, b["recv_lo"], lo)]
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()   # the current stream waits on the transfers; the host does not
        else:
            hb = self.hbuf
            cur = self.torch.cuda.current_stream()
            for k in ("send_lo", "send_hi"):
                hb[k].copy_(b[k], non_blocking=True)
            if interior is not None:
                interior()
            cur.synchronize()
            reqs = [self.dist.isend(hb["send_lo"], lo, tag=0), self.dist.isend(hb["send_hi"], hi, tag=1),
                    self.dist.irecv(hb["recv_hi"], hi, tag=0), self.dist.irecv(hb["recv_lo"], lo, tag=1)]
            for r in reqs:
                r.wait()
            for k in ("recv_hi", "recv_lo"):
                b[k].copy_(hb[k], non_blocking=True)
        hs.hs_slab_unpack(h, colour, hs.HALO_ABOVE, b["recv_hi"])
        hs.hs_slab_unpack(h, colour, hs.HALO_BELOW, b["recv_lo"])

    def _accumulate_sweep(self):
        h = self.slab.h
        hs.hs_read_sums_device(h, self.sums)
        if self.world == 1:
            pass
        elif self.transport == "nccl":
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
                    if self.ov is None:
                        self.slab.sweep_pass(beta, c)
                        self._exchange(c)
                        continue
                    self.slab.sweep_part(beta, c, hs.HS_PART_BOUNDARY)
                    self.ov.begin()
                    with self.torch.cuda.stream(self.ov.comm):
                        self._exchange(c, interior=lambda c=c: self.slab.sweep_part(beta, c, hs.HS_PART_INTERIOR))
                    self.ov.end()
                if self.accumulating:
                    self._accumulate_sweep()

    def last_observables(self) -> dict:
        """E, M, |M|, ... of the last sweep of the whole lattice (host)."""
        sums = self.torch.as_tensor(self.slab.read_sums(), dtype=self.torch.float64)
        if self.world > 1:
            if self.transport == "nccl":
                sums = sums.cuda()
            self.dist.all_reduce(sums)
        return combine_sums([sums.cpu().numpy()], self.n_sites, self.e)

    def close(self):
        if self.ov is not None:
            self.ov.comm.synchronize()
        self.slab.close()


class _nullcontext:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

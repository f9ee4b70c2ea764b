"""x-slab decomposition of one channel over several ranks (one GPU each).

The channel's x columns are cut into consecutive slabs; each rank steps its
slab with its own library handle (lbm_set_slab), and before every step the
halo -- the five populations per face that stream across a cut -- moves
between neighbouring ranks (lbm_halo_pack / lbm_halo_unpack around a
point-to-point exchange).  The statistics, summed per (x, y) column over z, are
assembled by one all-reduce.  With the halo moved exactly, every rank's owned
columns are bit for bit those of the undivided channel.

Transports: `P2PTransport` moves the buffers with torch.distributed
point-to-point operations between ranks -- device buffers under NCCL, or
staged through host memory under gloo; `LocalTransport` connects slabs that
live in one process (tests on one GPU).  The library does no communication
itself.
"""
import ctypes as ct

import numpy as np

from . import _abi
from .channel import LBMChannel

GHOST = 4          # ghost columns per side with a neighbour (keeps local widths a multiple of 4)


def split(nx, nranks, quantum=4):
    """Owned global column ranges [(lo, hi)] of nranks slabs: as equal as
    possible, every cut at a multiple of `quantum`."""
    if nx % quantum or nx // quantum < nranks:
        raise ValueError(f"nx = {nx} cannot be cut into {nranks} slabs of multiples of {quantum}")
    units = nx // quantum
    bounds = [quantum * (units * r // nranks) for r in range(nranks + 1)]
    return [(bounds[r], bounds[r + 1]) for r in range(nranks)]


class SlabChannel:
    """Rank `rank` of `nranks`: the slab of the nx x ny x nz channel it owns.
    Other keyword arguments go to LBMChannel (the same on every rank: the
    same STG draws, storage and options)."""

    def __init__(self, nx, ny, nz, rank, nranks, transport, ghost=GHOST, **kw):
        import torch
        self.nx_global, self.ny, self.nz = nx, ny, nz
        self.rank, self.nranks = rank, nranks
        self.lo, self.hi = split(nx, nranks)[rank]
        self.left, self.right = rank > 0, rank < nranks - 1
        gl, gr = (ghost if self.left else 0), (ghost if self.right else 0)
        self.nx_local = gl + (self.hi - self.lo) + gr
        self.own = (gl, gl + self.hi - self.lo)           # owned local columns
        self.ch = LBMChannel(self.nx_local, ny, nz, **kw)
        self.lib, self.h = self.ch.lib, self.ch.h
        _abi.check(self.lib.lbm_set_slab(self.h, nx, self.lo - gl, *self.own), "lbm_set_slab")
        nb = ct.c_size_t()
        _abi.check(self.lib.lbm_halo_bytes(self.h, ct.byref(nb)), "lbm_halo_bytes")
        mk = lambda: torch.empty(nb.value, dtype=torch.uint8, device=self.ch.device)   # noqa: E731
        self.send = {f: mk() for f, on in ((0, self.left), (1, self.right)) if on}
        self.recv = {f: mk() for f in self.send}
        self.transport = transport
        transport.attach(self)

    # ---- one step: halo in, then the step ----
    def pack(self):
        for f, buf in self.send.items():
            _abi.check(self.lib.lbm_halo_pack(self.h, f, ct.c_void_p(buf.data_ptr())), "lbm_halo_pack")

    def unpack(self):
        for f, buf in self.recv.items():
            _abi.check(self.lib.lbm_halo_unpack(self.h, f, ct.c_void_p(buf.data_ptr())), "lbm_halo_unpack")

    def step(self, n=1):
        for _ in range(int(n)):
            self.pack()
            self.transport.exchange(self)
            self.unpack()
            self.ch.step(1)

    def set_sponge(self, cells, nu_max):
        self.ch.set_sponge(cells, nu_max)

    # ---- results on the owned columns ----
    def fields(self):
        rho, u = self.ch.fields()
        a, b = self.own
        return rho[..., a:b], u[:, :, a:b, :]

    def populations(self):
        a, b = self.own
        return self.ch.populations()[..., a:b]

    def stats(self, all_reduce=None):
        """The statistics of the whole channel: (sums [ny][nx][7], utau sums
        [2][nx], samples).  Each rank fills its owned columns; `all_reduce`
        (a callable summing a float64 numpy array over the ranks, in place)
        assembles them -- one call."""
        s, ut, n = self.ch.stats()
        a, b = self.own
        flat = np.zeros(self.ny * self.nx_global * 7 + 2 * self.nx_global)
        S = flat[:self.ny * self.nx_global * 7].reshape(self.ny, self.nx_global, 7)
        U = flat[self.ny * self.nx_global * 7:].reshape(2, self.nx_global)
        S[:, self.lo:self.hi, :] = s[:, a:b, :]
        U[:, self.lo:self.hi] = ut[:, a:b]
        if all_reduce is not None:
            all_reduce(flat)
        return S, U, n

    def sync(self):
        self.ch.sync()

    def close(self):
        self.ch.close()


class LocalTransport:
    """Slabs of one process: the exchange copies each slab's send buffers
    into its neighbours' receive buffers (device to device).  step_all runs
    one step of every slab, halos first."""

    def __init__(self):
        self.slabs = {}

    def attach(self, s):
        self.slabs[s.rank] = s

    def exchange(self, s):
        raise RuntimeError("slabs of one process step together: use LocalTransport.step_all")

    def step_all(self, n=1):
        ranks = sorted(self.slabs)
        for _ in range(int(n)):
            for r in ranks:
                self.slabs[r].pack()
            for r in ranks:
                s = self.slabs[r]
                if s.left:
                    s.recv[0].copy_(self.slabs[r - 1].send[1])
                if s.right:
                    s.recv[1].copy_(self.slabs[r + 1].send[0])
            for r in ranks:
                self.slabs[r].unpack()
                self.slabs[r].ch.step(1)


class P2PTransport:
    """Point-to-point exchange with the neighbouring ranks of a
    torch.distributed process group (rank r's slab neighbours are ranks r - 1
    and r + 1).  With a backend that takes device tensors (NCCL) the device
    buffers are sent as they are; otherwise (gloo) through host copies."""

    def __init__(self, device_buffers):
        self.device_buffers = device_buffers
        self.host = {}

    def attach(self, s):
        import torch
        if not self.device_buffers:
            self.host = {k: (torch.empty_like(v, device="cpu"), torch.empty_like(v, device="cpu"))
                         for k, v in s.send.items()}

    def exchange(self, s):
        import torch
        import torch.distributed as dist
        peer = {0: s.rank - 1, 1: s.rank + 1}
        if self.device_buffers:
            ops = []
            for f in s.send:
                ops.append(dist.P2POp(dist.isend, s.send[f], peer[f]))
                ops.append(dist.P2POp(dist.irecv, s.recv[f], peer[f]))
            for w in dist.batch_isend_irecv(ops) if ops else []:
                w.wait()
            return
        if any(b.is_cuda for b in s.send.values()):
            torch.cuda.current_stream(s.send[next(iter(s.send))].device).synchronize()   # the packs are done
        for f in s.send:
            self.host[f][0].copy_(s.send[f])
        reqs = []
        for f in s.send:
            reqs.append(dist.isend(self.host[f][0], peer[f]))
            reqs.append(dist.irecv(self.host[f][1], peer[f]))
        for r in reqs:
            r.wait()
        for f in s.send:
            s.recv[f].copy_(self.host[f][1], non_blocking=False)

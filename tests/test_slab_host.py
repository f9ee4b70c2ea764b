"""Host logic of the x-slab decomposition on the CPU: the column split, the
point-to-point halo exchange between neighbouring ranks over gloo (world sizes
2 and 3, buffers staged through host memory), and the assembly of the whole
channel's statistics by one all-reduce."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_cuts_at_multiples_of_four():
    sys.path.insert(0, ROOT)
    from paper_2304_04214_gb300.slab import split
    assert split(96, 1) == [(0, 96)]
    assert split(96, 3) == [(0, 32), (32, 64), (64, 96)]
    assert split(1536, 8)[3] == (576, 768)
    parts = split(100, 3)
    assert parts[0][0] == 0 and parts[-1][1] == 100
    assert all(a % 4 == 0 and b % 4 == 0 and b > a for a, b in parts)
    assert all(parts[r][1] == parts[r + 1][0] for r in range(2))
    with pytest.raises(ValueError):
        split(98, 2)                        # not a multiple of four
    with pytest.raises(ValueError):
        split(8, 3)                         # fewer units than ranks


class _FakeCh:
    def __init__(self, nx_local, ny, own, value):
        self.nx_local, self.ny, self.own, self.value = nx_local, ny, own, value

    def stats(self):
        s = np.full((self.ny, self.nx_local, 7), -1.0)      # ghost columns: not to be used
        a, b = self.own
        s[:, a:b, :] = self.value
        ut = np.full((2, self.nx_local), -1.0)
        ut[:, a:b] = 10 * self.value
        return s, ut, 5


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2304_04214_gb300.slab import P2PTransport, SlabChannel, split
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    s = object.__new__(SlabChannel)              # the slab's host side, no library handle
    s.rank, s.nranks = rank, ws
    s.left, s.right = rank > 0, rank < ws - 1
    s.send = {f: torch.full((64,), 16 * rank + f, dtype=torch.uint8) for f, on in ((0, s.left), (1, s.right)) if on}
    s.recv = {f: torch.zeros(64, dtype=torch.uint8) for f in s.send}
    tr = P2PTransport(device_buffers=False)
    tr.attach(s)
    tr.exchange(s)
    got = {f: int(v[0]) for f, v in s.recv.items()} if all(bool((v == v[0]).all()) for v in s.recv.values()) else None
    # statistics: owned columns of every rank assembled by one all-reduce
    nx, ny = 24, 3
    s.nx_global, s.ny = nx, ny
    s.lo, s.hi = split(nx, ws)[rank]
    gl = 4 if s.left else 0
    s.own = (gl, gl + s.hi - s.lo)
    s.ch = _FakeCh(gl + s.hi - s.lo + (4 if s.right else 0), ny, s.own, float(rank + 1))

    def all_reduce(a):
        t = torch.from_numpy(a)
        dist.all_reduce(t)

    S, U, n = s.stats(all_reduce)
    q.put((rank, got, S[0, :, 0].tolist(), U[1].tolist(), n))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_halo_exchange_and_statistics_over_gloo(ws):
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    ps = [mp.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in ps:
        p.start()
    res = {r: (got, S, U, n) for r, got, S, U, n in (q.get(timeout=120) for _ in ps)}
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2304_04214_gb300.slab import split  # noqa: E402 (ROOT on the path via conftest)
    want_S = np.concatenate([np.full(b - a, r + 1.0) for r, (a, b) in enumerate(split(24, ws))])
    for r in range(ws):
        got, S, U, n = res[r]
        exp = {}
        if r > 0:
            exp[0] = 16 * (r - 1) + 1            # the left neighbour's right-face buffer
        if r < ws - 1:
            exp[1] = 16 * (r + 1) + 0            # the right neighbour's left-face buffer
        assert got == exp, (r, got)
        assert np.array_equal(S, want_S) and np.array_equal(U, 10 * want_S) and n == 5

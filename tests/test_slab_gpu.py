"""x-slab decomposition on one GPU: the channel cut into two or three slabs
(one library handle each, halos moved before every step) against the same
channel undivided -- owned populations, friction velocities and the assembled
statistics bit for bit -- and against the FP64 oracle, inlet and outlet
included.  Also two processes with a host-staged gloo transport (the
transport of a CPU-only process group): the kernels of the two processes never
wait on each other, the host moves the halos between steps."""
import os

import numpy as np
import pytest

from oracle.oracle import Oracle, default_config
from paper_2304_04214_gb300.inputs import stg_uniforms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _whole(nx, ny, nz, **kw):
    from paper_2304_04214_gb300.channel import LBMChannel
    return LBMChannel(nx, ny, nz, **kw)


@pytest.mark.parametrize("nranks,precision,sponge", [(2, "fp32", None), (3, "fp16", (40, 0.05)),
                                                      (3, "bf16", None), (2, "fp16row", None),
                                                      (2, "fp32", (48, 0.05))])
def test_slabs_are_bit_identical_to_the_undivided_channel(nranks, precision, sponge):
    from paper_2304_04214_gb300.slab import LocalTransport, SlabChannel
    nx, ny, nz, N, seed = 96, 16, 8, 16, 5
    kw = dict(re_tau=1000.0, n_modes=N, uniforms=stg_uniforms(N, seed), precision=precision, stats_every=3)
    ref = _whole(nx, ny, nz, **kw)
    tr = LocalTransport()
    slabs = [SlabChannel(nx, ny, nz, r, nranks, tr, **kw) for r in range(nranks)]
    if sponge:
        ref.set_sponge(*sponge)
        for s in slabs:
            s.set_sponge(*sponge)
    ref.set_graphs(False)
    ref.step(150)
    tr.step_all(150)
    f = ref.populations()
    ut = ref.utau()
    S, U, n = ref.stats()
    Sg, Ug = np.zeros_like(S), np.zeros_like(U)
    for s in slabs:
        a, b = s.own
        assert np.array_equal(s.populations(), f[..., s.lo:s.hi]), (s.rank, precision)
        assert np.array_equal(s.ch.utau()[..., a:b], ut[..., s.lo:s.hi]), s.rank
        Ss, Us, ns = s.stats()
        assert ns == n == 50
        Sg += Ss
        Ug += Us
    assert np.array_equal(Sg, S) and np.array_equal(Ug, U)
    for s in slabs:
        s.close()
    ref.close()


def test_slabs_match_the_oracle_inlet_and_outlet_included():
    """200 steps of three slabs against the oracle's undivided channel (FP32
    storage: 1e-3 after 200 steps, the stated bar)."""
    from paper_2304_04214_gb300.slab import LocalTransport, SlabChannel
    nx, ny, nz, N, seed = 96, 16, 8, 16, 6
    un = stg_uniforms(N, seed)
    o = Oracle(default_config(nx, ny, nz, re_tau=1000.0, n_modes=N), uniforms=un)
    tr = LocalTransport()
    slabs = [SlabChannel(nx, ny, nz, r, 3, tr, re_tau=1000.0, n_modes=N, uniforms=un) for r in range(3)]
    o.step(200)
    tr.step_all(200)
    ro, uo = o.fields()
    rg = np.concatenate([s.fields()[0] for s in slabs], axis=-1)
    ug = np.concatenate([s.fields()[1] for s in slabs], axis=2)
    assert np.max(np.abs(rg - ro)) < 1e-3 * np.max(np.abs(ro))
    assert np.max(np.abs(ug - uo)) < 1e-3 * np.max(np.abs(uo))
    for s in slabs:
        s.close()


def _two_process_rank(rank, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    torch.cuda.set_device(0)
    from paper_2304_04214_gb300.slab import P2PTransport, SlabChannel
    nx, ny, nz, N, seed = 96, 16, 8, 16, 5
    s = SlabChannel(nx, ny, nz, rank, 2, P2PTransport(device_buffers=False), re_tau=1000.0, n_modes=N,
                    uniforms=stg_uniforms(N, seed), stats_every=3, device="cuda:0")

    def all_reduce(a):
        t = torch.from_numpy(a)
        dist.all_reduce(t)
        a[:] = t.numpy()

    s.step(200)
    S, U, n = s.stats(all_reduce)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), f=s.populations(), S=S, U=U, n=n)
    s.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_with_host_staged_transport(tmp_path):
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    mp.start_processes(_two_process_rank, args=(port, str(tmp_path)), nprocs=2, start_method="spawn")
    nx, ny, nz, N, seed = 96, 16, 8, 16, 5
    ref = _whole(nx, ny, nz, re_tau=1000.0, n_modes=N, uniforms=stg_uniforms(N, seed), stats_every=3)
    ref.set_graphs(False)
    ref.step(200)
    f = ref.populations()
    S, U, n = ref.stats()
    got = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    assert np.array_equal(np.concatenate([g["f"] for g in got], axis=-1), f)
    for g in got:                 # every rank holds the whole channel's statistics
        assert int(g["n"]) == n and np.array_equal(g["S"], S) and np.array_equal(g["U"], U)
    ref.close()

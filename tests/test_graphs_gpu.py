"""lbm_step launches whole STG ring periods (64 steps here) as CUDA graphs.
A graph replays launch parameters captured from the host state at the start
of its period, so these tests hold graph and separate launches to bit
identity over runs that cross many periods, with the statistics phase, the
timing phase, the parameters, the sponge and the inlet profile changing in
between, and check the host bookkeeping that replays advance (time, samples,
launch counts, timed launches)."""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pair(precision, **kw):
    from paper_2304_04214_gb300.channel import LBMChannel
    a = LBMChannel(128, 32, 16, n_modes=32, seed=21, precision=precision, stats_every=10, **kw)
    b = LBMChannel(128, 32, 16, n_modes=32, seed=21, precision=precision, stats_every=10, **kw)
    b.set_graphs(False)
    return a, b


def _same(a, b):
    a.sync()
    b.sync()
    assert a.time == b.time
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.utau(), b.utau())
    sa, ua, na = a.stats()
    sb, ub, nb = b.stats()
    assert na == nb
    assert np.array_equal(sa, sb) and np.array_equal(ua, ub)


@pytest.mark.parametrize("precision", ["fp32", "fp16", "fp16row"])
def test_graph_periods_are_bit_identical_to_separate_launches(precision):
    a, b = _pair(precision)
    for n in (300, 1, 399, 64, 128):
        a.step(n)
        b.step(n)
    _same(a, b)
    on, n = a.graph_info()
    assert on and n == 9                  # the whole periods (3 + 5 + 0 + 1) ran as graphs
    assert b.graph_info() == (False, 0)
    a.close()
    b.close()


def test_graphs_follow_parameter_sponge_and_profile_changes():
    a, b = _pair("fp32")
    dp = lambda x: x.ctypes.data_as(ct.POINTER(ct.c_double))   # noqa: E731
    U, R = np.empty(a.ny), np.empty(6 * a.ny)
    a.lib.lbm_get_inlet_profile(a.h, dp(U), dp(R))
    for c in (a, b):
        c.step(200)
        c.set_params([0.5, 1.2, 0.41, 7.6])
        c.step(200)
        c.set_sponge(16, 0.05)
        c.step(200)
        assert c.lib.lbm_set_inlet_profile(c.h, dp(U * 1.01), dp(R * 0.95)) == 0
        c.step(200)
        c.reset_stats()
        c.step(150)
    _same(a, b)
    a.close()
    b.close()


def test_graph_replays_keep_the_instrumentation_counts():
    """Separately launched steps are timed every 16th step, a graph as a whole
    for its 64 steps; all launches are counted alike (plus the graph's time
    setter), and the per-step times agree."""
    a, b = _pair("fp32")
    res = []
    for c in (a, b):
        c.step(70)
        c.sync()
        assert c.lib.lbm_profile_enable(c.h, 16) == 0
        ms, nk, nall = ct.c_double(), ct.c_long(), ct.c_long()
        c.lib.lbm_profile_read(c.h, ct.byref(ms), ct.byref(nk), ct.byref(nall))
        c.step(640)
        c.lib.lbm_profile_read(c.h, ct.byref(ms), ct.byref(nk), ct.byref(nall))
        res.append((ms.value, nk.value, nall.value))
    (ma, ka, la), (mb, kb, lb) = res
    graphs = a.graph_info()[1]
    assert graphs == 9                    # the periods starting at t = 128, 192, ..., 640
    assert kb == 40 and la == lb + graphs
    assert ka == 4 + 64 * graphs          # t = 70, 86, 102, 118 separately, then the graphs
    assert 0.5 < (ma / ka) / (mb / kb) < 2.0
    _same(a, b)
    a.close()
    b.close()


def test_adjoint_windows_between_graph_periods():
    """An adjoint window (its own forward steps, checkpoints and the STG work
    on the second stream) between graph periods: J, dJ/dtheta (to the
    rounding of its atomic sums) and the state after the steps that follow are
    the same as without graphs."""
    a, b = _pair("fp32")
    out = []
    for c in (a, b):
        c.step(200)
        J, dJ = c.adjoint_step(64, 8, (24, 48, 40))
        c.step(200)
        out.append((J, dJ))
    # J from the same forward states; dJ/dtheta sums FP64 atomics, whose
    # order varies from run to run
    assert out[0][0] == out[1][0]
    assert np.allclose(out[0][1], out[1][1], rtol=1e-9, atol=0)
    assert a.graph_info()[1] >= 4
    _same(a, b)
    a.close()
    b.close()


def test_wall_shear_after_graph_periods():
    """The asynchronous wall-shear reduction right after steps that ran as a
    graph reads the forces of the graph's last step: it equals the
    synchronous reduction and the same call after separate launches."""
    import torch
    a, b = _pair("fp32")
    outs = []
    for c in (a, b):
        c.step(192)                       # two periods as graphs in a
        pinned = torch.empty(2 * c.nx, dtype=torch.float64).pin_memory()
        c.wall_shear_async(pinned)
        c.sync()
        outs.append((pinned.numpy().copy(), c.wall_shear().reshape(-1)))
    assert a.graph_info()[1] == 2
    assert np.array_equal(outs[0][0], outs[0][1])
    assert np.array_equal(outs[0][0], outs[1][0])
    a.close()
    b.close()

"""Checkpoint files (lbm_save / lbm_load): a run saved at one step and resumed
in a second channel created alike continues bit for bit like the run that
never stopped -- populations, u_tau and the statistics -- and a corrupted,
truncated or foreign file is refused without changing the channel."""
import numpy as np
import pytest

from paper_2304_04214_gb300.inputs import stg_uniforms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _channel(precision="fp32", nz=6, seed=3):
    from paper_2304_04214_gb300.channel import LBMChannel
    return LBMChannel(72, 16, nz, n_modes=24, uniforms=stg_uniforms(24, seed), precision=precision,
                      stats_every=3)


def _custom_profile(ch):
    import ctypes as ct
    U = np.empty(ch.ny)
    R = np.empty(6 * ch.ny)
    dp = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))   # noqa: E731
    ch.lib.lbm_get_inlet_profile(ch.h, dp(U), dp(R))
    U *= 1.02
    R *= 0.9
    ch.lib.lbm_set_inlet_profile(ch.h, dp(U), dp(R))


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16", "fp16row"])
def test_resume_is_bit_identical(tmp_path, precision):
    a = _channel(precision)
    _custom_profile(a)
    a.set_sponge(12, 0.05)            # restored from the file too
    a.step(7)
    path = tmp_path / "a.lbm"
    a.save(path)
    a.step(9)
    b = _channel(precision)
    b.step(2)                       # some other state, to be overwritten
    b.load(path)
    assert b.time == 7
    b.step(9)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.utau(), b.utau())
    sa, ua, na = a.stats()
    sb, ub, nb = b.stats()
    assert na == nb == 5 and np.array_equal(sa, sb) and np.array_equal(ua, ub)


def test_bad_files_are_refused_and_change_nothing(tmp_path):
    from paper_2304_04214_gb300 import _abi
    a = _channel()
    a.step(4)
    good = tmp_path / "good.lbm"
    a.save(good)
    raw = good.read_bytes()
    b = _channel()
    b.step(3)
    before = b.populations()
    cases = {"corrupt": raw[:-100] + bytes([raw[-100] ^ 1]) + raw[-99:], "truncated": raw[:len(raw) // 2],
             "foreign": b"not a checkpoint" * 64}
    for name, data in cases.items():
        p = tmp_path / f"{name}.lbm"
        p.write_bytes(data)
        assert b.lib.lbm_load(b.h, str(p).encode()) == _abi.LBM_EINVAL, name
    # a channel created differently (other grid, other STG draws) refuses a good file
    for other in (_channel(nz=8), _channel(seed=4)):
        assert other.lib.lbm_load(other.h, str(good).encode()) == _abi.LBM_EINVAL
    assert b.lib.lbm_load(b.h, str(tmp_path / "missing.lbm").encode()) == _abi.LBM_EINVAL
    assert np.array_equal(b.populations(), before) and b.time == 3


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_load_right_after_steps_needs_no_sync(tmp_path, precision):
    """lbm_load directly after lbm_step, with the steps (and a wall-shear
    reduction on the side stream, an STG refill on the second stream) still in
    flight: the load waits for them, so what it restores is not overwritten
    and the next steps match the run that saved, bit for bit."""
    import torch
    a = _channel(precision)
    a.step(5)
    path = tmp_path / "a.lbm"
    a.save(path)
    a.step(70)                      # across an STG ring period
    b = _channel(precision)
    b.step(130)                     # many steps enqueued, none waited for
    b.wall_shear_async(torch.empty(2 * b.nx, dtype=torch.float64).pin_memory())
    b.load(path)
    b.step(70)
    assert b.time == 75
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.utau(), b.utau())
    sa, ua, na = a.stats()
    sb, ub, nb = b.stats()
    assert na == nb and np.array_equal(sa, sb) and np.array_equal(ua, ub)

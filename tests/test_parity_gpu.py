"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (max-norm error normalized by the oracle's max |.|):
  FP32 storage  1e-5 after one step, 1e-3 after 200 steps.
  FP16 deviations: the stored deviation f - w (|f - w| <~ 5e-3) carries a
    relative rounding error of 2^-11, i.e. <~ 2.5e-6 absolute per population;
    summed over the ten populations that make up a velocity component this is
    <~ 2.5e-5 absolute against |u| ~ 0.06, so 1e-3 after one step.
  BF16 deviations: 2^-8 relative, eight times more: 8e-3 after one step.
  Over n steps the rounding errors add like a random walk: the half-precision
    tolerances grow with sqrt(n) (x 14 at 200 steps).
"""
import math

import numpy as np
import pytest

from gpu_helpers import field_errors, make_pair, set_both
from paper_2304_04214_gb300.inputs import noise

pytestmark = pytest.mark.gpu

TOL1 = {"fp32": 1e-5, "fp16": 1e-3, "bf16": 8e-3, "fp16row": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("shape", [(64, 32, 32), (70, 16, 6)])
def test_first_step_from_the_library_init(shape):
    """Each side builds its own tables and initial state; one step agrees."""
    o, g = make_pair(*shape, n_modes=32, seed=3)
    o.step(1)
    g.step(1)
    er, eu = field_errors(o, g)
    assert er < 1e-5 and eu < 1e-5, (er, eu)
    ut_o, ut_g = o.utau(), g.utau()
    assert np.max(np.abs(ut_g - ut_o)) < 1e-5 * np.max(ut_o)


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16", "fp16row"])
@pytest.mark.parametrize("inlet", [1, 0])
def test_one_step_perturbed_state(precision, inlet):
    """Non-equilibrium state (2% noise on every population): every term of the
    collision, the SGS closure, the wall model and the inlet is active."""
    nx, ny, nz = 70, 16, 6
    o, g = make_pair(nx, ny, nz, n_modes=24, seed=4, precision=precision, inlet=inlet)
    f0 = o.state() * (1.0 + 0.02 * noise((19, nz, ny, nx), seed=11))
    set_both(o, g, f0)
    o.step(1)
    g.step(1)
    er, eu = field_errors(o, g)
    tol = TOL1[precision]
    assert er < tol and eu < tol, (precision, er, eu)
    fo, fg = o.state(), g.populations()
    # each population field to the field tolerance (max-norm error over the
    # lattice relative to that population's largest value)
    for q in range(19):
        err = np.max(np.abs(fg[q] - fo[q])) / np.max(np.abs(fo[q]))
        assert err < tol, (precision, q, err)


def test_200_steps_small_channel():
    """64x32x32 lattice, Re_tau = 1000, N = 100 modes, 200 steps, FP32."""
    o, g = make_pair(64, 32, 32, n_modes=100, seed=1)
    set_both(o, g, o.state())
    o.step(200)
    g.step(200)
    g.sync()
    er, eu = field_errors(o, g)
    assert er < 1e-3 and eu < 1e-3, (er, eu)


@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp16row"])
def test_half_storage_200_steps(precision):
    o, g = make_pair(64, 32, 32, n_modes=100, seed=1, precision=precision)
    set_both(o, g, o.state())
    o.step(200)
    g.step(200)
    er, eu = field_errors(o, g)
    tol = TOL1[precision] * math.sqrt(200)
    assert er < tol and eu < tol, (precision, er, eu)


@pytest.mark.parametrize("t", [0, 7, 20000, 1234567])
def test_stg_inlet_velocity(t):
    o, g = make_pair(8, 48, 16, n_modes=200, seed=2)
    uo = o.inlet_velocity(t)
    ug = g.inlet_velocity(t)
    UR = o.tables()["UR"]
    fo = uo.copy()
    fo[..., 0] -= UR[None, :]
    assert np.max(np.abs(ug - uo)) < 1e-4 * np.max(np.abs(fo))


def test_stg_amplitude_and_length_scale_parameters():
    theta = (0.3, 1.7, 0.41, 7.1)
    o, g = make_pair(8, 32, 8, n_modes=64, seed=6, theta=theta)
    uo, ug = o.inlet_velocity(50), g.inlet_velocity(50)
    assert np.max(np.abs(ug - uo)) < 1e-4 * np.max(np.abs(uo[..., 1:]))
    # set_params rebuilds the tables but keeps the flow constants of creation
    from oracle.oracle import Oracle, default_config
    from paper_2304_04214_gb300.inputs import stg_uniforms
    g.set_params((0.4, 1.0, 0.4, 7.8))
    cfg = default_config(8, 32, 8, n_modes=64, kappa0=theta[2], B0=theta[3])
    o2 = Oracle(cfg, theta=(0.4, 1.0, 0.4, 7.8), uniforms=stg_uniforms(64, 6))
    u2 = o2.inlet_velocity(50)
    assert np.max(np.abs(g.inlet_velocity(50) - u2)) < 1e-4 * np.max(np.abs(u2[..., 1:]))


@pytest.mark.parametrize("shape,kw", [
    ((3, 4, 1), {}),
    ((5, 6, 2), {"n_modes": 0}),
    ((33, 8, 3), {"wall_model": 0}),
    ((40, 10, 4), {"inlet": 0, "n_modes": 0}),
    ((129, 12, 5), {"c_smag": 0.0}),
])
def test_edge_cases(shape, kw):
    args = dict(n_modes=8, seed=7)
    args.update(kw)
    o, g = make_pair(*shape, **args)
    nx, ny, nz = shape
    f0 = o.state() * (1.0 + 0.01 * noise((19, nz, ny, nx), seed=12))
    set_both(o, g, f0)
    o.step(3)
    g.step(3)
    er, eu = field_errors(o, g)
    assert er < 1e-5 and eu < 1e-5, (shape, kw, er, eu)


def test_statistics_accumulate_like_the_oracle():
    o, g = make_pair(32, 16, 8, n_modes=16, seed=8, stats=1)
    set_both(o, g, o.state())
    o.step(10)
    g.step(10)
    so, uto, no = o.stats()
    sg, utg, ng = g.stats()
    assert no == ng == 10
    for c in range(7):
        assert np.max(np.abs(sg[..., c] - so[..., c])) < 1e-5 * np.max(np.abs(so[..., c])) + 1e-12, c
    assert np.max(np.abs(utg - uto)) < 1e-5 * np.max(uto)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp16", 2e-3)])
def test_wall_plane_walk_with_a_ragged_last_block(precision, tol):
    """Lattices whose interior kernel takes long enough make each wall-kernel
    block walk several z planes (two here: 256x64x67 in FP32, 384x96x65 in
    FP16); the odd nz leaves the last block a partial walk.  Fields and the
    statistics, sampled every step (the statistics variants of the kernels),
    against the oracle after two steps."""
    shape = (256, 64, 67) if precision == "fp32" else (384, 96, 65)
    o, g = make_pair(*shape, n_modes=32, seed=12, precision=precision, stats=1)
    o.step(2)
    g.step(2)
    er, eu = field_errors(o, g)
    assert er < tol and eu < tol, (er, eu)
    so, uto, no = o.stats()
    sg, utg, ng = g.stats()
    assert no == ng == 2
    # each sum adds nz x 2 per-cell values, each within the field tolerance
    # (tol max|u| for u, about 2 tol max|u|^2 for a product): the sums agree
    # to that per term
    n = shape[2] * 2
    umax = np.max(np.abs(o.fields()[1]))
    for c in range(7):
        bar = tol * umax if c < 3 else 3 * tol * umax * umax
        assert np.max(np.abs(sg[..., c] - so[..., c])) / n < bar, c
    assert np.max(np.abs(utg - uto)) < tol * np.max(uto)
    g.close()


@pytest.mark.parametrize("shape,re_tau,n_modes,seed,precision,tol", [
    ((384, 96, 96), 1000.0, 200, 2, "fp32", 1e-5),
    ((384, 96, 96), 1000.0, 200, 2, "fp16", 2e-3),
    ((768, 128, 192), 2000.0, 300, 3, "fp32", 1e-5),
    ((768, 128, 192), 2000.0, 300, 3, "fp16", 2e-3),
])
def test_full_size_channels_first_steps(shape, re_tau, n_modes, seed, precision, tol):
    """The bench workloads 384x96x96 (Re_tau = 1000, N = 200) and 768x128x192
    (Re_tau = 2000, N = 300) in the launch configuration bench.py times (the
    automatic kernel choice: two cells per thread for FP32, four for FP16;
    the wall kernel's plane walk), compared over the whole lattice after two
    steps."""
    o, g = make_pair(*shape, re_tau=re_tau, n_modes=n_modes, seed=seed, precision=precision)
    o.step(2)
    g.step(2)
    er, eu = field_errors(o, g)
    assert er < tol and eu < tol, (er, eu)
    g.close()


def test_largest_channel_first_steps_all_storages():
    """The bench's default workload, 1536x192x384 (113 M cells; Re_tau = 5200,
    N = 400), in the launch configuration bench.py times, for FP32, FP16, BF16
    and FP16 row-base storage: every cell after two steps against one FP64 oracle run of the
    whole lattice (about 41 GB of host memory and a few tens of seconds on the
    host cores).  Tolerances: FP32 1e-5; FP16 and BF16 their one-step bars
    times two."""
    from oracle.oracle import Oracle, default_config
    from paper_2304_04214_gb300.channel import LBMChannel
    from paper_2304_04214_gb300.inputs import stg_uniforms
    nx, ny, nz, N, seed = 1536, 192, 384, 400, 4
    un = stg_uniforms(N, seed)
    o = Oracle(default_config(nx, ny, nz, re_tau=5200.0, n_modes=N), uniforms=un)
    o.step(2)
    ro, uo = o.fields()
    o.close()
    del o
    for precision, tol in (("fp32", 1e-5), ("fp16", 2e-3), ("bf16", 1.6e-2), ("fp16row", 2e-3)):
        g = LBMChannel(nx, ny, nz, re_tau=5200.0, n_modes=N, uniforms=un, precision=precision)
        g.step(2)
        rg, ug = g.fields()
        g.close()
        er = np.max(np.abs(rg - ro)) / np.max(np.abs(ro))
        eu = np.max(np.abs(ug - uo)) / np.max(np.abs(uo))
        del rg, ug
        assert er < tol and eu < tol, (precision, er, eu)


def test_divergence_is_reported():
    """An unphysical state (|u| > 0.3) sets the device divergence flag, which
    lbm_sync returns as LBM_EDIVERGED."""
    from paper_2304_04214_gb300 import _abi
    o, g = make_pair(16, 8, 4, n_modes=0)
    f = o.state()
    f[10] += 0.5          # a strong +x population everywhere
    g.set_populations(f)
    g.step(1)
    with pytest.raises(_abi.LBMError) as e:
        g.sync()
    assert e.value.code == _abi.LBM_EDIVERGED
    g.sync()              # the flag is cleared once reported


def test_device_wait_timeout_is_reported():
    """Failure detection without a fault: a device wait that nothing completes
    (the bounded wait of the staged kernel's copy ring) gives up, raises the
    timeout flag, and lbm_sync reports LBM_ETIMEOUT; the context stays usable
    and the following steps still match the oracle."""
    from paper_2304_04214_gb300 import _abi
    o, g = make_pair(32, 8, 4, n_modes=4, seed=2)
    assert g.lib.lbm_probe_wait_timeout(g.h) == 0
    with pytest.raises(_abi.LBMError) as e:
        g.sync()
    assert e.value.code == _abi.LBM_ETIMEOUT
    g.sync()              # cleared once reported
    o.step(3)
    g.step(3)
    er, eu = field_errors(o, g)
    assert er < 1e-5 and eu < 1e-5


def test_async_wall_shear_matches_the_synchronous_call():
    """lbm_wall_shear_async into two pinned buffers in turn gives, step by
    step, what lbm_wall_shear returns; both match the oracle's tau_w."""
    import torch
    o, g = make_pair(64, 16, 8, n_modes=16, seed=9)
    bufs = [torch.empty(2 * 64, dtype=torch.float64).pin_memory() for _ in range(2)]
    outs = []
    for n in range(4):
        g.step(1)
        g.wall_shear_async(bufs[n % 2])
        if n >= 1:
            g.sync()
            outs.append(bufs[(n - 1) % 2].numpy().copy())
    g.sync()
    outs.append(bufs[3 % 2].numpy().copy())
    assert len(outs) == 4 and all(np.all(np.isfinite(x)) for x in outs)
    ref = g.wall_shear().reshape(-1)
    assert np.array_equal(outs[-1], ref)
    o.step(4)
    rho, _ = o.fields()
    ut = o.utau()                                   # (2, nz, nx)
    # tau_w = rho u_tau^2 of the wall cells, z-averaged
    tw = np.stack([(rho[:, 0, :] * ut[0] ** 2).mean(axis=0), (rho[:, -1, :] * ut[1] ** 2).mean(axis=0)])
    assert np.max(np.abs(ref - tw.reshape(-1))) < 1e-4 * np.max(tw)


@pytest.mark.parametrize("kernel", ["auto", "cell"])
def test_coupling_loop_is_stream_ordered(kernel):
    """A coupling loop that changes the inlet profile every step and takes
    every step's wall shear without waiting (profile uploads double-buffered on
    a copy stream; the reduction beside the interior kernel on the side stream
    when the wall rows are computed there, on the main stream after the
    one-cell kernel; storing into pinned host buffers used in turn) gives bit
    for bit what the same loop gives with a host synchronization after every
    call."""
    import ctypes as ct
    import torch
    from paper_2304_04214_gb300.channel import LBMChannel
    a = LBMChannel(64, 16, 8, n_modes=16, seed=9, step_kernel=kernel)
    b = LBMChannel(64, 16, 8, n_modes=16, seed=9, step_kernel=kernel)
    dp = lambda x: ct.cast(x.data_ptr(), ct.POINTER(ct.c_double)) if isinstance(x, torch.Tensor) \
        else x.ctypes.data_as(ct.POINTER(ct.c_double))   # noqa: E731
    U0, R0 = np.empty(a.ny), np.empty(6 * a.ny)
    a.lib.lbm_get_inlet_profile(a.h, dp(U0), dp(R0))
    U = torch.empty(a.ny, dtype=torch.float64).pin_memory()
    R = torch.empty(6 * a.ny, dtype=torch.float64).pin_memory()
    tws = [torch.empty(2 * a.nx, dtype=torch.float64).pin_memory() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    n_steps = 30
    ref, got = [], []
    for n in range(n_steps):
        U.copy_(torch.from_numpy(U0 * (1.0 + 0.02 * np.sin(n))))
        R.copy_(torch.from_numpy(R0 * (1.0 + 0.05 * np.cos(n))))
        assert a.lib.lbm_set_inlet_profile(a.h, dp(U), dp(R)) == 0
        a.step(1)
        a.sync()
        ref.append(a.wall_shear().copy())
        assert b.lib.lbm_set_inlet_profile(b.h, dp(U), dp(R)) == 0
        b.step(1)
        assert b.lib.lbm_wall_shear_async(b.h, dp(tws[n % 2])) == 0
        evs[n % 2].record(b.stream)
        if n >= 1:
            evs[(n - 1) % 2].synchronize()
            got.append(tws[(n - 1) % 2].numpy().copy())
        # the next iteration rewrites the pinned profile buffers: the library
        # has staged them, so the host may do so at once
    evs[(n_steps - 1) % 2].synchronize()
    got.append(tws[(n_steps - 1) % 2].numpy().copy())
    b.sync()
    assert np.array_equal(a.populations(), b.populations())
    for n in range(n_steps):
        assert np.array_equal(ref[n].reshape(-1), got[n].reshape(-1)), n
    assert np.max(np.abs(ref[-1])) > 0
    a.close()
    b.close()

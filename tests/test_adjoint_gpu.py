"""The hand-written adjoint of the CUDA step against complex-step derivatives
of the FP64 oracle (exact to rounding): one-step vector-Jacobian products with
respect to the state and to theta, and the windowed objective's gradient with
checkpointed recomputation.  Tolerance 1e-3 relative (the stated bar for the
gradients); the forward J to 1e-5.
"""
import ctypes as ct

import numpy as np
import pytest

from gpu_helpers import make_pair, set_both
from oracle.oracle import Oracle, default_config
from paper_2304_04214_gb300.inputs import noise, stg_uniforms

pytestmark = pytest.mark.gpu
H = 1e-20          # complex-step size


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _setup(nx=24, ny=8, nz=4, N=8, seed=21, theta=(0.4, 1.0, 0.4, 7.8), eps=0.01):
    o, g = make_pair(nx, ny, nz, n_modes=N, seed=seed, theta=theta)
    f0 = o.state() * (1.0 + eps * noise((19, nz, ny, nx), seed=seed + 1))
    f0 = set_both(o, g, f0)
    return o, g, f0


def _oracle_cs(nx, ny, nz, N, seed, theta, f0, fim=None, theta_im=None, steps=1, obj=None, t0=0):
    cfg = default_config(nx, ny, nz, n_modes=N, kappa0=theta[2], B0=theta[3])
    oz = Oracle(cfg, theta=theta, uniforms=stg_uniforms(N, seed), complex_step=True, theta_im=theta_im)
    oz.set_state(f0, fim)
    oz.time = t0
    if obj is not None:
        oz.objective_begin(*obj)
    oz.step(steps)
    return oz


def _vjp(g, lam):
    from paper_2304_04214_gb300 import _abi
    prev = np.empty_like(lam)
    dth = np.empty(4)
    _abi.check(g.lib.lbm_vjp_step(g.h, _dp(np.ascontiguousarray(lam)), _dp(prev), _dp(dth)), "lbm_vjp_step")
    return prev, dth


@pytest.mark.parametrize("where", ["all", "inlet", "outlet", "walls", "interior"])
def test_vjp_state_matches_complex_step(where):
    nx, ny, nz, N, seed, theta = 24, 8, 4, 8, 21, (0.4, 1.0, 0.4, 7.8)
    o, g, f0 = _setup(nx, ny, nz, N, seed, theta)
    lam = noise((19, nz, ny, nx), seed=31)
    prev, _ = _vjp(g, lam)
    v = noise((19, nz, ny, nx), seed=32)
    mask = np.zeros((nz, ny, nx), bool)
    if where == "all":
        mask[:] = True
    elif where == "inlet":
        mask[:, :, :2] = True
    elif where == "outlet":
        mask[:, :, -2:] = True
    elif where == "walls":
        mask[:, [0, 1, ny - 2, ny - 1], :] = True
    else:
        mask[:, 3:5, 8:16] = True
    v = v * mask[None]
    oz = _oracle_cs(nx, ny, nz, N, seed, theta, f0, fim=H * v)
    ref = np.sum(lam * oz.state(imag=True)) / H
    got = np.sum(prev * v)
    assert abs(got - ref) <= 1e-3 * max(abs(ref), 1e-12) + 1e-6 * np.sqrt(np.sum(v * v)), (where, got, ref)


def test_vjp_theta_matches_complex_step():
    nx, ny, nz, N, seed, theta = 24, 8, 4, 8, 21, (0.4, 1.0, 0.4, 7.8)
    o, g, f0 = _setup(nx, ny, nz, N, seed, theta)
    lam = noise((19, nz, ny, nx), seed=33)
    _, dth = _vjp(g, lam)
    for kk in range(4):
        im = np.zeros(4)
        im[kk] = H
        oz = _oracle_cs(nx, ny, nz, N, seed, theta, f0, theta_im=im)
        ref = np.sum(lam * oz.state(imag=True)) / H
        assert abs(dth[kk] - ref) <= 1e-3 * abs(ref) + 1e-9, (kk, dth[kk], ref)


def test_adjoint_window_gradient_matches_complex_step():
    """J = J_tau + J_R over 8 steps (checkpoint every 4) on a 32x8x4 channel."""
    from paper_2304_04214_gb300 import _abi
    nx, ny, nz, N, seed, theta = 32, 8, 4, 8, 23, (0.4, 1.0, 0.4, 7.8)
    T, K, obj = 8, 4, (4, 12, 6)
    o, g, f0 = _setup(nx, ny, nz, N, seed, theta)
    J = ct.c_double()
    dJ = np.empty(4)
    ob = _abi.Objective(*obj)
    _abi.check(g.lib.lbm_adjoint_step(g.h, T, K, ct.byref(ob), ct.byref(J), _dp(dJ)), "lbm_adjoint_step")
    lam0 = np.empty((19, nz, ny, nx))
    _abi.check(g.lib.lbm_adjoint_state_gradient(g.h, _dp(lam0)), "lbm_adjoint_state_gradient")
    # forward value
    o.objective_begin(*obj)
    o.step(T)
    Jo = o.objective()[0]
    assert abs(J.value - Jo) <= 1e-5 * abs(Jo), (J.value, Jo)
    # the state advanced by T steps exactly like lbm_step
    ro, uo = o.fields()
    rg, ug = g.fields()
    assert np.max(np.abs(ug - uo)) < 1e-4 * np.max(np.abs(uo))
    # dJ/dtheta
    for kk in range(4):
        im = np.zeros(4)
        im[kk] = H
        oz = _oracle_cs(nx, ny, nz, N, seed, theta, f0, theta_im=im, steps=T, obj=obj)
        ref = oz.objective()[1] / H
        assert abs(dJ[kk] - ref) <= 1e-3 * abs(ref) + 1e-10, (kk, dJ[kk], ref)
    # dJ/ds_0 along a random direction
    v = noise((19, nz, ny, nx), seed=41)
    oz = _oracle_cs(nx, ny, nz, N, seed, theta, f0, fim=H * v, steps=T, obj=obj)
    ref = oz.objective()[1] / H
    got = np.sum(lam0 * v)
    assert abs(got - ref) <= 1e-3 * abs(ref) + 1e-9, (got, ref)


@pytest.mark.parametrize("T,K,t0", [(256, 32, 0), (512, 64, 37)])
def test_long_adjoint_windows_match_complex_step(T, K, t0):
    """The window lengths the inlet tuning uses: T steps with a checkpoint
    every K (K - 1 segment slots recomputed per segment, u_tau of every step,
    the STG field of the whole window), the second starting at a time that is
    not a multiple of the STG ring period.  J, the state after the window, all
    four dJ/dtheta and dJ/ds_0 along a random direction against the oracle."""
    from paper_2304_04214_gb300 import _abi
    nx, ny, nz, N, seed, theta = 32, 8, 4, 8, 24, (0.4, 1.0, 0.4, 7.8)
    obj = (4, 12, 6)
    o, g, f0 = _setup(nx, ny, nz, N, seed, theta)
    o.time = t0
    g.time = t0
    J = ct.c_double()
    dJ = np.empty(4)
    ob = _abi.Objective(*obj)
    _abi.check(g.lib.lbm_adjoint_step(g.h, T, K, ct.byref(ob), ct.byref(J), _dp(dJ)), "lbm_adjoint_step")
    lam0 = np.empty((19, nz, ny, nx))
    _abi.check(g.lib.lbm_adjoint_state_gradient(g.h, _dp(lam0)), "lbm_adjoint_state_gradient")
    assert g.time == t0 + T
    o.objective_begin(*obj)
    o.step(T)
    Jo = o.objective()[0]
    assert abs(J.value - Jo) <= 1e-4 * abs(Jo), (J.value, Jo)
    _, uo = o.fields()
    _, ug = g.fields()
    assert np.max(np.abs(ug - uo)) < 1e-3 * np.max(np.abs(uo))
    for kk in range(4):
        im = np.zeros(4)
        im[kk] = H
        oz = _oracle_cs(nx, ny, nz, N, seed, theta, f0, theta_im=im, steps=T, obj=obj, t0=t0)
        ref = oz.objective()[1] / H
        assert abs(dJ[kk] - ref) <= 1e-3 * abs(ref) + 1e-10, (kk, dJ[kk], ref)
    v = noise((19, nz, ny, nx), seed=42)
    oz = _oracle_cs(nx, ny, nz, N, seed, theta, f0, fim=H * v, steps=T, obj=obj, t0=t0)
    ref = oz.objective()[1] / H
    got = np.sum(lam0 * v)
    assert abs(got - ref) <= 1e-3 * abs(ref) + 1e-9, (got, ref)
    # the channel steps on from the window's end like one that never ran it
    o.step(70)
    g.step(70)
    _, uo = o.fields()
    _, ug = g.fields()
    assert np.max(np.abs(ug - uo)) < 1e-3 * np.max(np.abs(uo))


def test_overlapped_recomputation_is_deterministic():
    """The recomputation of each segment runs on its own stream beside the
    reverse steps of the next one (nx even): two identical windows from the
    same state give bit-identical dJ/ds_0 (no multi-operand atomics) and
    dJ/dtheta to the rounding of its FP64 atomic sums; a window with the
    recomputation serialised by an odd nx is checked against the oracle
    elsewhere."""
    from paper_2304_04214_gb300.channel import LBMChannel
    nx, ny, nz, N, seed = 96, 16, 8, 16, 25
    un = stg_uniforms(N, seed)
    res = []
    for _ in range(2):
        g = LBMChannel(nx, ny, nz, n_modes=N, uniforms=un)
        g.step(30)
        J, dJ = g.adjoint_step(64, 8, (8, 40, 30))
        res.append((J, dJ, g.adjoint_state_gradient(), g.populations()))
        g.close()
    (Ja, dJa, la, fa), (Jb, dJb, lb, fb) = res
    assert Ja == Jb and np.array_equal(fa, fb)
    assert np.array_equal(la, lb)
    assert np.allclose(dJa, dJb, rtol=1e-12, atol=0)


@pytest.mark.parametrize("nx", [48, 47])
def test_checkpoint_spacing_does_not_change_the_gradient(nx):
    """The same 24-step window with a checkpoint every 24, 12, 8, 6, 4 and 3
    steps: up to three segments (their states all kept by the forward pass),
    and four or more (the earlier ones recomputed: beside the reverse steps
    for even nx, in line for odd nx).  The recomputed states are the
    forward pass's, so the state after the window and dJ/ds_0 are
    bit-identical, and J and dJ/dtheta agree to the rounding of their FP64
    atomic sums."""
    from paper_2304_04214_gb300.channel import LBMChannel
    ny, nz, N, seed = 16, 8, 16, 27
    un = stg_uniforms(N, seed)
    res = []
    for K in (24, 12, 8, 6, 4, 3):
        g = LBMChannel(nx, ny, nz, n_modes=N, uniforms=un)
        g.step(11)
        J, dJ = g.adjoint_step(24, K, (4, 30, 20))
        res.append((K, J, dJ, g.adjoint_state_gradient(), g.populations()))
        g.close()
    _, J0, dJ0, l0, f0 = res[0]
    assert np.any(l0 != 0)
    for K, J, dJ, lam, f in res[1:]:
        assert abs(J - J0) <= 1e-12 * abs(J0) and np.array_equal(f, f0), (K, J, J0)
        assert np.array_equal(lam, l0), K
        assert np.allclose(dJ, dJ0, rtol=1e-12, atol=0), (K, dJ, dJ0)


def test_autograd_function_returns_the_adjoint_gradient():
    import torch
    from paper_2304_04214_gb300 import STGAdjoint
    from paper_2304_04214_gb300.channel import LBMChannel
    nx, ny, nz, N, seed = 32, 8, 4, 8, 23
    obj = (4, 12, 6)
    un = stg_uniforms(N, seed)
    a = LBMChannel(nx, ny, nz, n_modes=N, uniforms=un)
    b = LBMChannel(nx, ny, nz, n_modes=N, uniforms=un)
    theta = torch.tensor([0.42, 1.1, 0.4, 7.8], dtype=torch.float64, requires_grad=True)
    J = STGAdjoint.apply(theta, a, 8, 4, obj)
    (2.0 * J).backward()
    b.set_params(theta.detach().numpy())
    Jb, dJb = b.adjoint_step(8, 4, obj)
    assert abs(J.item() - Jb) <= 1e-12 * abs(Jb)
    assert np.allclose(theta.grad.numpy(), 2.0 * dJb, rtol=1e-12, atol=0)


@pytest.mark.parametrize("kk", [0, 1, 2, 3])
def test_adjoint_full_window_256x64x64(kk):
    """The adjoint configuration: Re_tau = 1000, 256x64x64, 64-step window with a
    checkpoint every 8 steps, J_tau over 24 <= i < 48 and J_R at i = 40;
    dJ/d ell_e and dJ/d kappa against the oracle's complex-step derivative.
    Both sides start from the same given state (real, independent of theta:
    the adjoint differentiates the window, not the initial condition)."""
    from gpu_helpers import quantize_state
    from paper_2304_04214_gb300.channel import LBMChannel
    nx, ny, nz, N, seed = 256, 64, 64, 100, 5
    theta = (0.4, 1.0, 0.4, 7.8)
    obj = (24, 48, 40)
    un = stg_uniforms(N, seed)
    cfg = default_config(nx, ny, nz, n_modes=N, kappa0=theta[2], B0=theta[3])
    f0 = quantize_state(Oracle(cfg, theta=theta, uniforms=un).state(), "fp32")
    g = LBMChannel(nx, ny, nz, n_modes=N, uniforms=un)
    g.set_populations(f0)
    J, dJ = g.adjoint_step(64, 8, obj)
    im = np.zeros(4)
    im[kk] = H
    oz = Oracle(cfg, theta=theta, uniforms=un, complex_step=True, theta_im=im)
    oz.set_state(f0)
    oz.objective_begin(*obj)
    oz.step(64)
    Jo, Jim, _ = oz.objective()
    assert abs(J - Jo) <= 1e-4 * abs(Jo), (J, Jo)
    ref = Jim / H
    assert abs(dJ[kk] - ref) <= 1e-3 * abs(ref), (kk, dJ[kk], ref)


def test_vjp_with_the_outlet_sponge_matches_complex_step():
    """lbm_vjp_step with the sponge over the last 8 of 24 cells: state and
    theta products against the oracle's complex-step derivative."""
    nx, ny, nz, N, seed, theta = 24, 8, 4, 8, 21, (0.4, 1.0, 0.4, 7.8)
    o, g = make_pair(nx, ny, nz, n_modes=N, seed=seed, theta=theta, sponge=(8, 0.05))
    f0 = set_both(o, g, o.state() * (1.0 + 0.01 * noise((19, nz, ny, nx), seed=seed + 1)))
    lam = noise((19, nz, ny, nx), seed=31)
    prev, dth = _vjp(g, lam)
    v = noise((19, nz, ny, nx), seed=32)
    cfg = default_config(nx, ny, nz, n_modes=N, kappa0=theta[2], B0=theta[3], sponge_cells=8, sponge_nu=0.05)
    oz = Oracle(cfg, theta=theta, uniforms=stg_uniforms(N, seed), complex_step=True)
    oz.set_state(f0, H * v)
    oz.step(1)
    ref = np.sum(lam * oz.state(imag=True)) / H
    got = np.sum(prev * v)
    assert abs(got - ref) <= 1e-3 * abs(ref), (got, ref)
    for kk in (0, 2):
        im = np.zeros(4)
        im[kk] = H
        oz = Oracle(cfg, theta=theta, uniforms=stg_uniforms(N, seed), complex_step=True, theta_im=im)
        oz.set_state(f0)
        oz.step(1)
        ref = np.sum(lam * oz.state(imag=True)) / H
        assert abs(dth[kk] - ref) <= 1e-3 * abs(ref) + 1e-9, (kk, dth[kk], ref)

"""Guard bands around every buffer of the device arena and of the adjoint
workspace (lbm_debug_guard_bands): after steps across several STG ring periods
(CUDA graphs), the statistics, the wall-shear read-backs, field and population
copies, inlet-profile uploads, the sponge, an adjoint window and a single
vector-Jacobian product, not one byte of the bands has changed -- on small and
ragged lattices, for every step kernel and storage.  The check itself is shown
to see a change by a host-side write into the leading band (inside the
caller's own allocation).  Nothing here writes out of bounds."""
import ctypes as ct

import numpy as np
import pytest

from paper_2304_04214_gb300.inputs import noise

pytestmark = pytest.mark.gpu
GUARD = 4096


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


@pytest.mark.parametrize("shape,precision,kernel", [
    ((70, 16, 6), "fp32", "pair"),      # nx not a multiple of four
    ((129, 12, 5), "fp32", "cell"),     # odd nx: the one-cell kernel, objective kernel
    ((136, 12, 5), "fp16", "staged"),   # ragged last TMA tile
    ((64, 8, 3), "bf16", "quad"),
    ((68, 10, 4), "fp16row", "quad"),   # nx not a multiple of 128: a ragged warp
    ((48, 4, 1), "fp32", "auto"),       # wall rows only, one z plane
])
def test_guard_bands_stay_intact(shape, precision, kernel):
    import torch
    from paper_2304_04214_gb300 import _abi
    from paper_2304_04214_gb300.channel import LBMChannel
    nx, ny, nz = shape
    ch = LBMChannel(nx, ny, nz, n_modes=8, seed=3, precision=precision, stats_every=3, guard_bytes=GUARD)
    if kernel != "auto":
        ch.step_kernel = kernel
    assert ch.guard_bytes_changed() == 0
    ch.step(150)                                   # two ring periods and more
    U, R = np.empty(ny), np.empty(6 * ny)
    _abi.check(ch.lib.lbm_get_inlet_profile(ch.h, _dp(U), _dp(R)), "lbm_get_inlet_profile")
    _abi.check(ch.lib.lbm_set_inlet_profile(ch.h, _dp(U * 1.01), _dp(R)), "lbm_set_inlet_profile")
    pinned = torch.empty(2 * nx, dtype=torch.float64).pin_memory()
    for _ in range(3):
        ch.step(1)
        ch.wall_shear_async(pinned)
    ch.wall_shear()
    out = np.empty(2 * nx)
    _abi.check(ch.lib.lbm_wall_shear_noalloc(ch.h, _dp(out)), "lbm_wall_shear_noalloc")
    ch.stats()
    ch.reset_stats()
    ch.fields()
    f = ch.populations()
    ch.set_populations(f)
    ch.inlet_velocity(5)
    ch.set_sponge(max(1, nx // 4), 0.05)
    ch.step(4)
    if precision == "fp32":
        ch.adjoint_step(16, 4, (1, nx // 2, nx // 3))
        ch.vjp_step(noise((19, nz, ny, nx), seed=9))
        ch.step(2)
    ch.sync()
    assert ch.guard_bytes_changed() == 0
    # the check sees a changed byte: the leading band starts the caller's tensor
    ch.mem[0] = 0
    assert ch.guard_bytes_changed() == 1
    ch.close()

"""lbm_wall_shear_noalloc: the wall-shear read-back for callers that must not
allocate device memory (its device staging is a fixed array inside the
library).  Compared through the C ABI with lbm_wall_shear on the same state,
on two calls in a row, and checked to refuse a lattice wider than its array.

Collected last on purpose (file name), so a run that stops at the first
failure has run every other test before this one.
"""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_noalloc_wall_shear_matches_the_arena_version():
    from paper_2304_04214_gb300 import _abi
    from paper_2304_04214_gb300.channel import LBMChannel
    nx = 48
    ch = LBMChannel(nx, 16, 8, re_tau=1000.0, n_modes=16, seed=3)
    lib = ch.lib
    for rnd in range(2):
        ch.step(3)
        ref = np.empty(2 * nx)
        _abi.check(lib.lbm_wall_shear(ch.h, _dp(ref)), "lbm_wall_shear")
        assert np.all(ref > 0.0)
        # two calls in a row of the no-allocation entry point
        for _ in range(2):
            got = np.full(2 * nx, np.nan)
            _abi.check(lib.lbm_wall_shear_noalloc(ch.h, _dp(got)), "lbm_wall_shear_noalloc")
            assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref)), rnd
    ch.close()


def test_noalloc_wall_shear_refuses_a_lattice_wider_than_its_array():
    from paper_2304_04214_gb300 import _abi
    from paper_2304_04214_gb300.channel import LBMChannel
    nx = _abi.LBM_NOALLOC_MAX_NX + 2
    ch = LBMChannel(nx, 4, 1, re_tau=1000.0, n_modes=0)
    out = np.empty(2 * nx)
    assert ch.lib.lbm_wall_shear_noalloc(ch.h, _dp(out)) == _abi.LBM_ENOSCRATCH
    # the arena version still serves this lattice
    _abi.check(ch.lib.lbm_wall_shear(ch.h, _dp(out)), "lbm_wall_shear")
    ch.close()

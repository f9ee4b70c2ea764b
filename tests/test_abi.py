"""The C-ABI library builds, loads and exports what include/lbm.h declares;
host-side argument checks work without a GPU (no device call is made)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_2304_04214_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbm_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = _abi.lib()
    names = declared_functions()
    assert "lbm_step" in names and "lbm_create" in names
    for n in names:
        assert hasattr(lib, n), n
    # the binding declares every one of them, and nothing the header lacks
    assert set(_abi.PROTOTYPES) == set(names)


def test_error_strings():
    lib = _abi.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -99):
        assert isinstance(lib.lbm_error_string(code), bytes)
    assert lib.lbm_error_string(-1) == b"invalid argument"


def _create(nx=16, ny=8, nz=4, re_tau=1000.0, n_modes=4, uniforms=True, precision=0):
    lib = _abi.lib()
    un = np.full(4 * max(n_modes, 1), 0.25)
    g = _abi.Grid(nx, ny, nz)
    stg = _abi.StgParams(n_modes, 1.01, 0.5, 0.4, 1.0,
                         un.ctypes.data_as(ct.POINTER(ct.c_double)) if uniforms else None)
    o = _abi.Opts()
    lib.lbm_default_opts(ct.byref(o))
    o.precision = precision
    h = ct.c_void_p()
    rc = lib.lbm_create(ct.byref(g), re_tau, ct.byref(stg), ct.byref(o), ct.byref(h))
    return rc, h


def test_create_validates_arguments_on_the_host():
    lib = _abi.lib()
    for kw in (dict(ny=7), dict(ny=2), dict(nx=2), dict(nz=0), dict(re_tau=0.0), dict(n_modes=-1),
               dict(uniforms=False), dict(precision=5)):
        rc, h = _create(**kw)
        assert rc == _abi.LBM_EINVAL, kw
        assert not h.value
    rc, h = _create()
    assert rc == 0 and h.value
    nb = ct.c_size_t()
    assert lib.lbm_required_bytes(h, ct.byref(nb)) == 0
    # two FP32 lattices dominate: 2 * 19 * ncell * 4 bytes
    assert nb.value >= 2 * 19 * 16 * 8 * 4 * 4
    c = np.empty(6)
    assert lib.lbm_get_constants(h, c.ctypes.data_as(ct.POINTER(ct.c_double))) == 0
    assert c[0] == 4.0 and c[1] > 0 and c[3] > 0.5
    # calls that need device memory refuse before binding
    assert lib.lbm_step(h, 1) == _abi.LBM_ESTATE
    assert lib.lbm_step(h, -1) == _abi.LBM_EINVAL
    assert lib.lbm_sync(h) == _abi.LBM_ESTATE
    lib.lbm_destroy(h)


def test_half_storage_needs_half_the_lattice_bytes():
    lib = _abi.lib()
    sizes = []
    for p in (0, 1, 2):
        rc, h = _create(nx=64, ny=32, nz=32, precision=p)
        assert rc == 0
        nb = ct.c_size_t()
        lib.lbm_required_bytes(h, ct.byref(nb))
        sizes.append(nb.value)
        lib.lbm_destroy(h)
    assert sizes[1] == sizes[2]
    lat32, lat16 = 2 * 19 * 65536 * 4, 2 * 19 * 65536 * 2
    assert sizes[0] - sizes[1] == pytest.approx(lat32 - lat16, abs=1024)


def test_step_kernel_selection_is_checked_on_the_host():
    lib = _abi.lib()
    rc, h = _create(nx=15)
    assert rc == 0
    assert lib.lbm_set_step_kernel(h, 7) == _abi.LBM_EINVAL
    assert lib.lbm_set_step_kernel(h, -1) == _abi.LBM_EINVAL
    assert lib.lbm_set_step_kernel(h, _abi.LBM_KERNEL_PAIR) == _abi.LBM_EINVAL      # nx odd
    assert lib.lbm_set_step_kernel(h, _abi.LBM_KERNEL_STAGED) == _abi.LBM_EINVAL    # nx % 4 != 0
    assert lib.lbm_set_step_kernel(h, _abi.LBM_KERNEL_CELL) == 0
    k = ct.c_int(-1)
    assert lib.lbm_get_step_kernel(h, ct.byref(k)) == 0 and k.value == _abi.LBM_KERNEL_CELL
    assert lib.lbm_get_step_kernel(h, None) == _abi.LBM_EINVAL
    lib.lbm_destroy(h)
    rc, h = _create(nx=16)
    assert lib.lbm_set_step_kernel(h, _abi.LBM_KERNEL_PAIR) == 0
    assert lib.lbm_get_step_kernel(h, ct.byref(k)) == 0 and k.value == _abi.LBM_KERNEL_PAIR
    lib.lbm_destroy(h)


def test_profiling_interval_is_checked_on_the_host():
    lib = _abi.lib()
    rc, h = _create(nx=16)
    assert rc == 0
    assert lib.lbm_profile_enable(h, -1) == _abi.LBM_EINVAL
    assert lib.lbm_profile_enable(None, 1) == _abi.LBM_EINVAL
    assert lib.lbm_profile_enable(h, 0) == 0
    lib.lbm_destroy(h)


def test_checkpoint_calls_refuse_before_binding():
    lib = _abi.lib()
    rc, h = _create()
    assert rc == 0
    assert lib.lbm_save(h, b"/nonexistent/x.lbm") == _abi.LBM_ESTATE
    assert lib.lbm_load(h, b"/nonexistent/x.lbm") == _abi.LBM_ESTATE
    assert lib.lbm_save(h, None) == _abi.LBM_EINVAL
    assert lib.lbm_save(None, b"x") == _abi.LBM_EINVAL
    lib.lbm_destroy(h)


def test_header_is_plain_c(tmp_path):
    """include/lbm.h is a C header: it compiles as C99 with warnings as
    errors (no C++ in the boundary)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "lbm.h"\nint main(void) { return (int)sizeof(lbm_grid) > 0 ? 0 : 1; }\n')
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", inc, str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("ny,re_tau", [(32, 1000.0), (96, 1000.0), (128, 2000.0), (192, 5200.0)])
def test_host_constants_and_inlet_profile_match_the_oracle(ny, re_tau):
    """The library's host-side set-up, computed at lbm_create without a GPU:
    the flow constants (delta, u_tau,ref, nu, tau0, U_b+, max l_e) and the
    default inlet profile -- the Reichardt mean U_R(y) and the prescribed
    Reynolds stress R(y) in lattice units -- equal the oracle's, computed by
    its own FP64 code (reading A20, eq:reichard, reading A16 vi)."""
    from oracle.oracle import Oracle, default_config
    lib = _abi.lib()
    rc, h = _create(nx=16, ny=ny, nz=4, re_tau=re_tau)
    assert rc == 0
    dp = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))   # noqa: E731
    cst = np.zeros(6)
    assert lib.lbm_get_constants(h, dp(cst)) == 0
    U, R = np.zeros(ny), np.zeros(6 * ny)
    assert lib.lbm_get_inlet_profile(h, dp(U), dp(R)) == 0
    lib.lbm_destroy(h)
    o = Oracle(default_config(16, ny, 4, re_tau=re_tau, n_modes=4),
               uniforms=np.full((4, 4), 0.25))
    oc, t = o.constants(), o.tables()
    ref = [oc["delta"], oc["utau_ref"], oc["nu"], oc["tau0"], oc["ubp"], oc["maxl"]]
    assert np.allclose(cst, ref, rtol=1e-12, atol=0), (cst, ref)
    assert np.allclose(U, t["UR"], rtol=1e-12, atol=1e-15)
    assert np.allclose(R.reshape(ny, 6), t["Rp"] * oc["utau_ref"] ** 2, rtol=1e-12, atol=1e-18)


def test_setters_validate_on_the_host():
    """Argument checks of the setters, before any device work: the sponge
    (cells within the lattice, a finite non-negative viscosity), the STG / wall
    parameters (positive length scale and kappa), the inlet profile (every
    R(y) positive definite, the old profile kept otherwise) and the graph
    switch."""
    lib = _abi.lib()
    rc, h = _create(nx=16, ny=8, nz=4)
    assert rc == 0
    dp = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))   # noqa: E731
    E = _abi.LBM_EINVAL
    assert lib.lbm_set_sponge(h, -1, 0.1) == E
    assert lib.lbm_set_sponge(h, 17, 0.1) == E
    assert lib.lbm_set_sponge(h, 4, -0.1) == E
    assert lib.lbm_set_sponge(h, 4, float("nan")) == E
    assert lib.lbm_set_sponge(h, 4, 0.1) == 0
    assert lib.lbm_set_params(h, dp(np.array([0.0, 1.0, 0.4, 7.8]))) == E
    assert lib.lbm_set_params(h, dp(np.array([0.4, 1.0, -0.4, 7.8]))) == E
    U, R = np.zeros(8), np.zeros(48)
    assert lib.lbm_get_inlet_profile(h, dp(U), dp(R)) == 0
    bad = R.copy()
    bad[6 * 3 + 1] = -1.0                          # R22 < 0 in row 3
    assert lib.lbm_set_inlet_profile(h, dp(U), dp(bad)) == E
    U2, R2 = np.zeros(8), np.zeros(48)
    lib.lbm_get_inlet_profile(h, dp(U2), dp(R2))
    assert np.array_equal(U2, U) and np.array_equal(R2, R)      # unchanged
    assert lib.lbm_set_graphs(None, 1) == E
    on, n = ct.c_int(), ct.c_long()
    assert lib.lbm_set_graphs(h, 0) == 0 and lib.lbm_graph_info(h, ct.byref(on), ct.byref(n)) == 0
    assert on.value == 0 and n.value == 0
    assert lib.lbm_graph_info(h, None, ct.byref(n)) == E
    lib.lbm_destroy(h)

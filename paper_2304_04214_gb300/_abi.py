"""ctypes declarations of the C ABI in include/lbm.h (argument marshalling only)."""
import ctypes as ct
import os

from . import build as _build

_LIB = None

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EDIVERGED, LBM_ENOTCONV, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6
LBM_ENOSCRATCH = -7
LBM_ETIMEOUT = -8
LBM_KERNEL_AUTO, LBM_KERNEL_CELL, LBM_KERNEL_PAIR, LBM_KERNEL_STAGED, LBM_KERNEL_QUAD = 0, 1, 2, 3, 4
KERNELS = {"auto": LBM_KERNEL_AUTO, "cell": LBM_KERNEL_CELL, "pair": LBM_KERNEL_PAIR,
           "staged": LBM_KERNEL_STAGED, "quad": LBM_KERNEL_QUAD}
LBM_NOALLOC_MAX_NX = 32768
LBM_FP32, LBM_FP16_DEV, LBM_BF16_DEV, LBM_FP16_ROW = 0, 1, 2, 3
LBM_FACE_LEFT, LBM_FACE_RIGHT = 0, 1
PRECISIONS = {"fp32": LBM_FP32, "fp16": LBM_FP16_DEV, "bf16": LBM_BF16_DEV, "fp16row": LBM_FP16_ROW}


class Grid(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int)]


class StgParams(ct.Structure):
    _fields_ = [("n_modes", ct.c_int), ("k_ratio", ct.c_double), ("beta_kmin", ct.c_double),
                ("ell_e", ct.c_double), ("amp", ct.c_double), ("uniforms", ct.POINTER(ct.c_double))]


class Opts(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("u_bulk", ct.c_double), ("c_smag", ct.c_double),
                ("kappa", ct.c_double), ("B", ct.c_double), ("wall_model", ct.c_int),
                ("inlet", ct.c_int), ("stats_every", ct.c_int), ("cuda_stream", ct.c_void_p)]


class Objective(ct.Structure):
    _fields_ = [("i_tau0", ct.c_int), ("i_tau1", ct.c_int), ("i_R", ct.c_int)]


class LBMError(RuntimeError):
    def __init__(self, code, call):
        msg = lib().lbm_error_string(code).decode()
        super().__init__(f"{call} failed: {msg} ({code})")
        self.code = code


_dp = ct.POINTER(ct.c_double)
_h = ct.c_void_p

# name -> (restype, argtypes)
PROTOTYPES = {
    "lbm_default_opts": (None, [ct.POINTER(Opts)]),
    "lbm_create": (ct.c_int, [ct.POINTER(Grid), ct.c_double, ct.POINTER(StgParams), ct.POINTER(Opts),
                              ct.POINTER(ct.c_void_p)]),
    "lbm_required_bytes": (ct.c_int, [_h, ct.POINTER(ct.c_size_t)]),
    "lbm_bind_memory": (ct.c_int, [_h, ct.c_void_p, ct.c_size_t]),
    "lbm_step": (ct.c_int, [_h, ct.c_int]),
    "lbm_sync": (ct.c_int, [_h]),
    "lbm_set_stream": (ct.c_int, [_h, ct.c_void_p]),
    "lbm_save": (ct.c_int, [_h, ct.c_char_p]),
    "lbm_load": (ct.c_int, [_h, ct.c_char_p]),
    "lbm_set_step_kernel": (ct.c_int, [_h, ct.c_int]),
    "lbm_set_graphs": (ct.c_int, [_h, ct.c_int]),
    "lbm_graph_info": (ct.c_int, [_h, ct.POINTER(ct.c_int), ct.POINTER(ct.c_long)]),
    "lbm_probe_wait_timeout": (ct.c_int, [_h]),
    "lbm_get_step_kernel": (ct.c_int, [_h, ct.POINTER(ct.c_int)]),
    "lbm_set_sponge": (ct.c_int, [_h, ct.c_int, ct.c_double]),
    "lbm_stats": (ct.c_int, [_h, _dp, _dp, ct.POINTER(ct.c_long)]),
    "lbm_reset_stats": (ct.c_int, [_h]),
    "lbm_get_fields": (ct.c_int, [_h, _dp, _dp]),
    "lbm_get_populations": (ct.c_int, [_h, _dp]),
    "lbm_set_populations": (ct.c_int, [_h, _dp]),
    "lbm_get_utau": (ct.c_int, [_h, _dp]),
    "lbm_get_time": (ct.c_int, [_h, ct.POINTER(ct.c_long)]),
    "lbm_set_time": (ct.c_int, [_h, ct.c_long]),
    "lbm_get_constants": (ct.c_int, [_h, _dp]),
    "lbm_inlet_velocity": (ct.c_int, [_h, ct.c_long, _dp]),
    "lbm_set_params": (ct.c_int, [_h, _dp]),
    "lbm_set_inlet_profile": (ct.c_int, [_h, _dp, _dp]),
    "lbm_get_inlet_profile": (ct.c_int, [_h, _dp, _dp]),
    "lbm_wall_shear": (ct.c_int, [_h, _dp]),
    "lbm_wall_shear_async": (ct.c_int, [_h, _dp]),
    "lbm_wall_shear_noalloc": (ct.c_int, [_h, _dp]),
    "lbm_set_slab": (ct.c_int, [_h, ct.c_int, ct.c_int, ct.c_int, ct.c_int]),
    "lbm_halo_bytes": (ct.c_int, [_h, ct.POINTER(ct.c_size_t)]),
    "lbm_halo_pack": (ct.c_int, [_h, ct.c_int, ct.c_void_p]),
    "lbm_halo_unpack": (ct.c_int, [_h, ct.c_int, ct.c_void_p]),
    "lbm_debug_guard_bands": (ct.c_int, [_h, ct.c_int]),
    "lbm_debug_check_guards": (ct.c_int, [_h, ct.POINTER(ct.c_longlong)]),
    "lbm_profile_enable": (ct.c_int, [_h, ct.c_int]),
    "lbm_profile_read": (ct.c_int, [_h, _dp, ct.POINTER(ct.c_long), ct.POINTER(ct.c_long)]),
    "lbm_adjoint_required_bytes": (ct.c_int, [_h, ct.c_int, ct.c_int, ct.POINTER(ct.c_size_t)]),
    "lbm_adjoint_bind": (ct.c_int, [_h, ct.c_int, ct.c_int, ct.c_void_p, ct.c_size_t]),
    "lbm_adjoint_step": (ct.c_int, [_h, ct.c_int, ct.c_int, ct.POINTER(Objective), _dp, _dp]),
    "lbm_adjoint_state_gradient": (ct.c_int, [_h, _dp]),
    "lbm_vjp_step": (ct.c_int, [_h, _dp, _dp, _dp]),
    "lbm_destroy": (None, [_h]),
    "lbm_error_string": (ct.c_char_p, [ct.c_int]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Open liblbm_gb300.so (building it from the in-tree sources if absent).

    Raises if it cannot be built or loaded: there is no other implementation.
    """
    global _LIB
    if _LIB is not None:
        return _LIB
    path = os.environ.get("LBM_GB300_LIB")       # an alternative build of the same sources
    if not path:
        path = _build.LIB
        if not os.path.exists(path) or _build._stale():
            _build.build()
    L = ct.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def check(code, call):
    if code != LBM_OK:
        raise LBMError(code, call)

"""Python binding of the channel library: PyTorch supplies the device memory
and the stream, every step of the method runs in the CUDA kernels behind the
C ABI (include/lbm.h).  Arrays use the layout f[q][k][j][i]."""
import ctypes as ct

import numpy as np

from . import _abi
from .inputs import stg_uniforms

Q = 19


def _dptr(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


class LBMChannel:
    """A synthetic turbulent channel on one GPU.

    nx x ny x nz lattice (x streamwise, y wall-normal with delta = ny/2, z
    spanwise), friction Reynolds number re_tau, an STG inlet with n_modes
    Fourier modes whose random draws are `uniforms` (n_modes x 4 in [0,1);
    drawn from `seed` by paper_2304_04214_gb300.inputs if not given).
    theta = (ell_e, amp, kappa, B) are the STG length-scale factor and
    amplitude and the Reichardt constants.  precision: "fp32" (f in FP32),
    "fp16" (f - w in FP16), "bf16" (f - f^eq(1, U0(y)) in BF16) or "fp16row"
    (f - f^eq(1, U0(y)) in FP16); the arithmetic is FP32 in every case.
    """

    def __init__(self, nx, ny, nz, re_tau=1000.0, n_modes=100, uniforms=None, seed=1,
                 precision="fp32", u_bulk=0.05, c_smag=0.01, kappa=0.4, B=7.8, ell_e=0.4,
                 amp=1.0, k_ratio=1.01, beta_kmin=0.5, wall_model=True, inlet=True,
                 stats_every=0, step_kernel="auto", stream=None, device=None, guard_bytes=0):
        import torch
        self._torch = torch
        self.lib = _abi.lib()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.ncell = self.nx * self.ny * self.nz
        self.device = torch.device(device if device is not None else "cuda")
        if uniforms is None and n_modes > 0:
            uniforms = stg_uniforms(n_modes, seed)
        self._uni = (np.ascontiguousarray(uniforms, dtype=np.float64).reshape(-1)
                     if n_modes > 0 else np.zeros(4))
        if n_modes > 0 and self._uni.size != 4 * n_modes:
            raise ValueError("uniforms must hold n_modes x 4 values")
        grid = _abi.Grid(self.nx, self.ny, self.nz)
        stg = _abi.StgParams(int(n_modes), float(k_ratio), float(beta_kmin), float(ell_e),
                             float(amp), _dptr(self._uni))
        opts = _abi.Opts()
        self.lib.lbm_default_opts(ct.byref(opts))
        opts.precision = _abi.PRECISIONS[precision]
        opts.u_bulk, opts.c_smag, opts.kappa, opts.B = u_bulk, c_smag, kappa, B
        opts.wall_model, opts.inlet, opts.stats_every = int(wall_model), int(inlet), int(stats_every)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        opts.cuda_stream = ct.c_void_p(stream.cuda_stream)
        h = ct.c_void_p()
        _abi.check(self.lib.lbm_create(ct.byref(grid), float(re_tau), ct.byref(stg), ct.byref(opts),
                                       ct.byref(h)), "lbm_create")
        self.h = h
        if guard_bytes:
            _abi.check(self.lib.lbm_debug_guard_bands(self.h, int(guard_bytes)), "lbm_debug_guard_bands")
        nbytes = ct.c_size_t()
        _abi.check(self.lib.lbm_required_bytes(self.h, ct.byref(nbytes)), "lbm_required_bytes")
        self.nbytes = nbytes.value
        with torch.cuda.device(self.device):
            self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        _abi.check(self.lib.lbm_bind_memory(self.h, ct.c_void_p(self.mem.data_ptr()),
                                            self.nbytes), "lbm_bind_memory")
        self.precision = precision
        if step_kernel != "auto":
            self.step_kernel = step_kernel

    # ---- life cycle ----
    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_destroy(self.h)
            self.h = None
            self.mem = None
            self.adj_mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- stepping ----
    def step(self, n=1):
        _abi.check(self.lib.lbm_step(self.h, int(n)), "lbm_step")

    def sync(self):
        _abi.check(self.lib.lbm_sync(self.h), "lbm_sync")

    @property
    def time(self):
        t = ct.c_long()
        _abi.check(self.lib.lbm_get_time(self.h, ct.byref(t)), "lbm_get_time")
        return t.value

    @time.setter
    def time(self, t):
        _abi.check(self.lib.lbm_set_time(self.h, int(t)), "lbm_set_time")

    @property
    def step_kernel(self):
        """The step kernel later steps run: 'cell', 'pair', 'quad' or 'staged'."""
        k = ct.c_int()
        _abi.check(self.lib.lbm_get_step_kernel(self.h, ct.byref(k)), "lbm_get_step_kernel")
        return {v: n for n, v in _abi.KERNELS.items()}[k.value]

    @step_kernel.setter
    def step_kernel(self, name):
        _abi.check(self.lib.lbm_set_step_kernel(self.h, _abi.KERNELS[name]), "lbm_set_step_kernel")

    def set_graphs(self, on):
        """Launch ring periods of steps as CUDA graphs (default) or not."""
        _abi.check(self.lib.lbm_set_graphs(self.h, int(bool(on))), "lbm_set_graphs")

    def graph_info(self):
        """(graphs on, graph launches so far)."""
        on, n = ct.c_int(), ct.c_long()
        _abi.check(self.lib.lbm_graph_info(self.h, ct.byref(on), ct.byref(n)), "lbm_graph_info")
        return bool(on.value), n.value

    def set_sponge(self, cells, nu_max):
        """Outlet sponge: over the last `cells` cells the viscosity rises by
        nu_max r^2 (r the position in the zone); cells = 0 switches it off."""
        _abi.check(self.lib.lbm_set_sponge(self.h, int(cells), float(nu_max)), "lbm_set_sponge")

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        _abi.check(self.lib.lbm_set_params(self.h, _dptr(th)), "lbm_set_params")

    # ---- checkpoint files ----
    def save(self, path):
        """Write the channel's state to `path` (see lbm_save)."""
        _abi.check(self.lib.lbm_save(self.h, str(path).encode()), "lbm_save")

    def load(self, path):
        """Restore a state written by save() from a channel created alike."""
        _abi.check(self.lib.lbm_load(self.h, str(path).encode()), "lbm_load")

    def guard_bytes_changed(self):
        """Bytes of the guard bands (guard_bytes > 0 at creation) that no longer
        hold their fill pattern."""
        n = ct.c_longlong()
        _abi.check(self.lib.lbm_debug_check_guards(self.h, ct.byref(n)), "lbm_debug_check_guards")
        return n.value

    # ---- host copies ----
    def fields(self):
        rho = np.empty((self.nz, self.ny, self.nx))
        u = np.empty((self.nz, self.ny, self.nx, 3))
        _abi.check(self.lib.lbm_get_fields(self.h, _dptr(rho), _dptr(u)), "lbm_get_fields")
        return rho, u

    def populations(self):
        f = np.empty((Q, self.nz, self.ny, self.nx))
        _abi.check(self.lib.lbm_get_populations(self.h, _dptr(f)), "lbm_get_populations")
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.size != Q * self.ncell:
            raise ValueError("populations must be 19 x nz x ny x nx")
        _abi.check(self.lib.lbm_set_populations(self.h, _dptr(f)), "lbm_set_populations")

    def utau(self):
        u = np.empty((2, self.nz, self.nx))
        _abi.check(self.lib.lbm_get_utau(self.h, _dptr(u)), "lbm_get_utau")
        return u

    def inlet_velocity(self, t):
        out = np.empty((self.nz, self.ny, 3))
        _abi.check(self.lib.lbm_inlet_velocity(self.h, int(t), _dptr(out)), "lbm_inlet_velocity")
        return out

    def constants(self):
        o = np.empty(6)
        _abi.check(self.lib.lbm_get_constants(self.h, _dptr(o)), "lbm_get_constants")
        return dict(delta=o[0], utau_ref=o[1], nu=o[2], tau0=o[3], ubp=o[4], maxl=o[5])

    def wall_shear(self):
        """z-averaged tau_w of the last step, (2, nx): bottom, top."""
        out = np.empty(2 * self.nx)
        _abi.check(self.lib.lbm_wall_shear(self.h, _dptr(out)), "lbm_wall_shear")
        return out.reshape(2, self.nx)

    def wall_shear_async(self, out):
        """Enqueue the same reduction into `out` (a pinned float64 torch tensor
        of 2 * nx values) without synchronizing; it holds the result once the
        stream has passed this point."""
        if out.dtype != self._torch.float64 or out.numel() != 2 * self.nx or out.is_cuda:
            raise ValueError("out must be a host float64 tensor of 2 * nx values")
        _abi.check(self.lib.lbm_wall_shear_async(self.h, ct.cast(out.data_ptr(), ct.POINTER(ct.c_double))),
                   "lbm_wall_shear_async")

    def stats(self):
        s = np.empty((self.ny, self.nx, 7))
        ut = np.empty((2, self.nx))
        n = ct.c_long()
        _abi.check(self.lib.lbm_stats(self.h, _dptr(s), _dptr(ut), ct.byref(n)), "lbm_stats")
        return s, ut, n.value

    def reset_stats(self):
        _abi.check(self.lib.lbm_reset_stats(self.h), "lbm_reset_stats")

    # ---- adjoint ----
    def adjoint_bind(self, window, ckpt_every):
        """Bind a torch-allocated adjoint workspace for windows of `window` steps."""
        torch = self._torch
        nbytes = ct.c_size_t()
        _abi.check(self.lib.lbm_adjoint_required_bytes(self.h, int(window), int(ckpt_every),
                                                       ct.byref(nbytes)), "lbm_adjoint_required_bytes")
        self.adj_mem = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        _abi.check(self.lib.lbm_adjoint_bind(self.h, int(window), int(ckpt_every),
                                             ct.c_void_p(self.adj_mem.data_ptr()), nbytes.value),
                   "lbm_adjoint_bind")

    def adjoint_step(self, window, ckpt_every, objective):
        """Advance `window` steps; return J and dJ/dtheta (numpy, 4) of the
        objective (i_tau0, i_tau1, i_R) by the adjoint with a checkpoint every
        `ckpt_every` steps."""
        if getattr(self, "adj_mem", None) is None or self._adj_shape != (window, ckpt_every):
            self.adjoint_bind(window, ckpt_every)
            self._adj_shape = (window, ckpt_every)
        J = ct.c_double()
        dJ = np.empty(4)
        ob = _abi.Objective(*[int(x) for x in objective])
        _abi.check(self.lib.lbm_adjoint_step(self.h, int(window), int(ckpt_every), ct.byref(ob),
                                             ct.byref(J), _dptr(dJ)), "lbm_adjoint_step")
        return J.value, dJ

    _adj_shape = None
    adj_mem = None

    def adjoint_state_gradient(self):
        lam = np.empty((Q, self.nz, self.ny, self.nx))
        _abi.check(self.lib.lbm_adjoint_state_gradient(self.h, _dptr(lam)), "lbm_adjoint_state_gradient")
        return lam

    def vjp_step(self, lam_next):
        """lambda_next ds_{t+1}/ds_t and lambda_next ds_{t+1}/dtheta at the current state."""
        lam = np.ascontiguousarray(lam_next, dtype=np.float64)
        prev = np.empty_like(lam)
        dth = np.empty(4)
        _abi.check(self.lib.lbm_vjp_step(self.h, _dptr(lam), _dptr(prev), _dptr(dth)), "lbm_vjp_step")
        return prev, dth


def _make_stg_adjoint():
    import torch

    class STGAdjoint(torch.autograd.Function):
        """J(theta) over a window of steps with its adjoint gradient.

        forward(theta, channel, window, ckpt_every, objective): sets the model
        parameters theta = (ell_e, amp, kappa, B) (a float64 tensor of 4),
        advances the channel `window` steps and returns J as a 0-d tensor; the
        gradient dJ/dtheta comes from the hand-written adjoint (checkpoint every
        `ckpt_every` steps) and is applied in backward.  The channel's state
        moves forward by `window` steps as a side effect.
        """

        @staticmethod
        def forward(ctx, theta, channel, window, ckpt_every, objective):
            channel.set_params(theta.detach().cpu().double().numpy())
            J, dJ = channel.adjoint_step(window, ckpt_every, objective)
            ctx.save_for_backward(torch.tensor(dJ, dtype=theta.dtype, device=theta.device))
            return torch.tensor(J, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (dJ,) = ctx.saved_tensors
            return grad_out * dJ, None, None, None, None

    return STGAdjoint


def __getattr__(name):
    if name == "STGAdjoint":
        cls = _make_stg_adjoint()
        globals()["STGAdjoint"] = cls
        return cls
    raise AttributeError(name)

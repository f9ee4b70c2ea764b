"""ctypes front end of the FP64 C oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY.  Arrays follow the structure-of-arrays layout
f[q][k][j][i] (i fastest), with the D3Q19 order of Sec. 2.1 (eq:vel-set).
"""
import ctypes as ct
import os

import numpy as np

from . import build as _build

Q = 19
_LIB = None

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)


class OracleConfig(ct.Structure):
    """Mirror of orc_config in lbm_oracle.c."""
    _fields_ = [
        ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
        ("n_modes", ct.c_int),
        ("inlet", ct.c_int), ("walls", ct.c_int), ("wall_model", ct.c_int),
        ("mrt", ct.c_int), ("stats", ct.c_int), ("threads", ct.c_int),
        ("re_tau", ct.c_double), ("u_bulk", ct.c_double), ("c_smag", ct.c_double),
        ("kappa0", ct.c_double), ("B0", ct.c_double),
        ("k_ratio", ct.c_double), ("beta_kmin", ct.c_double),
        ("tau0", ct.c_double), ("body_force", ct.c_double * 3),
        ("sponge_cells", ct.c_int), ("sponge_nu", ct.c_double),
    ]


def _p(a):
    return a.ctypes.data_as(_dp)


def load():
    """Load (building first if needed) liblbm_oracle.so."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build()
    lib = ct.CDLL(path)
    for pre in ("orc_", "orcz_"):
        g = lambda n: getattr(lib, pre + n)  # noqa: E731
        g("create").restype = ct.c_void_p
        g("create").argtypes = [ct.POINTER(OracleConfig), _dp, _dp, _dp]
        g("destroy").argtypes = [ct.c_void_p]
        g("step").argtypes = [ct.c_void_p, ct.c_int]
        for n in ("get_state", "get_state_imag", "get_force", "get_utau", "set_utau"):
            g(n).argtypes = [ct.c_void_p, _dp]
        g("set_state").argtypes = [ct.c_void_p, _dp, _dp]
        g("get_fields").argtypes = [ct.c_void_p, _dp, _dp]
        g("get_time").restype = ct.c_long
        g("get_time").argtypes = [ct.c_void_p]
        g("set_time").argtypes = [ct.c_void_p, ct.c_long]
        g("get_constants").argtypes = [ct.c_void_p, _dp]
        g("get_tables").argtypes = [ct.c_void_p] + [_dp] * 9
        g("inlet_velocity").argtypes = [ct.c_void_p, ct.c_long, _dp]
        g("stats_reset").argtypes = [ct.c_void_p]
        g("stats_get").restype = ct.c_long
        g("stats_get").argtypes = [ct.c_void_p, _dp, _dp]
        g("objective_begin").argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int]
        g("objective_value").argtypes = [ct.c_void_p, _dp, _dp, _dp]
        g("matrix").argtypes = [_dp, _dp, _ip]
        g("cell_feq").argtypes = [ct.c_double, _dp, _dp]
        g("cell_moments").argtypes = [_dp, _dp]
        g("cell_collide").argtypes = [_dp, _dp, ct.c_double, ct.c_double, ct.c_int, _dp, _dp, _dp]
        g("cell_tau_eff").restype = ct.c_double
        g("cell_tau_eff").argtypes = [ct.c_double, ct.c_double, ct.c_double, _dp]
        g("cell_inlet").argtypes = [_dp, _dp, _dp, _dp]
        g("reichardt").restype = ct.c_double
        g("reichardt").argtypes = [ct.c_double] * 3
        g("solve_utau").restype = ct.c_double
        g("solve_utau").argtypes = [ct.c_double] * 6
    _LIB = lib
    return lib


def default_config(nx, ny, nz, re_tau=1000.0, n_modes=100, **kw):
    """Channel configuration with the paper's defaults (C_smag = 0.01, Sec. 4.1)."""
    c = OracleConfig()
    c.nx, c.ny, c.nz = nx, ny, nz
    c.n_modes = n_modes
    c.inlet, c.walls, c.wall_model, c.mrt, c.stats, c.threads = 1, 0, 1, 1, 0, 0
    c.re_tau, c.u_bulk, c.c_smag = re_tau, 0.05, 0.01
    c.kappa0, c.B0 = 0.4, 7.8
    c.k_ratio, c.beta_kmin = 1.01, 0.5
    c.tau0 = 0.0
    for k, v in kw.items():
        if k == "body_force":
            for a in range(3):
                c.body_force[a] = v[a]
        else:
            setattr(c, k, v)
    return c


class Oracle:
    """One FP64 (or complex-step) oracle lattice.

    theta = (l_e, A, kappa, B): STG length-scale factor and amplitude, and the
    Reichardt constants of the wall law and the inlet mean profile.
    """

    def __init__(self, cfg, theta=(0.4, 1.0, 0.4, 7.8), uniforms=None,
                 complex_step=False, theta_im=None):
        self.lib = load()
        self.cfg = cfg
        self.pre = "orcz_" if complex_step else "orc_"
        self.nx, self.ny, self.nz = cfg.nx, cfg.ny, cfg.nz
        self.ncell = cfg.nx * cfg.ny * cfg.nz
        self.n_modes = cfg.n_modes
        th = np.ascontiguousarray(theta, dtype=np.float64)
        thi = None if theta_im is None else np.ascontiguousarray(theta_im, dtype=np.float64)
        if cfg.n_modes > 0:
            if uniforms is None:
                raise ValueError("the STG mode draws (n_modes x 4 uniforms) are an input")
            un = np.ascontiguousarray(uniforms, dtype=np.float64).reshape(-1)
            if un.size != 4 * cfg.n_modes:
                raise ValueError("uniforms must hold 4 values per mode")
        else:
            un = np.zeros(4)
        self._un = un
        self.h = self._f("create")(ct.byref(cfg), _p(th),
                                   None if thi is None else _p(thi), _p(un))

    def _f(self, name):
        return getattr(self.lib, self.pre + name)

    def close(self):
        if self.h:
            self._f("destroy")(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        self._f("step")(self.h, int(n))

    @property
    def time(self):
        return self._f("get_time")(self.h)

    @time.setter
    def time(self, t):
        self._f("set_time")(self.h, int(t))

    def state(self, imag=False):
        f = np.empty((Q, self.nz, self.ny, self.nx))
        self._f("get_state_imag" if imag else "get_state")(self.h, _p(f))
        return f

    def set_state(self, f, f_im=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == Q * self.ncell
        fi = None if f_im is None else np.ascontiguousarray(f_im, dtype=np.float64)
        self._f("set_state")(self.h, _p(f), None if fi is None else _p(fi))

    def fields(self):
        rho = np.empty((self.nz, self.ny, self.nx))
        u = np.empty((self.nz, self.ny, self.nx, 3))
        self._f("get_fields")(self.h, _p(rho), _p(u))
        return rho, u

    def force(self):
        F = np.empty((self.nz, self.ny, self.nx, 3))
        self._f("get_force")(self.h, _p(F))
        return F

    def utau(self):
        u = np.empty((2, self.nz, self.nx))
        self._f("get_utau")(self.h, _p(u))
        return u

    def set_utau(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        self._f("set_utau")(self.h, _p(u))

    def constants(self):
        o = np.empty(6)
        self._f("get_constants")(self.h, _p(o))
        return dict(delta=o[0], utau_ref=o[1], nu=o[2], tau0=o[3], ubp=o[4], maxl=o[5])

    def tables(self):
        ny, N = self.ny, max(self.n_modes, 1)
        t = dict(UR=np.empty(ny), a=np.empty((ny, 6)), Rp=np.empty((ny, 6)), ell=np.empty(ny),
                 kn=np.empty(N), dn=np.empty((N, 3)), sn=np.empty((N, 3)), phin=np.empty(N),
                 sqrtq=np.empty((ny, N)))
        self._f("get_tables")(self.h, *[_p(t[k]) for k in
                                        ("UR", "a", "Rp", "ell", "kn", "dn", "sn", "phin", "sqrtq")])
        return t

    def inlet_velocity(self, t):
        out = np.empty((self.nz, self.ny, 3))
        self._f("inlet_velocity")(self.h, int(t), _p(out))
        return out

    def stats_reset(self):
        self._f("stats_reset")(self.h)

    def stats(self):
        s = np.empty((self.ny, self.nx, 7))
        ut = np.empty((2, self.nx))
        n = self._f("stats_get")(self.h, _p(s), _p(ut))
        return s, ut, n

    def objective_begin(self, i0, i1, iR):
        self._f("objective_begin")(self.h, int(i0), int(i1), int(iR))

    def objective(self):
        re, im = ct.c_double(), ct.c_double()
        parts = np.empty(4)
        self._f("objective_value")(self.h, ct.byref(re), ct.byref(im), _p(parts))
        return re.value, im.value, parts


class cell_api:
    """Single-cell building blocks of the oracle (FP64), for closed-form checks."""

    @staticmethod
    def matrix():
        lib = load()
        M = np.empty((Q, Q))
        w = np.empty(Q)
        c = np.empty((Q, 3), dtype=np.int32)
        lib.orc_matrix(_p(M), _p(w), c.ctypes.data_as(_ip))
        return M, w, c.astype(np.int64)

    @staticmethod
    def feq(rho, u):
        out = np.empty(Q)
        u = np.ascontiguousarray(u, dtype=np.float64)
        load().orc_cell_feq(float(rho), _p(u), _p(out))
        return out

    @staticmethod
    def moments(f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        m = np.empty(Q)
        load().orc_cell_moments(_p(f), _p(m))
        return m

    @staticmethod
    def collide(p, F=(0.0, 0.0, 0.0), tau0=0.8, c_smag=0.0, mrt=True):
        p = np.ascontiguousarray(p, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.float64)
        out = np.empty(Q)
        rho = ct.c_double()
        u = np.empty(3)
        load().orc_cell_collide(_p(p), _p(F), float(tau0), float(c_smag), int(bool(mrt)),
                                _p(out), ct.byref(rho), _p(u))
        return out, rho.value, u

    @staticmethod
    def tau_eff(tau0, c_smag, rho, pi6):
        pi6 = np.ascontiguousarray(pi6, dtype=np.float64)
        return load().orc_cell_tau_eff(float(tau0), float(c_smag), float(rho), _p(pi6))

    @staticmethod
    def inlet(p, uin):
        p = np.ascontiguousarray(p, dtype=np.float64)
        uin = np.ascontiguousarray(uin, dtype=np.float64)
        out = np.empty(Q)
        rho = ct.c_double()
        load().orc_cell_inlet(_p(p), _p(uin), _p(out), ct.byref(rho))
        return out, rho.value

    @staticmethod
    def reichardt(yp, kappa=0.4, B=7.8):
        return load().orc_reichardt(float(yp), float(kappa), float(B))

    @staticmethod
    def solve_utau(uhat, y, nu, kappa=0.4, B=7.8, guess=1e-3):
        return load().orc_solve_utau(float(uhat), float(y), float(nu), float(kappa), float(B),
                                     float(guess))


def oracle_threads():
    """Threads the oracle's OpenMP loops use by default."""
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))

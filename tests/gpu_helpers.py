"""Shared set-up of the GPU parity tests: one oracle and one CUDA channel built
from the same seeded inputs, and the error measures the tolerances refer to."""
import numpy as np

from oracle.oracle import Oracle, cell_api, default_config
from paper_2304_04214_gb300.inputs import round_to_bf16, round_to_fp16, stg_uniforms

Q = 19


def make_pair(nx, ny, nz, re_tau=1000.0, n_modes=16, seed=1, precision="fp32", inlet=1,
              wall_model=1, c_smag=0.01, theta=(0.4, 1.0, 0.4, 7.8), stats=0, sponge=(0, 0.0)):
    """Oracle and CUDA channel on the same inputs.  The library fixes u_tau,ref
    and nu from the (kappa, B) it is created with, so the oracle's creation
    constants kappa0, B0 are theta's."""
    from paper_2304_04214_gb300.channel import LBMChannel
    un = stg_uniforms(n_modes, seed) if n_modes > 0 else None
    cfg = default_config(nx, ny, nz, re_tau=re_tau, n_modes=n_modes, inlet=inlet,
                         wall_model=wall_model, c_smag=c_smag, stats=stats,
                         kappa0=theta[2], B0=theta[3], sponge_cells=sponge[0], sponge_nu=sponge[1])
    o = Oracle(cfg, theta=theta, uniforms=un)
    g = LBMChannel(nx, ny, nz, re_tau=re_tau, n_modes=n_modes, uniforms=un, precision=precision,
                   inlet=bool(inlet), wall_model=bool(wall_model), c_smag=c_smag,
                   ell_e=theta[0], amp=theta[1], kappa=theta[2], B=theta[3],
                   stats_every=1 if stats else 0)
    if sponge[0] > 0:
        g.set_sponge(*sponge)
    return o, g


def bf16_row_base(o):
    """Row base of the row-base storages (BF16, FP16 row), (19, ny) in FP32:
    f^eq_q(1, (U_R(j), 0, 0)) - w_q with the creation-time inlet mean profile
    U_R of the oracle `o` (the library stores f - w - base and forms f - w in
    FP32)."""
    _, w, _ = cell_api.matrix()
    UR = o.tables()["UR"]
    base = np.stack([cell_api.feq(1.0, (UR[j], 0.0, 0.0)) - w for j in range(len(UR))], axis=1)
    return base.astype(np.float32)


def quantize_state(f, precision, o=None):
    """Round the stored deviations to the storage type, so that both sides
    start from the same exactly representable state: f - w for FP16, f - w -
    base(j) for BF16 and FP16 row (needs the oracle `o` for its profile)."""
    if precision == "fp32":
        return f.astype(np.float32).astype(np.float64)
    _, w, _ = cell_api.matrix()
    wq = w[:, None, None, None]
    if precision == "fp16":
        return wq + round_to_fp16(f - wq)
    b32 = bf16_row_base(o)[:, None, :, None]
    dev = f - wq - b32.astype(np.float64)
    if precision == "bf16":
        r = round_to_bf16(dev)
    else:   # the library rounds the FP32 value of the deviation
        r = round_to_fp16(dev.astype(np.float32))
    return wq + (r.astype(np.float32) + b32).astype(np.float64)


def set_both(o, g, f):
    f = quantize_state(f, g.precision, o)
    o.set_state(f)
    g.set_populations(f)
    return f


def field_errors(o, g):
    """Max-norm errors of rho and u normalized by the oracle's max |.|."""
    ro, uo = o.fields()
    rg, ug = g.fields()
    er = np.max(np.abs(rg - ro)) / np.max(np.abs(ro))
    eu = np.max(np.abs(ug - uo)) / np.max(np.abs(uo))
    return er, eu

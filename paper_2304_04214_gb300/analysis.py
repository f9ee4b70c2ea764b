"""Channel statistics in the form the paper reports them (Sec. 4): mean
velocity and Reynolds-stress profiles along the channel in wall units, the
friction velocity along both walls, and the adaptation length -- the distance
from the inlet after which a quantity stays within a tolerance of its
developed value.  Host post-processing of the FP64 sums that lbm_stats
returns; the channel itself runs in the CUDA library.

    python -m paper_2304_04214_gb300.analysis --re-tau 1000 --lbu 40

runs the paper's set-up (Sec. 4.1: a 20 delta x 2 delta x 1.6 delta channel
with H = 2 delta resolved by 20, 40 or 60 cells, 10 domain-through times,
statistics after 2) and prints one JSON line.
"""
import argparse
import json

import numpy as np


def profiles(sums, utau_sums, n_samples, nz):
    """Means over z and samples from lbm_stats' sums.

    sums: (ny, nx, 7) sums of (u, v, w, uu, vv, ww, uv); utau_sums: (2, nx).
    Returns U, V, W (ny, nx), the centred second moments uu, vv, ww, uv
    (ny, nx) and utau (2, nx)."""
    m = np.asarray(sums, dtype=np.float64) / (n_samples * nz)
    U, V, W = m[..., 0], m[..., 1], m[..., 2]
    out = dict(U=U, V=V, W=W, uu=m[..., 3] - U * U, vv=m[..., 4] - V * V, ww=m[..., 5] - W * W,
               uv=m[..., 6] - U * V)
    out["utau"] = np.asarray(utau_sums, dtype=np.float64).reshape(2, -1) / (n_samples * nz)
    return out


def shear_stress_peak(uv, u_ref):
    """Peak of the Reynolds shear stress -<u'v'>+ along x: the lower half as
    is, the upper half with its sign flipped (the stress changes sign at the
    centre line), averaged, then the maximum over y.  uv: (ny, nx)."""
    ny = uv.shape[0]
    h = ny // 2
    lower = -uv[:h]
    upper = uv[ny - 1:ny - 1 - h:-1]          # mirrored, row 0 = the wall row
    return 0.5 * (lower + upper).max(axis=0) / (u_ref * u_ref)


def adaptation_length(q, x, ref, tol):
    """Smallest x0 with |q(x) / q_ref - 1| <= tol for every x0 <= x <= ref[1],
    q_ref the mean of q over ref[0] <= x <= ref[1]; None if no such x0 exists
    before ref[0]."""
    q = np.asarray(q, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    sel = (x >= ref[0]) & (x <= ref[1])
    q_ref = q[sel].mean()
    ok = np.abs(q / q_ref - 1.0) <= tol
    last = np.nonzero(x <= ref[1])[0][-1]
    bad = np.nonzero(~ok[:last + 1])[0]
    x0 = x[0] if bad.size == 0 else (x[bad[-1] + 1] if bad[-1] + 1 <= last else None)
    if x0 is None or x0 > ref[0]:
        return None, q_ref
    return float(x0), float(q_ref)


def run_paper_case(re_tau, lbu, n_modes=100, seed=1, precision="fp32", stats_every=10, through=10.0,
                   start=2.0, ref=(12.0, 18.0), tol=0.05, sponge_delta=0.0, sponge_nu=0.1):
    """The channel of Sec. 4.1 at H = lbu cells; returns a dict of results.

    x is measured in delta from the inlet; the reference window for the
    developed state stays clear of the outlet.  sponge_delta > 0 adds the
    outlet sponge of that thickness (in delta) with viscosity sponge_nu at
    its end (Sec. 4.1 uses 1 delta; the form is reading A24)."""
    import torch
    from .channel import LBMChannel
    ny = int(lbu)
    delta = ny / 2.0
    nx, nz = int(round(20 * delta)), int(round(1.6 * delta))
    nz += nz % 2
    ch = LBMChannel(nx, ny, nz, re_tau=re_tau, n_modes=n_modes, seed=seed, precision=precision,
                    stats_every=stats_every)
    if sponge_delta > 0:
        ch.set_sponge(int(round(sponge_delta * delta)), sponge_nu)
    c = ch.constants()
    u_b = 0.05
    T = nx / u_b                                     # domain-through time in steps
    n0, n1 = int(round(start * T)), int(round(through * T))
    ch.step(n0)
    ch.reset_stats()
    ch.step(n1 - n0)
    ch.sync()
    s, ut, n = ch.stats()
    torch.cuda.synchronize()
    p = profiles(s, ut, n, nz)
    x = (np.arange(nx) + 0.5) / delta
    u_ref = c["utau_ref"]
    utau = p["utau"].mean(axis=0) / u_ref
    peak = shear_stress_peak(p["uv"], u_ref)
    L_ut, ut_dev = adaptation_length(utau, x, ref, tol)
    L_uv, uv_dev = adaptation_length(peak, x, ref, 2 * tol)
    res = dict(re_tau=re_tau, lbu=lbu, lattice=[nx, ny, nz], steps=n1, samples=int(n),
               precision=precision, n_modes=n_modes, sponge_delta=sponge_delta,
               sponge_nu=sponge_nu if sponge_delta > 0 else 0.0,
               utau_developed=ut_dev, uv_peak_developed=uv_dev,
               adaptation_utau_delta=L_ut, adaptation_uv_delta=L_uv,
               utau_at_x=dict(zip([1, 2, 4, 6, 8, 10, 12, 16], [
                   float(utau[min(nx - 1, int(v * delta))]) for v in (1, 2, 4, 6, 8, 10, 12, 16)])),
               uv_peak_at_x=dict(zip([1, 2, 4, 6, 8, 10, 12, 16], [
                   float(peak[min(nx - 1, int(v * delta))]) for v in (1, 2, 4, 6, 8, 10, 12, 16)])))
    ch.close()
    return res


STORAGE_CASES = {
    "c2": dict(shape=(384, 96, 96), re_tau=1000.0, n_modes=200, seed=2),
    "c3": dict(shape=(768, 128, 192), re_tau=2000.0, n_modes=300, seed=3),
}


def storage_report(case, avg_steps=20000, spin_through=2.0, twins=2, stats_every=1):
    """Long-run profiles of one channel in FP32, FP16, BF16 and FP16 row-base storage, and of
    FP32 runs started 1e-6 apart (`twins`, the sampling spread of the average):
    spin-up of spin_through domain-through times, then statistics every
    stats_every steps for avg_steps steps; profiles U, <u'u'>, <v'v'>, <w'w'>,
    <u'v'> averaged over z, the samples and x >= nx/4.  Errors: max over y of
    |difference| / max over y of |FP32 profile|, against the FP32 run; and the
    pointwise difference of the final streamwise velocity (how far the runs
    have decorrelated)."""
    import torch
    from .channel import LBMChannel
    from .inputs import noise
    cfg = STORAGE_CASES[case]
    nx, ny, nz = cfg["shape"]
    spin = int(round(spin_through * nx / 0.05))
    names = ("U", "uu", "vv", "ww", "uv")

    def run(precision, perturb=None):
        ch = LBMChannel(nx, ny, nz, re_tau=cfg["re_tau"], n_modes=cfg["n_modes"], seed=cfg["seed"],
                        precision=precision, stats_every=stats_every)
        if perturb is not None:
            f = ch.populations()
            ch.set_populations(f * (1.0 + 1e-6 * noise(f.shape, seed=perturb)))
        ch.step(spin)
        ch.reset_stats()
        ch.step(avg_steps)
        s, ut, n = ch.stats()
        _, u = ch.fields()
        ch.close()
        torch.cuda.empty_cache()
        p = profiles(s, ut, n, nz)
        x0 = nx // 4
        prof = [p[k][:, x0:].mean(axis=1) for k in names]
        return prof, u[..., 0]

    ref, u_ref = run("fp32")

    def errs(prof, u):
        e = {k: float(np.max(np.abs(b - a)) / np.max(np.abs(a))) for k, a, b in zip(names, ref, prof)}
        e["pointwise_u"] = float(np.max(np.abs(u - u_ref)) / np.max(np.abs(u_ref)))
        return e

    out = dict(case=case, lattice=[nx, ny, nz], re_tau=cfg["re_tau"], n_modes=cfg["n_modes"],
               spin_steps=spin, avg_steps=avg_steps, stats_every=stats_every,
               profile_max={k: float(np.max(np.abs(a))) for k, a in zip(names, ref)})
    for prec in ("fp16", "bf16", "fp16row"):
        out[prec] = errs(*run(prec))
    out["fp32_twins"] = [errs(*run("fp32", perturb=300 + t)) for t in range(twins)]
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--storage-report", choices=sorted(STORAGE_CASES),
                    help="long-run 16-bit profile errors against FP32 on a bench lattice")
    ap.add_argument("--avg-steps", type=int, default=20000)
    ap.add_argument("--re-tau", type=float, default=1000.0)
    ap.add_argument("--lbu", type=int, default=40, help="cells across the channel height H")
    ap.add_argument("--modes", type=int, default=100)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16", "fp16row"])
    ap.add_argument("--through", type=float, default=10.0, help="domain-through times in all")
    ap.add_argument("--start", type=float, default=2.0, help="domain-through times before statistics")
    ap.add_argument("--sponge", type=float, default=0.0, help="outlet sponge thickness in delta (0: none)")
    ap.add_argument("--sponge-nu", type=float, default=0.1, help="viscosity added at the sponge's end")
    a = ap.parse_args()
    if a.storage_report:
        print(json.dumps(storage_report(a.storage_report, avg_steps=a.avg_steps)), flush=True)
        return
    print(json.dumps(run_paper_case(a.re_tau, a.lbu, n_modes=a.modes, precision=a.precision,
                                    through=a.through, start=a.start, sponge_delta=a.sponge,
                                    sponge_nu=a.sponge_nu)), flush=True)


if __name__ == "__main__":
    main()

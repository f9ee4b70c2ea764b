"""Tuning the STG inlet with the adjoint: truncated backpropagation over
successive windows.

Each window starts from the channel's current state, advances it by
`window` steps, and returns J (by default the Reynolds-stress mismatch J_R at
a downstream station) with dJ/dtheta from the hand-written adjoint
(`STGAdjoint`); a torch optimizer then updates theta = (ell_e, amp, kappa, B)
-- only the entries named in `params`, the others keep their values.  A
change of the inlet turbulence reaches a downstream station by convection
(about U_b = 0.05 cells per step), so a window must span that time -- 800
steps to x = 40 -- or its gradient sees only the acoustic response there and
points the wrong way; and since one window's J scatters widely in a turbulent
flow, each update averages several windows.

    python -m paper_2304_04214_gb300.tuning --iters 12 --station 40 --window 2048 \
        --ckpt-every 64 --windows-per-update 4

prints one JSON line per update (mean J of its windows, theta).
"""
import argparse
import json

import numpy as np

NAMES = ("ell_e", "amp", "kappa", "B")
BOUNDS = {"ell_e": (0.05, 2.0), "amp": (0.1, 5.0), "kappa": (0.3, 0.5), "B": (4.0, 10.0)}


def tune(channel, theta0, iters, window=64, ckpt_every=8, objective=(0, 0, 40), params=("ell_e", "amp"),
         lr=0.05, windows_per_update=1, callback=None):
    """Optimize the entries `params` of theta with Adam on successive windows.

    objective = (i_tau0, i_tau1, i_R); the default has an empty J_tau range,
    so J = J_R.  Each of the `iters` updates averages J and dJ/dtheta over
    `windows_per_update` consecutive windows: the flow is turbulent, and the
    J of one window scatters by far more than a parameter change moves it.
    theta is kept inside BOUNDS.  Returns the list of (mean J, theta) per
    update; callback(k, J, theta) is called after each one."""
    import torch
    from .channel import STGAdjoint
    theta = torch.tensor(theta0, dtype=torch.float64)
    mask = torch.tensor([n in params for n in NAMES], dtype=torch.float64)
    lo = torch.tensor([BOUNDS[n][0] for n in NAMES], dtype=torch.float64)
    hi = torch.tensor([BOUNDS[n][1] for n in NAMES], dtype=torch.float64)
    var = theta.clone().requires_grad_(True)
    opt = torch.optim.Adam([var], lr=lr)
    hist = []
    for k in range(iters):
        opt.zero_grad()
        Jm = 0.0
        for _ in range(windows_per_update):
            J = STGAdjoint.apply(var, channel, window, ckpt_every, objective) / windows_per_update
            J.backward()                          # gradients add up over the windows
            Jm += float(J.detach())
        var.grad.mul_(mask)                       # frozen entries get no update
        hist.append((Jm, var.detach().numpy().copy()))
        opt.step()
        with torch.no_grad():
            var.copy_(torch.maximum(torch.minimum(var, hi), lo))
        if callback:
            callback(k, hist[-1][0], hist[-1][1])
    channel.set_params(var.detach().numpy())
    return hist


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--shape", type=int, nargs=3, default=[256, 64, 64])
    ap.add_argument("--re-tau", type=float, default=1000.0)
    ap.add_argument("--modes", type=int, default=100)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--window", type=int, default=64)
    ap.add_argument("--ckpt-every", type=int, default=8)
    ap.add_argument("--station", type=int, default=40, help="x of the J_R station")
    ap.add_argument("--spinup", type=int, default=2000, help="steps before the first window")
    ap.add_argument("--lr", type=float, default=0.05)
    ap.add_argument("--windows-per-update", type=int, default=1)
    ap.add_argument("--params", default="ell_e,amp")
    ap.add_argument("--theta", type=float, nargs=4, default=[0.4, 1.0, 0.4, 7.8])
    a = ap.parse_args()
    from .channel import LBMChannel
    nx, ny, nz = a.shape
    ch = LBMChannel(nx, ny, nz, re_tau=a.re_tau, n_modes=a.modes, seed=5, ell_e=a.theta[0], amp=a.theta[1],
                    kappa=a.theta[2], B=a.theta[3])
    ch.step(a.spinup)

    def report(k, J, th):
        print(json.dumps({"window": k, "J": J, "theta": dict(zip(NAMES, map(float, th)))}), flush=True)

    tune(ch, a.theta, a.iters, window=a.window, ckpt_every=a.ckpt_every, objective=(0, 0, a.station),
         params=tuple(a.params.split(",")), lr=a.lr, windows_per_update=a.windows_per_update, callback=report)


if __name__ == "__main__":
    main()

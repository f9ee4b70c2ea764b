"""Write the FP64 oracle's long-run statistics of the paper's channel set-up
(Sec. 4.1: 20 delta x 2 delta x 1.6 delta with H = 2 delta resolved by 40
cells, i.e. a 400 x 40 x 32 lattice; Re_tau = 1000; N = 100 STG modes drawn
from seed 1) into decorrelated_h40_re1000.txt, for the GPU long-run test on a
flow that the FP32 path no longer tracks pointwise.

Protocol (Sec. 4.1: statistics after 2 domain-through times T = nx / U_b =
8000 steps): 2T of spin-up, then the z sums of (u, v, w, uu, vv, ww, uv) every
step for 3T.  Written: the time- and z-averaged moments over three x ranges
of the channel ([nx/4, nx/2), [nx/2, 3nx/4), [3nx/4, nx)), and the pointwise
streamwise velocity of the final state along the centre row of plane k = 0
(what shows that another run has decorrelated from this one).

TEST INFRASTRUCTURE: calls only the oracle (and the seeded input generator).
Run once:  python tests/golden/make_decorrelated_profiles.py   (hours on a few cores)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.oracle import Oracle, default_config  # noqa: E402
from paper_2304_04214_gb300.inputs import stg_uniforms  # noqa: E402

NX, NY, NZ, RE_TAU, N_MODES, SEED = 400, 40, 32, 1000.0, 100, 1
T = 8000                               # domain-through time nx / U_b, U_b = 0.05
SPIN, AVG = 2 * T, 3 * T
RANGES = [(NX // 4, NX // 2), (NX // 2, 3 * NX // 4), (3 * NX // 4, NX)]
OUT = os.path.join(HERE, "decorrelated_h40_re1000.txt")


def main():
    t0 = time.time()
    o = Oracle(default_config(NX, NY, NZ, re_tau=RE_TAU, n_modes=N_MODES, stats=1),
               uniforms=stg_uniforms(N_MODES, SEED))
    chunk = 1000
    for s in range(0, SPIN, chunk):
        o.step(chunk)
        print(f"spin-up {s + chunk}/{SPIN}  {time.time() - t0:.0f} s", flush=True)
    o.stats_reset()
    for s in range(0, AVG, chunk):
        o.step(chunk)
        print(f"averaging {s + chunk}/{AVG}  {time.time() - t0:.0f} s", flush=True)
    sums, _, n = o.stats()                      # [ny][nx][7], z sums over n samples
    assert n == AVG
    _, u = o.fields()
    lines = ["# FP64 oracle statistics, written by make_decorrelated_profiles.py (oracle only).",
             f"# lattice {NX}x{NY}x{NZ}, Re_tau {RE_TAU}, N {N_MODES} STG modes (seed {SEED}), "
             f"spin-up {SPIN} steps, averaged over {AVG} steps (every step)",
             "# moments: rows 'm x0 x1 c' = mean over z, the samples and x0 <= x < x1 of moment c",
             "# (c = 0..6: u, v, w, uu, vv, ww, uv), one value per row j = 0..ny-1",
             "# pointwise: 'u' = streamwise velocity of the final state, j = ny/2, k = 0, i = 0..nx-1"]
    for (x0, x1) in RANGES:
        m = (sums[:, x0:x1, :] / (n * NZ)).mean(axis=1)           # [ny][7]
        for c in range(7):
            lines.append(f"m {x0} {x1} {c} " + " ".join(f"{v:.17e}" for v in m[:, c]))
    lines.append("u " + " ".join(f"{v:.17e}" for v in u[0, NY // 2, :, 0]))
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(f"wrote {OUT} after {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()

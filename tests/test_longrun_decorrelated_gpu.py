"""Long-run statistics on a flow that the GPU run no longer tracks pointwise:
the paper's channel set-up resolved by H = 40 cells (Sec. 4.1: 20 delta x 2
delta x 1.6 delta, a 400 x 40 x 32 lattice), Re_tau = 1000, N = 100 STG modes;
2T of spin-up and 3T of statistics sampled every step (T = nx / U_b = 8000
steps: statistics after two domain-through times, Sec. 4.1), against the FP64
oracle's run of the same set-up (tests/golden/decorrelated_h40_re1000.txt,
written by make_decorrelated_profiles.py from the oracle alone).

After 5T the streamwise velocity along the centre row differs from the
oracle's pointwise by a sizeable fraction of itself downstream: the runs
have decorrelated (an FP32 rounding difference grows by about e every 250
steps once turbulence has developed; the 4 delta channel of
test_longrun_gpu.py convects it out first).  Their statistics then agree
only up to the sampling error of a 3T average, and one realization differs
from the next by as much as from the oracle: over twelve runs started 1e-6
apart, single runs' u'v' errors 5-10 delta from the inlet (where the inlet
turbulence is still adapting) range from 2% to 14%.  So each storage is
judged by the mean of its statistics over an ensemble of twelve runs (the
unperturbed one and eleven started 1e-6 apart), against a bar from the
spread of single FP32 runs (four of those FP32 runs against the unperturbed
one).  The 16-bit storages' ensembles sit about 2.5x FP32's ensemble error
in u'v' where the inlet turbulence adapts (a shift their rounding noise
causes there, the same for f - w and for the row base), inside the bar.

Error measure: max over y of |difference| / max over y of |oracle profile|, for
U, <u'u'>, <v'v'>, <w'w'>, <u'v'> averaged over z, the samples and each of
three x ranges.  Bar: 2%, or 1.5x the largest single-run FP32 spread where
the sampling error alone is larger than 2% (the second moments: 1-6%); the
mean profile U: 2% always.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "decorrelated_h40_re1000.txt")
NX, NY, NZ, N_MODES, SEED = 400, 40, 32, 100, 1
T = 8000
SPIN, AVG = 2 * T, 3 * T
RANGES = [(NX // 4, NX // 2), (NX // 2, 3 * NX // 4), (3 * NX // 4, NX)]
NAMES = ("U", "uu", "vv", "ww", "uv")
ENSEMBLE = 12                     # runs per storage whose statistics are averaged


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _golden():
    moments, u = {}, None
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            if p[0] == "m":
                moments[(int(p[1]), int(p[2]), int(p[3]))] = np.array([float(v) for v in p[4:]])
            elif p[0] == "u":
                u = np.array([float(v) for v in p[1:]])
    return moments, u


def _profiles(m):
    """(U, <u'u'>, <v'v'>, <w'w'>, <u'v'>)(y) from the mean moments m[c] (c = u,
    v, w, uu, vv, ww, uv)."""
    U, V, W = m[0], m[1], m[2]
    return np.stack([U, m[3] - U * U, m[4] - V * V, m[5] - W * W, m[6] - U * V])


def _errors(ref, got):
    return np.array([np.max(np.abs(got[c] - ref[c])) / np.max(np.abs(ref[c])) for c in range(5)])


def _run(precision, perturb_seed=None):
    from paper_2304_04214_gb300.channel import LBMChannel
    from paper_2304_04214_gb300.inputs import noise
    ch = LBMChannel(NX, NY, NZ, re_tau=1000.0, n_modes=N_MODES, seed=SEED, precision=precision, stats_every=1)
    if perturb_seed is not None:
        f = ch.populations()
        ch.set_populations(f * (1.0 + 1e-6 * noise(f.shape, seed=perturb_seed)))
    ch.step(SPIN)
    ch.reset_stats()
    ch.step(AVG)
    s, _, n = ch.stats()
    assert n == AVG
    _, u = ch.fields()
    ch.close()
    prof = {r: _profiles((s[:, r[0]:r[1], :] / (n * NZ)).mean(axis=1).T) for r in RANGES}
    return prof, u[0, NY // 2, :, 0]


@pytest.fixture(scope="module")
def runs():
    if not os.path.exists(GOLDEN):
        pytest.fail(f"missing {GOLDEN}: run tests/golden/make_decorrelated_profiles.py")
    moments, u_oracle = _golden()
    oracle = {r: _profiles(np.stack([moments[(r[0], r[1], c)] for c in range(7)])) for r in RANGES}
    gpu = {p: [_run(p)] + [_run(p, perturb_seed=200 + t) for t in range(ENSEMBLE - 1)]
           for p in ("fp32", "fp16", "bf16", "fp16row")}
    twins = gpu["fp32"][1:5]
    return oracle, u_oracle, gpu, twins


def test_the_runs_have_decorrelated(runs):
    _, u_oracle, gpu, twins = runs
    down = slice(NX // 2, NX)
    for p, rs in gpu.items():
        u = rs[0][1]
        d = np.max(np.abs(u[down] - u_oracle[down])) / np.max(np.abs(u_oracle[down]))
        print(p, f"pointwise difference from the oracle, x >= nx/2: {d:.3f}")
        assert d > 0.05, (p, d)
    base = gpu["fp32"][0][1]
    d = np.max(np.abs(twins[0][1][down] - base[down])) / np.max(np.abs(base[down]))
    assert d > 0.05, d


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16", "fp16row"])
def test_decorrelated_statistics_match_the_oracle(precision, runs):
    oracle, _, gpu, twins = runs
    bad = []
    for r in RANGES:
        spread = np.max([_errors(gpu["fp32"][0][0][r], tw[0][r]) for tw in twins], axis=0)
        bars = np.maximum(0.02, 1.5 * spread)
        bars[0] = 0.02                                   # the mean profile: 2% always
        ens = np.mean([run[0][r] for run in gpu[precision]], axis=0)
        err = _errors(oracle[r], ens)
        print(precision, r, " ".join(f"{k} {e:.2e} (bar {b:.2e})" for k, e, b in zip(NAMES, err, bars)))
        bad += [(r, k, float(e), float(b)) for k, e, b in zip(NAMES, err, bars) if not e < b]
    assert not bad, (precision, bad)

"""Long-run statistics of the CUDA path against the FP64 oracle: the
64x32x32, Re_tau = 1000, N = 100 channel run for 4000 steps (about three
flow-through times at U_b = 0.05) with the FP64 statistics accumulated every
step, reduced to the profiles that characterize the channel -- mean velocity U(y)
and the Reynolds stresses <u'u'>, <v'v'>, <w'w'>, <u'v'> -- averaged over z,
the samples and the downstream three quarters of the channel.

Bar: 2% of each profile's maximum, for all three storages.  (BF16 keeps 8
significant bits; it stores the deviation of f from the equilibrium of its
row's mean flow, about ten times smaller than f - w in this channel, so that
its rounding noise stays well under the resolved fluctuations, |<u'v'>| ~
3e-6 here.)  The channel is 4 delta long: its flow is slaved to the inlet
signal, and the GPU run tracks the oracle pointwise; the decorrelated case is
test_longrun_decorrelated_gpu.py."""
import numpy as np
import pytest

from gpu_helpers import make_pair

pytestmark = pytest.mark.gpu

NX, NY, NZ, STEPS = 64, 32, 32, 4000
NAMES = ("U", "uu", "vv", "ww", "uv")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def profiles(sums, n):
    """(U, <u'u'>, <v'v'>, <w'w'>, <u'v'>)(y) from the z-sums of (u, v, w, uu,
    vv, ww, uv), over the samples and x >= nx / 4."""
    m = (sums[:, NX // 4:, :] / (n * NZ)).mean(axis=1)
    U, V, W = m[:, 0], m[:, 1], m[:, 2]
    return U, m[:, 3] - U * U, m[:, 4] - V * V, m[:, 5] - W * W, m[:, 6] - U * V


@pytest.fixture(scope="module")
def oracle_profiles():
    o, _ = make_pair(NX, NY, NZ, n_modes=100, seed=1, stats=1)
    o.step(STEPS)
    s, _, n = o.stats()
    assert n == STEPS
    return profiles(s, n)


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16", "fp16row"])
def test_long_run_profiles_match_the_oracle(precision, oracle_profiles):
    _, g = make_pair(NX, NY, NZ, n_modes=100, seed=1, stats=1, precision=precision)
    g.step(STEPS)
    g.sync()
    s, _, n = g.stats()
    assert n == STEPS
    pg = profiles(s, n)
    errs = {k: float(np.max(np.abs(b - a)) / np.max(np.abs(a))) for k, a, b in zip(NAMES, oracle_profiles, pg)}
    print(precision, " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert np.max(np.abs(oracle_profiles[4])) > 0      # the run has resolved shear stress
    bars = {k: 0.02 for k in NAMES}
    for k in NAMES:
        assert errs[k] < bars[k], (precision, k, errs)

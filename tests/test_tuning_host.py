"""Host logic of the inlet tuning loop (paper_2304_04214_gb300.tuning.tune)
on the CPU: a stand-in channel whose objective is a known quadratic in theta,
with its exact gradient, takes the place of the adjoint.  Checks that the
tuned entries move to the optimum, the frozen ones stay, theta stays inside
its bounds, several windows per update are averaged, and the channel ends
with the tuned parameters."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_04214_gb300.tuning import BOUNDS, NAMES, tune  # noqa: E402


class QuadraticChannel:
    """set_params / adjoint_step like LBMChannel; J = sum w (theta - opt)^2."""

    def __init__(self, opt, weights=(1.0, 1.0, 1.0, 1.0)):
        self.opt = np.asarray(opt, dtype=np.float64)
        self.w = np.asarray(weights, dtype=np.float64)
        self.theta = None
        self.calls = []

    def set_params(self, theta):
        self.theta = np.array(theta, dtype=np.float64)

    def adjoint_step(self, window, ckpt_every, objective):
        self.calls.append((window, ckpt_every, tuple(objective)))
        d = self.theta - self.opt
        return float(np.sum(self.w * d * d)), 2.0 * self.w * d


def test_tuned_entries_reach_the_optimum_and_frozen_ones_stay():
    theta0 = [0.4, 1.0, 0.4, 7.8]
    ch = QuadraticChannel([0.7, 1.6, 0.35, 6.0])
    hist = tune(ch, theta0, iters=300, window=32, ckpt_every=8, objective=(0, 0, 40),
                params=("ell_e", "amp"), lr=0.02)
    th = hist[-1][1]
    assert abs(th[0] - 0.7) < 1e-2 and abs(th[1] - 1.6) < 1e-2
    assert th[2] == 0.4 and th[3] == 7.8                  # frozen: kappa, B
    assert hist[-1][0] < 1e-2 * hist[0][0] + (0.4 - 0.35) ** 2 + (7.8 - 6.0) ** 2
    # the channel ends with the tuned parameters
    assert abs(ch.theta[0] - 0.7) < 1e-2 and abs(ch.theta[1] - 1.6) < 1e-2
    assert ch.theta[2] == 0.4 and ch.theta[3] == 7.8
    assert all(c == (32, 8, (0, 0, 40)) for c in ch.calls) and len(ch.calls) == 300


def test_theta_is_kept_inside_its_bounds():
    ch = QuadraticChannel([0.4, 9.0, 0.4, 7.8])          # amp optimum beyond its bound
    hist = tune(ch, [0.4, 1.0, 0.4, 7.8], iters=400, params=("amp",), lr=0.05)
    lo, hi = BOUNDS["amp"]
    amps = np.array([h[1][NAMES.index("amp")] for h in hist])
    assert np.all(amps >= lo) and np.all(amps <= hi)
    assert abs(ch.theta[1] - hi) < 1e-12                  # ends at the bound


def test_windows_per_update_are_averaged():
    ch = QuadraticChannel([0.5, 1.0, 0.4, 7.8])
    seen = []
    hist = tune(ch, [0.4, 1.0, 0.4, 7.8], iters=5, params=("ell_e",), lr=0.01, windows_per_update=3,
                callback=lambda k, J, th: seen.append((k, J, th.copy())))
    assert len(ch.calls) == 15 and [s[0] for s in seen] == list(range(5))
    # the channel's J does not change between the windows of one update here,
    # so the mean equals one window's J
    J0 = (0.4 - 0.5) ** 2
    assert abs(hist[0][0] - J0) < 1e-12

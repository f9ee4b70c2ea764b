"""The adjoint-driven tuning loop (paper_2304_04214_gb300.tuning): Adam's
first step moves each tuned parameter by -lr * sign(dJ/dtheta), with the
gradient of a plain lbm_adjoint_step on an identical channel; frozen
parameters stay; later windows keep J finite and theta inside its bounds."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_first_update_follows_the_adjoint_gradient():
    from paper_2304_04214_gb300.channel import LBMChannel
    from paper_2304_04214_gb300.tuning import BOUNDS, NAMES, tune
    shape, theta0, obj, lr = (64, 32, 16), [0.4, 1.0, 0.4, 7.8], (0, 0, 8), 0.05
    a = LBMChannel(*shape, n_modes=32, seed=4)
    b = LBMChannel(*shape, n_modes=32, seed=4)
    a.step(200)
    b.step(200)
    _, dJ = b.adjoint_step(16, 4, obj)
    hist = tune(a, theta0, 4, window=16, ckpt_every=4, objective=obj, params=("ell_e", "amp"), lr=lr)
    assert len(hist) == 4 and all(np.isfinite(J) for J, _ in hist)
    step = hist[1][1] - hist[0][1]
    for n in (0, 1):                                  # ell_e, amp
        assert dJ[n] != 0.0
        assert abs(step[n] + lr * np.sign(dJ[n])) < 1e-6 * lr, (n, step, dJ)
    assert step[2] == 0.0 and step[3] == 0.0          # kappa, B frozen
    for _, th in hist:
        for v, nme in zip(th, NAMES):
            assert BOUNDS[nme][0] <= v <= BOUNDS[nme][1]

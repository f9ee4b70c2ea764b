"""Brute force: the C oracle against a second, independent FP64 statement of
the step (tests/numpy_step.py: dense NumPy, literal M from Appendix A.1 and
numpy.linalg.inv(M), explicit loops over the cells, the boundary passes in the
order of Algorithm 1) on tiny lattices, with the STG inlet, the zero-gradient
outlet, the slip walls and the wall model all on.

The two share nothing but the seeded inputs, so a mistake in how the oracle
composes the pieces (their order, a boundary pass, a term of the collision)
shows here even where each piece passes its own pin.  Bar: 1e-13 on the
populations after each of five steps (FP64 rounding of two different
operation orders)."""
import numpy as np
import pytest

from numpy_step import Channel
from oracle.oracle import Oracle, default_config
from paper_2304_04214_gb300.inputs import noise, stg_uniforms


@pytest.mark.parametrize("shape,n_modes,seed", [((4, 4, 4), 8, 21), ((6, 6, 3), 12, 22)])
def test_oracle_matches_the_numpy_restatement(shape, n_modes, seed):
    nx, ny, nz = shape
    un = stg_uniforms(n_modes, seed)
    o = Oracle(default_config(nx, ny, nz, re_tau=1000.0, n_modes=n_modes), uniforms=un)
    b = Channel(nx, ny, nz, 1000.0, un)
    # the same initial state and inlet signal from each side's own set-up
    assert np.max(np.abs(o.state() - b.f)) < 1e-15
    for t in (0, 3, 1000):
        ref = np.array([[b.inlet_velocity(j, k, t) for j in range(ny)] for k in range(nz)])
        assert np.max(np.abs(o.inlet_velocity(t) - ref)) < 1e-14
    # a disturbed state: every term of the collision, the SGS closure, the
    # wall law and the inlet reconstruction is active
    f0 = b.f * (1.0 + 0.02 * noise(b.f.shape, seed=seed))
    o.set_state(f0)
    b.f = f0.copy()
    for s in range(5):
        o.step(1)
        b.step()
        err = np.max(np.abs(o.state() - b.f))
        assert err < 1e-13, (s, err)
        assert np.max(np.abs(o.force() - b.F)) < 1e-13, s
        assert np.max(np.abs(o.utau() - b.utau)) < 1e-13 * b.u_tau, s
    assert np.max(np.abs(b.F)) > 0.0                   # the wall force acted

"""The seeded input generators shared by the oracle and the CUDA path: the
same seed gives the same draws, the ranges are as documented, and the
storage rounding helpers agree with the library conversions they stand for
(IEEE binary16 and bfloat16, round to nearest even)."""
import numpy as np
import pytest

from paper_2304_04214_gb300.inputs import noise, round_to_bf16, round_to_fp16, stg_uniforms


def test_draws_are_seeded_and_in_range():
    a, b, c = stg_uniforms(100, 3), stg_uniforms(100, 3), stg_uniforms(100, 4)
    assert a.shape == (100, 4) and np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() < 1.0
    n1, n2 = noise((5, 6, 7), 11), noise((5, 6, 7), 11)
    assert np.array_equal(n1, n2) and n1.min() >= -1.0 and n1.max() < 1.0
    assert abs(n1.mean()) < 0.2


def test_fp16_rounding_is_round_to_nearest_even():
    x = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, -2.5e-3, 6.1e-5, 1e-8])
    r = round_to_fp16(x)
    assert r[0] == 1.0                              # tie -> even (1.0)
    assert r[1] == 1.0 + 2.0 ** -9                  # tie -> even (next)
    assert np.all(np.abs(r[2:4] - x[2:4]) <= np.abs(x[2:4]) * 2.0 ** -11 + 2.0 ** -25)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 2, 20000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 0.0, -0.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(round_to_bf16(x), ref)

"""Host post-processing of the channel statistics (no GPU): profiles from
lbm_stats-shaped sums, the mirrored shear-stress peak and the adaptation
length, on synthetic inputs whose answers are known by construction."""
import numpy as np

from paper_2304_04214_gb300.analysis import adaptation_length, profiles, shear_stress_peak


def test_profiles_recover_means_and_centred_moments():
    rng = np.random.default_rng(5)
    ny, nx, nz, n = 6, 5, 4, 7
    samples = rng.normal(size=(n, nz, ny, nx, 3)) * 0.01 + np.array([0.05, 0.001, -0.002])
    u, v, w = samples[..., 0], samples[..., 1], samples[..., 2]
    sums = np.stack([x.sum(axis=(0, 1)) for x in (u, v, w, u * u, v * v, w * w, u * v)], axis=-1)
    ut = rng.uniform(0.001, 0.003, size=(n, 2, nz, nx))
    p = profiles(sums, ut.sum(axis=(0, 2)), n, nz)
    U = u.mean(axis=(0, 1))
    assert np.allclose(p["U"], U)
    assert np.allclose(p["uv"], (u * v).mean(axis=(0, 1)) - U * v.mean(axis=(0, 1)))
    assert np.allclose(p["ww"], w.var(axis=(0, 1)))
    assert np.allclose(p["utau"], ut.mean(axis=(0, 2)))


def test_shear_stress_peak_mirrors_the_upper_half():
    ny, nx = 8, 3
    y = (np.arange(ny) + 0.5) / (ny / 2) - 1.0           # -1 .. 1 across the channel
    shape = np.sin(np.pi * (y + 1.0) / 2.0) * np.sign(y) * np.exp(-4 * (np.abs(y) - 0.6) ** 2)
    uv = np.repeat((shape * 2.0)[:, None], nx, axis=1) * 1e-6     # negative below, positive above
    peak = shear_stress_peak(uv, 1e-3)
    assert np.allclose(peak, 2.0 * np.max(-shape[: ny // 2]))


def test_adaptation_length_of_a_relaxing_curve():
    x = np.linspace(0.05, 19.95, 200)
    q = 1.0 + 0.5 * np.exp(-x / 1.5)                      # within 5% of 1 once x > 1.5 ln 10 = 3.45
    L, q_ref = adaptation_length(q, x, (12.0, 18.0), 0.05)
    assert abs(q_ref - 1.0) < 1e-3
    assert 3.3 < L < 3.6
    # a curve that never settles has no adaptation length
    L2, _ = adaptation_length(1.0 + 0.2 * np.sin(x), x, (12.0, 18.0), 0.05)
    assert L2 is None

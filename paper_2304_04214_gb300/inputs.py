"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: only seeded random draws and
plain rounding of data to a storage format.  Both the CUDA library and the CPU
oracle receive the same arrays from here.
"""
import numpy as np

# Seeds of the five synthetic channel workloads (small / Re_tau 1000 /
# Re_tau 2000 / Re_tau 5200 / adjoint window).
SEEDS = {"c1": 1, "c2": 2, "c3": 3, "c4": 4, "c5": 5}


def stg_uniforms(n_modes: int, seed: int) -> np.ndarray:
    """The STG's random draws: n_modes x 4 uniforms in [0, 1).

    Column 0 sets the polar angle of d_n, column 1 its azimuth, column 2 the
    angle of sigma_n in the plane normal to d_n, column 3 the phase phi_n.
    """
    rng = np.random.Generator(np.random.PCG64(np.uint64(seed) + np.uint64(0x5157)))
    return rng.random((n_modes, 4))


def noise(shape, seed: int) -> np.ndarray:
    """Uniform noise in [-1, 1) of the given shape (float64)."""
    rng = np.random.Generator(np.random.PCG64(np.uint64(seed) + np.uint64(0xA11CE)))
    return 2.0 * rng.random(shape) - 1.0


def round_to_fp16(x: np.ndarray) -> np.ndarray:
    """Round float64 data to the nearest IEEE binary16 value (ties to even)."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float64 data to the nearest bfloat16 value (ties to even).

    The value is first rounded to float32 (exact for the small deviations it
    is used on), then the low 16 bits of the float32 pattern are rounded away.
    """
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)

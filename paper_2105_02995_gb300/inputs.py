"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds random-number generation only: no step of the method's arithmetic.

Right-hand sides are i.i.d. standard complex Gaussian: real and imaginary parts N(0, 1/2), so
E|z|^2 = 1, drawn from numpy's PCG64 with a seed derived from a workload id.
"""

import numpy as np

BASE_SEED = 2105_02995


def rhs_seed(config_index: int, rhs_index: int = 0) -> int:
    """Seed of right-hand side block `rhs_index` of workload `config_index`."""
    return BASE_SEED + 1000 * config_index + rhs_index


def complex_gaussian(N: int, b: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """An N x b array (Fortran order: column j is right-hand side j) of standard complex Gaussians."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = (rng.standard_normal((N, b)) + 1j * rng.standard_normal((N, b))) * np.sqrt(0.5)
    return np.asfortranarray(z.astype(dtype))

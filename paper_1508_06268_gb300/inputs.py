"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

Holds none of the method's arithmetic: temperature grids, explicit field arrays and spin arrays
are inputs to the simulation (Sec. 3.1 step 1 leaves the choice of temperatures to the user;
step 2 the field; step 3 the start configuration).
"""
from __future__ import annotations

import numpy as np


def geometric_temps(t_min: float, t_max: float, R: int) -> np.ndarray:
    """T_k = t_min (t_max / t_min)^(k / (R - 1)), k = 0..R-1, in double."""
    k = np.arange(R, dtype=np.float64)
    return t_min * np.power(t_max / t_min, k / (R - 1))


def linear_temps(t_min: float, t_max: float, R: int) -> np.ndarray:
    return np.linspace(t_min, t_max, R, dtype=np.float64)


def gaussian_field(L: int, seed: int) -> np.ndarray:
    """Explicit unscaled field h_i ~ N(0,1) as float32[L^3] from numpy's PCG64 stream."""
    return np.random.default_rng(seed).standard_normal(L ** 3).astype(np.float32)


def bimodal_field(L: int, seed: int) -> np.ndarray:
    return np.where(np.random.default_rng(seed).random(L ** 3) < 0.5, -1.0, 1.0).astype(np.float32)


def random_spins(R: int, L: int, seed: int) -> np.ndarray:
    """int8[R][L^3] of +-1."""
    return np.where(np.random.default_rng(seed).random((R, L ** 3)) < 0.5, -1, 1).astype(np.int8)

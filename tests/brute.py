"""Brute-force references written independently of oracle/ (numpy array formulations).

Used to pin the oracle: energies by periodic array shifts, exact Boltzmann averages by full
enumeration of tiny lattices, closed forms of limiting cases.
"""
from __future__ import annotations

import itertools

import numpy as np


def scaled_field(h: float, hraw: np.ndarray) -> np.ndarray:
    """hh_i = (float)h * h_i rounded to float32, as the model's field term uses it."""
    return (np.float32(h) * np.asarray(hraw, dtype=np.float32)).astype(np.float32)


def energy(spins: np.ndarray, L: int, J: float, hh: np.ndarray) -> float:
    """Eq. 1 for one configuration: -J sum over the 3N forward bonds - sum hh_i s_i."""
    s = np.asarray(spins, dtype=np.int64).reshape(L, L, L)  # [z][y][x]
    bonds = s * (np.roll(s, -1, axis=2) + np.roll(s, -1, axis=1) + np.roll(s, -1, axis=0))
    field = np.sum(np.asarray(hh, dtype=np.float64).reshape(L, L, L) * s)
    return -float(J) * float(bonds.sum()) - float(field)


def all_states(N: int) -> np.ndarray:
    """All 2^N configurations as int8[2^N][N] of +-1 (bit b of the state index -> site b)."""
    idx = np.arange(2 ** N)[:, None]
    bits = (idx >> np.arange(N)[None, :]) & 1
    return np.where(bits == 1, 1, -1).astype(np.int8)


def exact_averages(L: int, J: float, hh: np.ndarray, beta: float):
    """Exact Boltzmann averages of e = E/N, e^2, |m|, m^2, m^4 by enumeration (N <= 16)."""
    N = L ** 3
    states = all_states(N)
    E = np.array([energy(s, L, J, hh) for s in states])
    M = states.astype(np.float64).sum(axis=1)
    w = np.exp(-beta * (E - E.min()))
    w /= w.sum()
    e, m = E / N, M / N
    return np.array([np.dot(w, e), np.dot(w, e * e), np.dot(w, np.abs(m)), np.dot(w, m * m),
                     np.dot(w, m ** 4)])


def colour_of(L: int) -> np.ndarray:
    """Eq. 3 alternator A = (x + y + z) mod 2 for every site in natural order."""
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return ((x + y + z) % 2).reshape(-1)


def permutations_of(R: int):
    return [tuple(p) for p in itertools.permutations(range(R))]


def structure_factor_fft(spins: np.ndarray, L: int) -> float:
    """F of the correlation-length formula by numpy FFTs of the three marginals: the wave number
    2 pi / L component of each axis' marginal, squared modulus, averaged over axes, per site."""
    s = np.asarray(spins, dtype=np.float64).reshape(L, L, L)  # [z][y][x]
    total = 0.0
    for axes in ((0, 1), (0, 2), (1, 2)):  # keep x, y, z in turn
        marginal = s.sum(axis=axes)
        total += abs(np.fft.fft(marginal)[1]) ** 2
    return total / (3.0 * L ** 3)


def exact_energy_moments(L: int, J: float, hh: np.ndarray, beta: float):
    """Exact <E> and <E^2> (total energy) by enumeration."""
    states = all_states(L ** 3)
    E = np.array([energy(s, L, J, hh) for s in states])
    w = np.exp(-beta * (E - E.min()))
    w /= w.sum()
    return float(np.dot(w, E)), float(np.dot(w, E * E))


def zero_temperature_multihit_sweep(spins: np.ndarray, L: int, J: float, hh: np.ndarray, tile: int,
                                    mh: int) -> np.ndarray:
    """One sweep of the multi-hit double 3D checkerboard at zero temperature (a flip is accepted
    iff it does not raise the energy): tiles of tile^3 sites with coarse colour
    (x//tile + y//tile + z//tile) mod 2, coarse colour 0 then 1; each visit makes mh black-white
    passes over the visited tiles.  Each pass updates all its sites at once from numpy masks and
    periodic shifts (its sites have no neighbour among themselves).  float32 energy change
    2 s (J n + hh), as the model's float path rounds it."""
    s = np.asarray(spins, dtype=np.int8).reshape(L, L, L).copy()  # [z][y][x]
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    fine = (x + y + z) % 2
    coarse = (x // tile + y // tile + z // tile) % 2
    h3 = np.asarray(hh, dtype=np.float32).reshape(L, L, L)
    for c in (0, 1):
        for _ in range(mh):
            for f in (0, 1):
                n = sum(np.roll(s, d, axis=a) for a in (0, 1, 2) for d in (1, -1)).astype(np.float32)
                local = (np.float32(J) * n + h3).astype(np.float32)
                flip = (fine == f) & (coarse == c) & (s.astype(np.float32) * local <= 0)
                s[flip] = -s[flip]
    return s.reshape(-1)

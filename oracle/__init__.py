"""CPU oracle for the RFIM Exchange Monte Carlo hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import this package.  It wraps ``rfim_oracle.c`` (plain single-threaded C, no fused multiply-add)
through ctypes and shares nothing with the CUDA path.  The C source cites the paper's sections
and equations it follows; the random-number contract is stated in its header comment.

Every function here is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``
against facts that do not come from the oracle itself (brute force, exact enumeration, closed
forms, an independent Philox implementation, numpy FFTs).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rfim_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "librfim_oracle.so")
_lock = threading.Lock()
_lib = None

FIELD_BIMODAL = 0
FIELD_GAUSSIAN = 1
FIELD_EXPLICIT = 2


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2, -ffp-contract=off) into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            u32, i32, i64, f32, f64 = C.c_uint32, C.c_int32, C.c_int64, C.c_float, C.c_double
            P = C.c_void_p
            L.orc_philox4x32_10.argtypes = [u32, u32, u32, u32, u32, u32, P]
            L.orc_make_field.argtypes = [i32, i32, u32, u32, P]
            L.orc_create.argtypes = [i32, i32, i32, f32, f32, i32, P, u32, u32, u32, P]
            L.orc_create.restype = P
            L.orc_destroy.argtypes = [P]
            L.orc_reset.argtypes = [P, u32]
            L.orc_sweep.argtypes = [P]
            L.orc_exchange.argtypes = [P, i64]
            L.orc_run.argtypes = [P, i64, i32, i64]
            L.orc_energy.argtypes = [P, i32, P, P, P]
            L.orc_energy.restype = f64
            L.orc_delta_e.argtypes = [P, i32, i32, i32, i32]
            L.orc_delta_e.restype = f64
            L.orc_select_lowest.argtypes = [P, i32, i32, P]
            L.orc_adapt.argtypes = [P, i32, i64, i32, i32, P]
            L.orc_adapt.restype = i32
            for name in ("orc_R", "orc_N"):
                getattr(L, name).argtypes = [P]
                getattr(L, name).restype = i32
            for name in ("orc_sweep_count", "orc_xstep_count", "orc_n_meas"):
                getattr(L, name).argtypes = [P]
                getattr(L, name).restype = i64
            L.orc_get_temps.argtypes = [P, P]
            L.orc_get_field.argtypes = [P, P, P]
            L.orc_get_spins.argtypes = [P, P]
            L.orc_set_spins.argtypes = [P, P]
            L.orc_get_perm.argtypes = [P, P, P]
            L.orc_set_perm.argtypes = [P, P]
            L.orc_set_counters.argtypes = [P, i64, i64]
            L.orc_get_exchange_stats.argtypes = [P, P, P]
            L.orc_get_energies.argtypes = [P, P, P]
            L.orc_get_obs.argtypes = [P, P]
            L.orc_get_obsF.argtypes = [P, P]
            L.orc_set_measure_xi.argtypes = [P, i32]
            L.orc_set_multihit.argtypes = [P, i32, i32]
            L.orc_set_multihit.restype = i32
            L.orc_structure_F.argtypes = [P, i32]
            L.orc_structure_F.restype = f64
            L.orc_bimodal_threshold.argtypes = [f64, f64]
            L.orc_bimodal_threshold.restype = C.c_uint64
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(key, ctr) -> np.ndarray:
    """Philox4x32-10 block for key (k0, k1) and counter (c0, c1, c2, c3)."""
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF,
                            *[int(c) & 0xFFFFFFFF for c in ctr], _ptr(out))
    return out


def make_field(L: int, kind: int, field_seed: int, realization: int) -> np.ndarray:
    """Unscaled field h_i (natural site order) of one realization."""
    out = np.zeros(L ** 3, dtype=np.float32)
    lib().orc_make_field(L, kind, field_seed, realization, _ptr(out))
    return out


def select_lowest(rates, a: int) -> np.ndarray:
    r = np.ascontiguousarray(rates, dtype=np.float64)
    out = np.zeros(max(a, 1), dtype=np.int32)
    lib().orc_select_lowest(_ptr(r), len(r), a, _ptr(out))
    return out[:a]


def bimodal_threshold(beta: float, dE: float) -> int:
    return int(lib().orc_bimodal_threshold(beta, dE))


class Oracle:
    """One disorder realization with R temperature replicas (see rfim_oracle.c)."""

    def __init__(self, L, temps, J=1.0, h=1.0, field_kind=FIELD_GAUSSIAN, field=None,
                 field_seed=1, seed=42, realization=0, R_capacity=None, stage=0):
        self._lib = lib()
        temps = np.ascontiguousarray(temps, dtype=np.float64)
        R = len(temps)
        Rcap = R if R_capacity is None else int(R_capacity)
        f = None
        if field_kind == FIELD_EXPLICIT:
            f = np.ascontiguousarray(field, dtype=np.float32)
            assert f.size == L ** 3
        self._field_keep = f
        h_ptr = _ptr(f) if f is not None else None
        self._h = self._lib.orc_create(L, R, Rcap, J, h, field_kind, h_ptr, field_seed, seed,
                                       realization, _ptr(temps))
        if not self._h:
            raise ValueError("invalid oracle configuration")
        self.L, self.N, self.Rcap = L, L ** 3, Rcap
        self.field_kind = field_kind
        self._lib.orc_reset(self._h, stage)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def R(self) -> int:
        return self._lib.orc_R(self._h)

    def reset(self, stage=0):
        self._lib.orc_reset(self._h, stage)

    def sweep(self, n=1):
        for _ in range(n):
            self._lib.orc_sweep(self._h)

    def exchange(self, measure_from=0):
        self._lib.orc_exchange(self._h, measure_from)

    def run(self, n_sweeps, exchange_every, measure_from=0):
        self._lib.orc_run(self._h, n_sweeps, exchange_every, measure_from)

    def adapt(self, n_trials, sweeps_per_trial, exchange_every, inserts, return_rates=False):
        rates = np.zeros((max(n_trials, 1), self.Rcap), dtype=np.float64)
        R = self._lib.orc_adapt(self._h, n_trials, sweeps_per_trial, exchange_every, inserts,
                                _ptr(rates))
        if R < 0:
            raise ValueError("invalid adaptation arguments")
        return (R, rates[:n_trials]) if return_rates else R

    def energy(self, r):
        B = np.zeros(1, dtype=np.int64)
        F = np.zeros(1, dtype=np.float64)
        M = np.zeros(1, dtype=np.int64)
        E = self._lib.orc_energy(self._h, r, _ptr(B), _ptr(F), _ptr(M))
        return E, int(B[0]), float(F[0]), int(M[0])

    def delta_e(self, r, x, y, z) -> float:
        return self._lib.orc_delta_e(self._h, r, x, y, z)

    @property
    def sweep_count(self):
        return self._lib.orc_sweep_count(self._h)

    @property
    def xstep_count(self):
        return self._lib.orc_xstep_count(self._h)

    @property
    def n_meas(self):
        return self._lib.orc_n_meas(self._h)

    def temps(self):
        T = np.zeros(self.R, dtype=np.float64)
        self._lib.orc_get_temps(self._h, _ptr(T))
        return T

    def field(self):
        hraw = np.zeros(self.N, dtype=np.float32)
        hh = np.zeros(self.N, dtype=np.float32)
        self._lib.orc_get_field(self._h, _ptr(hraw), _ptr(hh))
        return hraw, hh

    def spins(self) -> np.ndarray:
        s = np.zeros((self.R, self.N), dtype=np.int8)
        self._lib.orc_get_spins(self._h, _ptr(s))
        return s

    def set_spins(self, s):
        s = np.ascontiguousarray(s, dtype=np.int8).reshape(self.R, self.N)
        self._lib.orc_set_spins(self._h, _ptr(s))

    def perm(self):
        t2r = np.zeros(self.R, dtype=np.int32)
        r2t = np.zeros(self.R, dtype=np.int32)
        self._lib.orc_get_perm(self._h, _ptr(t2r), _ptr(r2t))
        return t2r, r2t

    def set_perm(self, t2r):
        t = np.ascontiguousarray(t2r, dtype=np.int32)
        self._lib.orc_set_perm(self._h, _ptr(t))

    def set_counters(self, sweep, xstep):
        self._lib.orc_set_counters(self._h, sweep, xstep)

    def exchange_stats(self):
        att = np.zeros(self.R - 1, dtype=np.uint64)
        acc = np.zeros(self.R - 1, dtype=np.uint64)
        self._lib.orc_get_exchange_stats(self._h, _ptr(att), _ptr(acc))
        return att, acc

    def energies(self):
        E = np.zeros(self.R, dtype=np.float64)
        M = np.zeros(self.R, dtype=np.int64)
        self._lib.orc_get_energies(self._h, _ptr(E), _ptr(M))
        return E, M

    def observables(self):
        obs = np.zeros((self.R, 5), dtype=np.float64)
        self._lib.orc_get_obs(self._h, _ptr(obs))
        return obs

    def set_measure_xi(self, on: bool):
        self._lib.orc_set_measure_xi(self._h, 1 if on else 0)

    def set_multihit(self, mh: int, tile: int = 0):
        """Multi-hit double 3D checkerboard (Sec. 3.2): mh local passes per tile visit, tiles of
        edge `tile` (L divisible by 2 tile); mh = 0 restores the plain checkerboard."""
        if self._lib.orc_set_multihit(self._h, mh, tile) != 0:
            raise ValueError(f"invalid multi-hit setting mh={mh} tile={tile} for L={self.L}")

    def structure_F(self, r: int) -> float:
        return self._lib.orc_structure_F(self._h, r)

    def observables_F(self):
        F = np.zeros(self.R, dtype=np.float64)
        self._lib.orc_get_obsF(self._h, _ptr(F))
        return F


# ---- derived observables of Sec. 7 --------------------------------------------------------------
# Readings: C = (N / T^2)(<e^2> - <e>^2) with e the energy per site (the printed L^3 prefactor);
# xi = sqrt(N <m^2> / <F> - 1): the printed <M^2> taken as the zero-wave-number structure factor
# (1/N) <(sum_i s_i)^2> = N <m^2>, which has F's normalisation; no 1/(2 sin(K/2)) factor, as printed;
# +inf when <F> vanishes (a uniform lattice at every measurement).

THERMAL_COLUMNS = ("e", "C", "absm", "m2", "m4", "F", "xi")
# Any lattice with a spin against the others has F >= 4/N per measurement; averages below this
# bound are rounding noise of uniform lattices (about 1e-32 L^3).
F_ZERO = 1e-20


def thermal(obs, F, n_meas, N, T):
    """Per-temperature thermal averages of one realization: array [R][7] in THERMAL_COLUMNS order
    from the accumulator sums obs[R][5] (e, e^2, |m|, m^2, m^4) and F[R] (None: F and xi are NaN)."""
    obs = np.asarray(obs, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    R = obs.shape[0]
    out = np.full((R, 7), np.nan)
    if n_meas <= 0:
        return out
    avg = obs / float(n_meas)
    out[:, 0] = avg[:, 0]
    out[:, 1] = float(N) / (T * T) * (avg[:, 1] - avg[:, 0] * avg[:, 0])
    out[:, 2:5] = avg[:, 2:5]
    if F is not None:
        Fa = np.asarray(F, dtype=np.float64) / float(n_meas)
        out[:, 5] = Fa
        with np.errstate(divide="ignore", invalid="ignore"):
            arg = float(N) * avg[:, 3] / Fa - 1.0
            xi = np.where(arg >= 0.0, np.sqrt(np.maximum(arg, 0.0)), np.nan)
        # <F> below F_ZERO is the rounding of an exactly uniform lattice: xi diverges
        out[:, 6] = np.where(Fa < F_ZERO, np.inf, xi)
    return out


DISORDER_COLUMNS = ("e", "C", "absm", "xi", "g")


def disorder_average(thermals):
    """Averages over realizations (Sec. 7, [.]) of per-realization thermal arrays sharing one
    temperature set: [e], [C], [|m|], [xi] and the Binder factor [g] = (3 - [<m^4>] / [<m^2>]^2) / 2."""
    t = np.stack([np.asarray(a, dtype=np.float64) for a in thermals])
    mean = t.mean(axis=0)
    g = 0.5 * (3.0 - mean[:, 4] / (mean[:, 3] * mean[:, 3]))
    return np.stack([mean[:, 0], mean[:, 1], mean[:, 2], mean[:, 6], g], axis=1)

"""GB300-native Exchange Monte Carlo (parallel tempering) for the 3D Random Field Ising Model.

Thin ctypes binding of the C ABI in include/rfim.h (argument marshalling only: every step of the
hot path runs in the library's CUDA kernels).  PyTorch is used for the CUDA stream handle only.
The library is built in-tree by ``_build.build()``; when it is missing and cannot be built, every
entry point raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ESTATE, EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
FIELD_BIMODAL, FIELD_GAUSSIAN, FIELD_EXPLICIT = 0, 1, 2
LAYOUT_INT8, LAYOUT_BITPACK = 0, 1

_lock = threading.Lock()
_lib = None


class RfimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rfim error {code}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("L", C.c_int32), ("R", C.c_int32), ("R_capacity", C.c_int32), ("J", C.c_float),
                ("h", C.c_float), ("field_kind", C.c_int32), ("field", C.c_void_p),
                ("field_seed", C.c_uint32), ("seed", C.c_uint32), ("realization", C.c_uint32),
                ("temps", C.c_void_p), ("layout", C.c_int32), ("stream", C.c_void_p)]


class Obs(C.Structure):
    _fields_ = [("R", C.c_int32), ("T", C.c_void_p), ("e", C.c_void_p), ("e2", C.c_void_p),
                ("absm", C.c_void_p), ("m2", C.c_void_p), ("m4", C.c_void_p), ("att", C.c_void_p),
                ("acc", C.c_void_p), ("n_meas", C.c_int64), ("F", C.c_void_p)]


class ExchangeBuffers(C.Structure):
    """rfim_exchange_buffers: caller-owned device buffers of the allocation-free exchange step."""
    _fields_ = [("L", C.c_int32), ("R", C.c_int32), ("J", C.c_float), ("h", C.c_float),
                ("field_kind", C.c_int32), ("seed", C.c_uint32), ("realization", C.c_uint32),
                ("stage", C.c_uint32), ("spins", C.c_void_p), ("field", C.c_void_p),
                ("beta", C.c_void_p), ("t2r", C.c_void_p), ("r2t", C.c_void_p), ("att", C.c_void_p),
                ("acc", C.c_void_p), ("obs", C.c_void_p), ("n_meas", C.c_void_p), ("E", C.c_void_p),
                ("M", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_uint64), ("max_slots", C.c_int32),
                ("intervals_per_launch", C.c_int32), ("measure_xi", C.c_int32),
                ("batch_shapes", C.c_char_p)]


class ServerInfo(C.Structure):
    _fields_ = [("queued", C.c_int64), ("resident", C.c_int64), ("completed", C.c_int64),
                ("graph_launches", C.c_int64), ("busy_s", C.c_double), ("attempts", C.c_double),
                ("grid", C.c_int32), ("intervals_per_launch", C.c_int32), ("batch_shapes", C.c_char * 64)]


class ServerTuneConfig(C.Structure):
    _fields_ = [("n", C.c_int32), ("L", C.c_void_p), ("R", C.c_void_p), ("field_kind", C.c_int32),
                ("exchange_every", C.c_int32), ("sweeps", C.c_int64), ("mem_budget_bytes", C.c_uint64)]


def debug_flavour() -> bool:
    """RFIM_LIBRARY=debug selects the bounds-checked build librfim_debug.so (same C ABI)."""
    return os.environ.get("RFIM_LIBRARY", "") == "debug"


def lib_path() -> str:
    return _build.lib_path(debug_flavour())


def load():
    """Loads librfim.so (librfim_debug.so with RFIM_LIBRARY=debug), building it first if it is
    missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(debug=debug_flavour())
            if not os.path.exists(path):
                raise RuntimeError(f"{os.path.basename(path)} is missing and could not be built")
            L = C.CDLL(path)
            P, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
            L.rfim_create.argtypes = [C.POINTER(Config), C.POINTER(C.c_void_p)]
            L.rfim_destroy.argtypes = [P]
            L.rfim_sweep.argtypes = [P, i64]
            L.rfim_exchange.argtypes = [P, i64]
            L.rfim_run.argtypes = [P, i64, i32, i64]
            L.rfim_adapt_temps.argtypes = [P, i32, i64, i32, i32, P, i32, P, P]
            L.rfim_observables.argtypes = [P, C.POINTER(Obs)]
            L.rfim_get_state.argtypes = [P, P, P, P, P, P]
            L.rfim_set_state.argtypes = [P, P, P, i64, i64]
            L.rfim_get_field.argtypes = [P, P]
            L.rfim_last_error.argtypes = [P]
            L.rfim_last_error.restype = C.c_char_p
            L.rfim_launch_count.argtypes = [P]
            L.rfim_launch_count.restype = i64
            L.rfim_selftest_bits.argtypes = [i32, u32]
            L.rfim_server_create.argtypes = [C.POINTER(ServerConfig), C.POINTER(C.c_void_p)]
            L.rfim_server_submit.argtypes = [P, C.POINTER(Config), i64, i32, i64, C.POINTER(C.c_uint64)]
            L.rfim_server_poll.argtypes = [P, C.c_uint64, C.POINTER(Obs), C.POINTER(C.c_double)]
            L.rfim_server_stats.argtypes = [P, C.POINTER(ServerInfo)]
            L.rfim_server_destroy.argtypes = [P]
            L.rfim_server_last_error.argtypes = [P]
            L.rfim_server_last_error.restype = C.c_char_p
            L.rfim_exchange_noalloc.argtypes = [C.POINTER(ExchangeBuffers), u32, i64, P]
            L.rfim_selftest_grid.argtypes = [i32, i32, i32]
            L.rfim_selftest_wait.argtypes = [i32, i32]
            L.rfim_debug_build.argtypes = []
            L.rfim_selftest_debug.argtypes = []
            L.rfim_set_measure_xi.argtypes = [P, i32]
            L.rfim_set_multihit.argtypes = [P, i32, i32]
            L.rfim_thermal.argtypes = [C.POINTER(Obs), i32, P]
            L.rfim_disorder_average.argtypes = [P, i32, i32, P]
            L.rfim_tune.argtypes = [i32, i32, i32, C.c_char_p, i32, C.POINTER(C.c_double)]
            L.rfim_server_tune.argtypes = [C.POINTER(ServerTuneConfig), C.c_char_p, i32, C.POINTER(i32),
                                           C.POINTER(C.c_double)]
            L.rfim_get_plan.argtypes = [P, C.c_char_p, i32]
            L.rfim_profile.argtypes = [P, C.c_int]
            L.rfim_profile_read.argtypes = [P, P, P, P, P]
            for name in ("rfim_create", "rfim_destroy", "rfim_sweep", "rfim_exchange", "rfim_run",
                         "rfim_adapt_temps", "rfim_observables", "rfim_get_state", "rfim_set_state",
                         "rfim_get_field", "rfim_selftest_bits", "rfim_profile",
                         "rfim_profile_read", "rfim_server_create", "rfim_server_submit",
                         "rfim_server_poll", "rfim_server_stats", "rfim_server_destroy",
                         "rfim_exchange_noalloc", "rfim_tune", "rfim_selftest_grid", "rfim_selftest_wait",
                         "rfim_set_measure_xi", "rfim_set_multihit", "rfim_thermal",
                         "rfim_disorder_average", "rfim_server_tune", "rfim_debug_build",
                         "rfim_selftest_debug", "rfim_get_plan"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _current_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def exchange_noalloc(buffers: ExchangeBuffers, j: int, measure_from: int, stream=None) -> None:
    """rfim_exchange_noalloc on caller-owned device buffers (no allocation by the library)."""
    lib = load()
    st = _current_stream() if stream is None else C.c_void_p(stream)
    rc = lib.rfim_exchange_noalloc(C.byref(buffers), j, measure_from, st)
    if rc != OK:
        raise RfimError(rc, lib.rfim_last_error(None).decode())


def tune(L: int, R: int, field_kind: int = FIELD_GAUSSIAN):
    """Runs the launch-shape tuner; returns ("S,G,GT,threads", attempts/ns of the best shape)."""
    lib = load()
    buf = C.create_string_buffer(64)
    rate = C.c_double()
    rc = lib.rfim_tune(L, R, field_kind, buf, 64, C.byref(rate))
    if rc != OK:
        raise RfimError(rc, lib.rfim_last_error(None).decode())
    return buf.value.decode(), rate.value


def server_tune(mix, field_kind: int = FIELD_GAUSSIAN, sweeps: int = 200, exchange_every: int = 10,
                mem_budget_bytes: int = 4 << 30):
    """Runs the batched-kernel tuner (rfim_server_tune) on an expected mix of (L, R) pairs; returns
    {"batch_shapes": "L:G:GT,...", "intervals_per_launch": K, "attempts_per_ns": rate}.  Servers
    created later with the defaults use the result."""
    lib = load()
    Ls = np.ascontiguousarray([m[0] for m in mix], dtype=np.int32)
    Rs = np.ascontiguousarray([m[1] for m in mix], dtype=np.int32)
    cfg = ServerTuneConfig(len(Ls), Ls.ctypes.data, Rs.ctypes.data, field_kind, exchange_every, sweeps,
                           mem_budget_bytes)
    buf = C.create_string_buffer(64)
    k = C.c_int32()
    rate = C.c_double()
    rc = lib.rfim_server_tune(C.byref(cfg), buf, 64, C.byref(k), C.byref(rate))
    if rc != OK:
        raise RfimError(rc, lib.rfim_server_last_error(None).decode())
    return {"batch_shapes": buf.value.decode(), "intervals_per_launch": k.value, "attempts_per_ns": rate.value}


def debug_build() -> bool:
    """True when the loaded library is the bounds-checked flavour."""
    return bool(load().rfim_debug_build())


def selftest_debug() -> int:
    """rfim_selftest_debug: OK when a deliberately out-of-range checked index was caught."""
    return load().rfim_selftest_debug()


def selftest_grid(L: int, R: int, P: int) -> int:
    return load().rfim_selftest_grid(L, R, P)


def selftest_bits(L: int, seed: int = 1) -> int:
    return load().rfim_selftest_bits(L, seed)


THERMAL_COLUMNS = ("e", "C", "absm", "m2", "m4", "F", "xi")
DISORDER_COLUMNS = ("e", "C", "absm", "xi", "g")


def thermal(obs: dict, N: int) -> np.ndarray:
    """rfim_thermal on an observables dict (Realization.observables or a served result)."""
    R = len(obs["T"])
    o = Obs()
    keep = {k: np.ascontiguousarray(obs[k], dtype=np.float64) for k in ("T", "e", "e2", "absm", "m2", "m4")}
    for k, a in keep.items():
        setattr(o, k, a.ctypes.data)
    F = obs.get("F")
    Fa = np.ascontiguousarray(F, dtype=np.float64) if F is not None else None
    o.F = Fa.ctypes.data if Fa is not None else None
    o.R, o.n_meas = R, int(obs["n_meas"])
    out = np.zeros((R, 7), dtype=np.float64)
    rc = load().rfim_thermal(C.byref(o), N, out.ctypes.data)
    if rc != OK:
        raise RfimError(rc, "rfim_thermal")
    return out


def disorder_average(thermals) -> np.ndarray:
    """rfim_disorder_average over per-realization thermal arrays sharing one temperature set."""
    t = np.ascontiguousarray(np.stack([np.asarray(a, dtype=np.float64) for a in thermals]))
    n, R = t.shape[0], t.shape[1]
    out = np.zeros((R, 5), dtype=np.float64)
    rc = load().rfim_disorder_average(t.ctypes.data, n, R, out.ctypes.data)
    if rc != OK:
        raise RfimError(rc, "rfim_disorder_average")
    return out


def selftest_wait(spin_limit: int, set_flag: bool) -> int:
    """Status of one bounded device wait on a flag that is unset (expires) or set."""
    return load().rfim_selftest_wait(spin_limit, 1 if set_flag else 0)


class Realization:
    """One disorder realization with R temperature replicas on the current CUDA device."""

    def __init__(self, L, temps, *, R_capacity=None, J=1.0, h=1.0, field_kind=FIELD_GAUSSIAN,
                 field=None, field_seed=1, seed=42, realization=0, layout=LAYOUT_BITPACK,
                 stream=None):
        self._lib = load()
        self._h = None
        temps = np.ascontiguousarray(temps, dtype=np.float64)
        self._field = None if field is None else np.ascontiguousarray(field, dtype=np.float32)
        cfg = Config()
        cfg.L, cfg.R = L, len(temps)
        cfg.R_capacity = len(temps) if R_capacity is None else int(R_capacity)
        cfg.J, cfg.h, cfg.field_kind = J, h, field_kind
        cfg.field = None if self._field is None else self._field.ctypes.data
        cfg.field_seed, cfg.seed, cfg.realization = field_seed, seed, realization
        cfg.temps = temps.ctypes.data
        cfg.layout = layout
        cfg.stream = (_current_stream() if stream is None else C.c_void_p(stream)).value
        out = C.c_void_p()
        rc = self._lib.rfim_create(C.byref(cfg), C.byref(out))
        if rc != OK:
            raise RfimError(rc, self._lib.rfim_last_error(None).decode())
        self._h = out
        self.L, self.N, self.R_capacity = L, L ** 3, cfg.R_capacity
        self._R = cfg.R

    def _check(self, rc):
        if rc != OK:
            raise RfimError(rc, self._lib.rfim_last_error(self._h).decode())

    def close(self):
        if self._h:
            self._lib.rfim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def R(self):
        return self._R

    def sweep(self, n=1):
        self._check(self._lib.rfim_sweep(self._h, n))

    def exchange(self, measure_from=0):
        self._check(self._lib.rfim_exchange(self._h, measure_from))

    def run(self, n_sweeps, exchange_every, measure_from=0):
        self._check(self._lib.rfim_run(self._h, n_sweeps, exchange_every, measure_from))

    def adapt_temps(self, n_trials, sweeps_per_trial, exchange_every, inserts, return_rates=False):
        T = np.zeros(self.R_capacity, dtype=np.float64)
        R = C.c_int32()
        rates = np.zeros((max(n_trials, 1), self.R_capacity), dtype=np.float64)
        self._check(self._lib.rfim_adapt_temps(self._h, n_trials, sweeps_per_trial, exchange_every,
                                               inserts, _ptr(T), self.R_capacity, C.byref(R),
                                               _ptr(rates)))
        self._R = R.value
        return (T[:self._R], rates[:n_trials]) if return_rates else T[:self._R]

    def observables(self):
        R = self._R
        arrs = {k: np.zeros(R, dtype=np.float64) for k in ("T", "e", "e2", "absm", "m2", "m4", "F")}
        att = np.zeros(max(R - 1, 1), dtype=np.uint64)
        acc = np.zeros(max(R - 1, 1), dtype=np.uint64)
        o = Obs()
        for k, a in arrs.items():
            setattr(o, k, a.ctypes.data)
        o.att, o.acc = att.ctypes.data, acc.ctypes.data
        self._check(self._lib.rfim_observables(self._h, C.byref(o)))
        arrs["att"], arrs["acc"] = att[:R - 1], acc[:R - 1]
        arrs["n_meas"] = int(o.n_meas)
        arrs["sums"] = np.stack([arrs[k] for k in ("e", "e2", "absm", "m2", "m4")], axis=1)
        return arrs

    def set_measure_xi(self, on=True):
        """Enables the structure-factor measurement behind the correlation length (Sec. 7)."""
        self._check(self._lib.rfim_set_measure_xi(self._h, 1 if on else 0))

    def set_multihit(self, mh, tile=8):
        """Multi-hit double 3D checkerboard (Sec. 3.2) for the following sweeps: mh black-white
        passes per visit of the tiles of edge `tile`; mh = 0 restores the plain checkerboard."""
        self._check(self._lib.rfim_set_multihit(self._h, mh, tile))

    def thermal(self):
        """Per-temperature thermal averages [R][7] (THERMAL_COLUMNS) from the accumulators."""
        return thermal(self.observables(), self.N)

    def get_state(self, spins=True, t2r=True, energies=False):
        R, N = self._R, self.N
        s = np.zeros((R, N), dtype=np.int8) if spins else None
        p = np.zeros(R, dtype=np.int32) if t2r else None
        E = np.zeros(R, dtype=np.float64) if energies else None
        sw, xs = C.c_int64(), C.c_int64()
        self._check(self._lib.rfim_get_state(self._h, _ptr(s), _ptr(p), _ptr(E), C.byref(sw),
                                             C.byref(xs)))
        return {"spins": s, "t2r": p, "E": E, "sweep": sw.value, "xstep": xs.value}

    def set_state(self, spins=None, t2r=None, sweep=0, xstep=0):
        s = None if spins is None else np.ascontiguousarray(spins, dtype=np.int8)
        p = None if t2r is None else np.ascontiguousarray(t2r, dtype=np.int32)
        self._check(self._lib.rfim_set_state(self._h, _ptr(s), _ptr(p), sweep, xstep))

    def field(self):
        out = np.zeros(self.N, dtype=np.float32)
        self._check(self._lib.rfim_get_field(self._h, _ptr(out)))
        return out

    def plan(self) -> str:
        """Launch shape of the sweep kernel ("S,G,GT,threads[,4][,int8]"; "" for the int8 kernels)."""
        buf = C.create_string_buffer(64)
        self._check(self._lib.rfim_get_plan(self._h, buf, 64))
        return buf.value.decode()

    def profile(self, enable=True):
        self._check(self._lib.rfim_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        sm, sl = C.c_double(), C.c_int64()
        em, el = C.c_double(), C.c_int64()
        self._check(self._lib.rfim_profile_read(self._h, C.byref(sm), C.byref(sl), C.byref(em),
                                                C.byref(el)))
        return {"sweep_ms": sm.value, "sweep_launches": sl.value, "exchange_ms": em.value,
                "exchange_launches": el.value}

    @property
    def launch_count(self):
        return int(self._lib.rfim_launch_count(self._h))


class Server:
    """Continuous-batching server of independent realizations (include/rfim.h, serving section)."""

    def __init__(self, mem_budget_bytes=4 << 30, max_slots=256, intervals_per_launch=4, measure_xi=False,
                 batch_shapes=None):
        """intervals_per_launch = 0 and batch_shapes = None take the last server_tune result of this
        process (else the built-in settings); batch_shapes is "L:G:GT,..." to fix them."""
        self._lib = load()
        self._h = None
        self._shapes = None if batch_shapes is None else batch_shapes.encode()
        cfg = ServerConfig(mem_budget_bytes, max_slots, intervals_per_launch, 1 if measure_xi else 0, self._shapes)
        out = C.c_void_p()
        rc = self._lib.rfim_server_create(C.byref(cfg), C.byref(out))
        if rc != OK:
            raise RfimError(rc, self._lib.rfim_server_last_error(None).decode())
        self._h = out
        self._R = {}

    def close(self):
        if self._h:
            self._lib.rfim_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _err(self, rc):
        return RfimError(rc, self._lib.rfim_server_last_error(self._h).decode())

    def submit(self, L, temps, n_sweeps, exchange_every, measure_from=0, *, J=1.0, h=1.0,
               field_kind=FIELD_GAUSSIAN, field=None, field_seed=1, seed=42, realization=0):
        temps = np.ascontiguousarray(temps, dtype=np.float64)
        fld = None if field is None else np.ascontiguousarray(field, dtype=np.float32)
        cfg = Config()
        cfg.L, cfg.R, cfg.R_capacity = L, len(temps), len(temps)
        cfg.J, cfg.h, cfg.field_kind = J, h, field_kind
        cfg.field = None if fld is None else fld.ctypes.data
        cfg.field_seed, cfg.seed, cfg.realization = field_seed, seed, realization
        cfg.temps = temps.ctypes.data
        cfg.layout, cfg.stream = LAYOUT_BITPACK, None
        t = C.c_uint64()
        rc = self._lib.rfim_server_submit(self._h, C.byref(cfg), n_sweeps, exchange_every,
                                          measure_from, C.byref(t))
        if rc != OK:
            raise self._err(rc)
        self._R[t.value] = len(temps)
        return t.value

    def poll(self, ticket):
        """None while queued or running; the observables dict (plus latency_s) once finished."""
        R = self._R.get(ticket, 2)
        arrs = {k: np.zeros(R, dtype=np.float64) for k in ("T", "e", "e2", "absm", "m2", "m4", "F")}
        att = np.zeros(max(R - 1, 1), dtype=np.uint64)
        acc = np.zeros(max(R - 1, 1), dtype=np.uint64)
        o = Obs()
        for k, a in arrs.items():
            setattr(o, k, a.ctypes.data)
        o.att, o.acc = att.ctypes.data, acc.ctypes.data
        lat = C.c_double()
        rc = self._lib.rfim_server_poll(self._h, ticket, C.byref(o), C.byref(lat))
        if rc == EBUSY:
            return None
        if rc != OK:
            self._R.pop(ticket, None)
            raise self._err(rc)
        self._R.pop(ticket, None)
        arrs["att"], arrs["acc"] = att[:R - 1], acc[:R - 1]
        arrs["n_meas"] = int(o.n_meas)
        arrs["sums"] = np.stack([arrs[k] for k in ("e", "e2", "absm", "m2", "m4")], axis=1)
        arrs["latency_s"] = lat.value
        return arrs

    def wait(self, ticket, timeout_s=600.0, interval_s=0.0005):
        import time
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError(f"ticket {ticket} not finished after {timeout_s} s")
            time.sleep(interval_s)

    def stats(self):
        info = ServerInfo()
        rc = self._lib.rfim_server_stats(self._h, C.byref(info))
        if rc != OK:
            raise self._err(rc)
        out = {k: getattr(info, k) for k, _ in ServerInfo._fields_}
        out["batch_shapes"] = info.batch_shapes.decode()
        return out

"""Benchmark: spin-flip attempts/ns of the Exchange Monte Carlo hot path at L = 64.

Workload (one step): one disorder realization, L = 64 periodic lattice (262144 sites), Gaussian
field h_i ~ N(0,1) with h = 1, J = 1, R = 128 temperatures geometric in [1, 5], 10^4 checkerboard
sweeps with an exchange step every 10 sweeps (1000 exchange steps with energy reduction, swap
decisions, temperature permutation and per-temperature measurement) -- every step of the hot path
runs on the GPU.  Steps continue the same Markov chain.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--layout bitpack|int8]

The JSON line also carries the other spin layout of the same workload (int8 by default), a
serving measurement (continuous batching vs per-realization launches on a C5-shaped stream of
128 realizations x 1000 sweeps, batched kernel tuned first) and the smaller configurations C1-C3
(C3 with its temperature adaptation and 10^5 production sweeps).

Under torchrun each rank runs its own realization (realization id = rank; weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L, R, T_MIN, T_MAX, H, J = 64, 128, 1.0, 5.0, 1.0, 1.0
SWEEPS, EX = 10_000, 10
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Philox4x32-10 needs 20 32x32->64 multiplies per block of 4 attempts; the IMAD.WIDE pipe issues
# 32 of them per SM per clock on GB300 (measured), which bounds the sweep at 6.4 attempts/clk/SM.
MULWIDE_PER_CLK_SM = 32.0
MULWIDE_PER_ATTEMPT = 5.0
# dram__bytes_read.sum + dram__bytes_write.sum of a launch of one exchange interval (3.36e8
# attempts) of the dominant kernel of each plan and layout, from one ncu capture of the current
# kernel version; None when the kernel changed since the capture.  (The grid-wide plan runs up to
# 64 intervals per launch in the timed steps; per interval it moves no more than this.)
SWEEP_TRAFFIC_BYTES = {"k_sweeps_bits": 6.654976e6, "k_sweeps_grid": 6.723328e6,
                       "k_sweeps_bits (int8 layout staged as bits)": 36.020992e6,
                       "k_sweeps_grid (int8 layout staged as bits)": 36.098304e6}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--layout", default="bitpack", choices=["bitpack", "int8"])
    p.add_argument("--sweeps", type=int, default=SWEEPS)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--workload", default="c4", choices=["c4", "serve", "adapt", "multihit", "profile"])
    p.add_argument("--profile-case", default="c4", choices=["c4", "c4-bimodal", "c4-int8", "serve", "multihit"])
    p.add_argument("--no-int8", action="store_true", help="skip the int8-layout sub-measurement")
    p.add_argument("--no-serve", action="store_true", help="skip the serving sub-measurement")
    p.add_argument("--no-configs", action="store_true", help="skip the C1-C3 sub-measurement")
    p.add_argument("--serve-realizations", type=int, default=128)
    p.add_argument("--adapt-L", type=int, default=32)
    p.add_argument("--realizations", type=int, default=128)
    p.add_argument("--serve-sweeps", type=int, default=2000)
    p.add_argument("--int-rates", action="store_true")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def temps():
    from paper_1508_06268_gb300 import inputs
    return inputs.geometric_temps(T_MIN, T_MAX, R)


def shard_for_rank(rank):
    """Realization-level sharding (weak scaling, no collective on the data path): rank r runs its
    own disorder realization r with field seed 1 + r."""
    return {"realization": rank, "field_seed": 1 + rank}


def max_over_ranks(value, dist, device):
    """The timed region's duration as the maximum over ranks (identity without a process group)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, max_ms):
    """Whole-job throughput: units processed by all ranks / slowest rank's time (units per ns)."""
    return units_per_rank * world / (max_ms * 1e6)


def _oracle_share(job):
    """One host process of the all-cores baseline: the oracle on a subset of the replicas."""
    import oracle
    temps_sub, sweeps = job
    o = oracle.Oracle(L, temps_sub, J=J, h=H, field_kind=oracle.FIELD_GAUSSIAN, field_seed=1, seed=42)
    t0 = time.perf_counter()
    o.run(sweeps, EX, 0)
    return L ** 3 * len(temps_sub) * sweeps, time.perf_counter() - t0


def cpu_baseline(budget_s=12.0):
    """The oracle as it stands (single thread) on a bounded sample of the same workload; beside it
    the same oracle in one process per host core, each on an equal share of the replicas."""
    import multiprocessing as mp
    import oracle
    T = temps()
    o = oracle.Oracle(L, T, J=J, h=H, field_kind=oracle.FIELD_GAUSSIAN, field_seed=1, seed=42)
    t0 = time.perf_counter()
    o.run(1, 0, 0)
    one = time.perf_counter() - t0
    n = max(1, min(30, int(budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    o.run(n, EX, 0)
    dt = time.perf_counter() - t0
    att = L ** 3 * R * n
    out = {"value": att / (dt * 1e9), "unit": "attempts/ns", "cores": 1, "kind": "oracle",
           "sample": f"L=64 Gaussian R=128, {n} sweeps (exchange every {EX}) of the 10^4-sweep workload, "
                     f"{dt:.1f} s single-threaded"}
    cores = max(1, min(os.cpu_count() or 1, R // 2))
    if cores > 1:
        per = R // cores
        sweeps = max(1, int(n * R / per))  # each process about as long as the single-core sample
        jobs = [(T[i * per:(i + 1) * per], sweeps) for i in range(cores)]
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(cores) as pool:  # spawn: CUDA is already initialised
            done = pool.map(_oracle_share, jobs)
        wall = time.perf_counter() - t0
        out["all_cores"] = {"value": sum(a for a, _ in done) / (wall * 1e9), "unit": "attempts/ns", "cores": cores,
                            "sample": f"{cores} processes x {per} replicas x {sweeps} sweeps, {wall:.1f} s wall "
                                      "(process start included)"}
    return out


def c4_workload(args):
    """The benchmarked workload, named the same way by both arms."""
    return (f"C4: L=64 (262144 sites) Gaussian h=1, J=1, R=128 geometric [1,5], {args.sweeps} sweeps/step, "
            f"exchange every {EX}")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    T = temps()
    o = oracle.Oracle(L, T, J=J, h=H, field_kind=oracle.FIELD_GAUSSIAN, field_seed=1, seed=42)
    per_step = 2
    for _ in range(args.warmup):
        o.run(per_step, EX, 0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.run(per_step, EX, 0)
    dt = time.perf_counter() - t0
    att = L ** 3 * R * per_step * args.steps
    value = att / (dt * 1e9)
    line = {
        "impl": "reference", "metric": "spin-flip attempts/ns at L=64", "value": value,
        "unit": "attempts/ns", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64/f32 (oracle)", "data": "synthetic",
        "config": {"workload": c4_workload(args), "layout": args.layout,
                   "sample": f"each step {per_step} of its sweeps, on the host cores"},
        "cpu_baseline": {"value": value, "unit": "attempts/ns", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} sweeps of all 128 replicas per step"},
        "e2e": {"value": value, "unit": "attempts/ns", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


SERVE_R = {8: 16, 16: 32, 32: 64, 64: 128}


def serve_requests(n, sweeps):
    """C5-shaped request stream: L uniform in {8,16,32,64} (seed 7), R matched to L, Gaussian h=1,
    Poisson arrival gaps of unit mean (seed 2024; scaled by the caller)."""
    rng = np.random.default_rng(7)
    Ls = rng.choice([8, 16, 32, 64], size=n)
    gaps = np.random.default_rng(2024).exponential(1.0, size=n)
    return [(int(L), SERVE_R[int(L)], i) for i, L in enumerate(Ls)], gaps


def serve_measure(n_real, sweeps, tune=True, with_xi=True):
    """Continuous batching vs plain per-realization launches on the same C5-shaped request stream
    (Poisson arrivals at 0.8 x the batched server's closed-loop capacity).  With `tune`, the
    batched kernel's shapes and intervals per replay come from rfim_server_tune on this mix."""
    import torch
    import paper_1508_06268_gb300 as rf
    from paper_1508_06268_gb300 import inputs
    reqs, gaps = serve_requests(n_real, sweeps)
    ex, sw = EX, sweeps
    mf = sw // ex // 2
    temps = {L: inputs.geometric_temps(T_MIN, T_MAX, R_) for L, R_ in SERVE_R.items()}
    work = sum(L ** 3 * R_ * sw for L, R_, _ in reqs)
    tuned = None
    if tune:
        t0 = time.perf_counter()
        tuned = rf.server_tune(sorted(SERVE_R.items()), field_kind=rf.FIELD_GAUSSIAN, sweeps=200, exchange_every=ex)
        tuned["seconds"] = round(time.perf_counter() - t0, 2)

    def batched(arrivals, xi=False):
        # intervals_per_launch 0 and no explicit shapes: the tuned settings (built-in ones untuned)
        srv = rf.Server(mem_budget_bytes=4 << 30, max_slots=256, intervals_per_launch=0 if tune else 4,
                        measure_xi=xi)
        t0 = time.perf_counter()
        pend, lat, i = {}, [], 0
        while len(lat) < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and arrivals[i] <= now:
                L, R_, k = reqs[i]
                pend[srv.submit(L, temps[L], sw, ex, mf, field_kind=rf.FIELD_GAUSSIAN, field_seed=1 + k,
                                realization=k)] = arrivals[i]
                i += 1
            for t in list(pend):
                r = srv.poll(t)
                if r is not None:
                    lat.append(r["latency_s"])
                    del pend[t]
            time.sleep(0.0002)
        span = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return np.array(lat), span, st

    def sequential(arrivals):
        t0 = time.perf_counter()
        lat = []
        for (L, R_, k), a in zip(reqs, arrivals):
            while time.perf_counter() - t0 < a:
                time.sleep(0.0002)
            g = rf.Realization(L, temps[L], field_kind=rf.FIELD_GAUSSIAN, field_seed=1 + k, realization=k,
                               layout=rf.LAYOUT_BITPACK)
            g.run(sw, ex, mf)
            g.observables()
            g.close()
            lat.append(time.perf_counter() - t0 - a)
        return np.array(lat), time.perf_counter() - t0

    # warm-up (module load, graph capture), then the closed-loop capacity of the batched server
    batched(np.zeros(len(reqs)))
    _, span_closed, _ = batched(np.zeros(len(reqs)))
    span_closed_xi = None
    if with_xi:  # the same with the structure factor of the correlation length in the batched kernel
        _, span_closed_xi, _ = batched(np.zeros(len(reqs)), xi=True)
    rate = 0.8 * len(reqs) / span_closed  # realizations / s offered to both servers
    arrivals = np.cumsum(gaps) / rate
    arrivals -= arrivals[0]
    lat_b, span_b, st = batched(arrivals)
    lat_s, span_s = sequential(arrivals)
    torch.cuda.synchronize()
    return {
        "metric": "served realizations: p50/p99 latency and spin-flip attempts/ns (batched vs per-realization)",
        "workload": "C5-shaped: Gaussian h=1, L uniform in {8,16,32,64}, R=16/32/64/128",
        "realizations": len(reqs), "sweeps_each": sw, "exchange_every": ex,
        "offered_rate_per_s": rate, "arrivals": "Poisson (seed 2024), 0.8 x closed-loop batched capacity",
        "tuned": tuned,
        "batched": {"p50_s": float(np.percentile(lat_b, 50)), "p99_s": float(np.percentile(lat_b, 99)),
                    "attempts_per_ns": work / (span_b * 1e9), "makespan_s": span_b,
                    "closed_loop_attempts_per_ns": work / (span_closed * 1e9),
                    "closed_loop_xi_attempts_per_ns": None if span_closed_xi is None
                    else work / (span_closed_xi * 1e9),
                    "graph_launches": st["graph_launches"], "grid": st["grid"],
                    "batch_shapes": st["batch_shapes"], "intervals_per_launch": st["intervals_per_launch"]},
        "per_realization": {"p50_s": float(np.percentile(lat_s, 50)), "p99_s": float(np.percentile(lat_s, 99)),
                            "attempts_per_ns": work / (span_s * 1e9), "makespan_s": span_s},
    }


def run_serve(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    print(json.dumps(serve_measure(args.realizations, args.serve_sweeps)), flush=True)


def run_profile(args):
    """Small fixed workloads for ncu captures of one kernel (commands in profiles/): the C4 shape
    (L = 64, R = 128, four exchange intervals of 10 sweeps; Gaussian, bimodal or int8 layout), the
    batched serving kernel on 16 C5-shaped Gaussian realizations of 400 sweeps submitted at once,
    or multi-hit sweeps (mh = 100, tiles 8^3, four launches of one sweep)."""
    import torch
    import paper_1508_06268_gb300 as rf
    from paper_1508_06268_gb300 import inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    case = args.profile_case
    if case == "serve":
        with rf.Server(mem_budget_bytes=2 << 30, max_slots=64, intervals_per_launch=4) as srv:
            tickets = [srv.submit(L_, inputs.geometric_temps(T_MIN, T_MAX, R_), 400, EX, 20,
                                  field_kind=rf.FIELD_GAUSSIAN, field_seed=1 + k, realization=k)
                       for k, (L_, R_) in enumerate(sorted(SERVE_R.items()) * 4)]
            for t in tickets:
                srv.wait(t)
        print("ok", len(tickets))
    elif case == "multihit":
        g = rf.Realization(L, inputs.geometric_temps(T_MIN, T_MAX, R), field_kind=rf.FIELD_GAUSSIAN)
        g.set_multihit(100, 8)
        g.run(4, 1, 0)
        print("ok", g.get_state(spins=False)["sweep"])
    else:
        layout = rf.LAYOUT_INT8 if case == "c4-int8" else rf.LAYOUT_BITPACK
        kind = rf.FIELD_BIMODAL if case == "c4-bimodal" else rf.FIELD_GAUSSIAN
        g = rf.Realization(L, inputs.geometric_temps(T_MIN, T_MAX, R), field_kind=kind, layout=layout)
        for _ in range(4):  # one exchange interval per call, so one per launch in every plan
            g.run(EX, EX, 0)
        print("ok", g.get_state(spins=False)["sweep"])
    torch.cuda.synchronize()


# Sec. 4 and the comparison of adaptive and homogeneous temperature sets (Table 1, the exchange-rate
# figure): per L, the trial runs and insertions the paper used, 2000 exchange steps of 10 sweeps per
# run, and equally spaced (homogeneous) sparse and dense sets on [T_MIN, T_MAX].  The text does not
# print the sparse and dense replica counts (they are in the figure labels), so they are chosen
# here: the adaptive set starts from the sparse one, and the dense one has more replicas than the
# adaptive set ends with.
ADAPT_CASES = {32: {"trials": 10, "inserts": 2, "sparse": 40, "dense": 80},
               64: {"trials": 32, "inserts": 3, "sparse": 64, "dense": 192}}


def run_adapt(args):
    """Adaptive vs sparse and dense homogeneous temperature sets on this GPU: wall time of the
    production runs of every realization and of the adaptation trials (run once, on realization 0,
    the set then shared), and the spread of the adjacent exchange rates."""
    import torch
    import paper_1508_06268_gb300 as rf
    from paper_1508_06268_gb300 import inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    Lx = args.adapt_L
    case = ADAPT_CASES[Lx]
    n_real = max(1, args.realizations if args.realizations != 128 else 4)
    steps, ex = 2000, EX
    sweeps = steps * ex

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    def rates(g):
        o = g.observables()
        att = o["att"].astype(np.float64)
        return np.where(att > 0, o["acc"] / np.maximum(att, 1), 0.0)

    res = {k: {"s": 0.0, "rates": []} for k in ("sparse-sim", "dense-sim", "adapt-trials", "adapt-sim")}

    def common(k):
        return dict(field_kind=rf.FIELD_GAUSSIAN, h=H, field_seed=1 + k, realization=k, layout=rf.LAYOUT_BITPACK)

    # the adaptation runs once (trials on realization 0); every realization then uses its set
    cap = case["sparse"] + case["trials"] * case["inserts"]
    g = rf.Realization(Lx, inputs.linear_temps(T_MIN, T_MAX, case["sparse"]), R_capacity=cap, **common(0))
    adapted, dt = timed(lambda: g.adapt_temps(case["trials"], sweeps, ex, case["inserts"]))
    res["adapt-trials"]["s"] = dt
    g.close()
    for k in range(n_real):
        for name, temps in (("sparse-sim", inputs.linear_temps(T_MIN, T_MAX, case["sparse"])),
                            ("dense-sim", inputs.linear_temps(T_MIN, T_MAX, case["dense"])),
                            ("adapt-sim", adapted)):
            g = rf.Realization(Lx, temps, **common(k))
            _, dt = timed(lambda: g.run(sweeps, ex, steps // 2))
            res[name]["s"] += dt
            res[name]["rates"].append(rates(g))
            g.close()
    line = {
        "metric": "adaptive vs homogeneous temperature sets: wall seconds and adjacent exchange rates",
        "workload": f"L={Lx} Gaussian h={H}, {n_real} realizations, {steps} exchange steps x {ex} sweeps per run, "
                    f"adaptation {case['trials']} trials x {case['inserts']} insertions, T in [{T_MIN}, {T_MAX}]",
        "replicas": {"sparse": case["sparse"], "dense": case["dense"], "adaptive_final": len(adapted)},
        "seconds": {k: round(v["s"], 3) for k, v in res.items()},
        "adapt_total_s": round(res["adapt-trials"]["s"] + res["adapt-sim"]["s"], 3),
        "exchange_rates": {k: {"min": float(np.mean([r.min() for r in v["rates"]])),
                               "mean": float(np.mean([r.mean() for r in v["rates"]])),
                               "max": float(np.mean([r.max() for r in v["rates"]]))}
                           for k, v in res.items() if v["rates"]},
        "paper_table1_s_2xK40_100_realizations": {"32": [670.25, 1417.04, 41.84, 1167, 1209.49],
                                                  "64": [10386.75, 26697.17, 1689.46, 19994.70, 21684.15]},
        "data": "synthetic",
    }
    print(json.dumps(line), flush=True)


def run_multihit(args):
    """Multi-hit double 3D checkerboard (Sec. 3.2; the paper's mh = 100 spin-level runs) against the
    plain checkerboard on the C4 shape: sweep-kernel time by CUDA events on the context's stream,
    every attempt counted (mh per site and sweep)."""
    import torch
    import paper_1508_06268_gb300 as rf
    from paper_1508_06268_gb300 import inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    L, R, attempts = 64, 128, 64 ** 3 * 128 * 400  # the work of 400 plain sweeps per measurement
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    rows = []
    for kind, kname in ((rf.FIELD_GAUSSIAN, "gaussian"), (rf.FIELD_BIMODAL, "bimodal")):
        for mh, tile in ((0, 0), (1, 8), (1, 32), (10, 8), (100, 8), (100, 16), (100, 32)):
            sweeps = 400 // max(mh, 1)
            ex = min(EX, sweeps)
            g = rf.Realization(L, inputs.geometric_temps(T_MIN, T_MAX, R), field_kind=kind,
                               layout=rf.LAYOUT_BITPACK)
            if mh:
                g.set_multihit(mh, tile)
            g.run(max(ex, sweeps // 4), ex, 0)  # warm-up
            g.profile(True)
            g.run(sweeps, ex, 0)
            p = g.profile_read()
            g.profile(False)
            g.close()
            rows.append({"field": kname, "mh": mh, "tile": tile, "sweeps": sweeps,
                         "attempts_per_ns": round(attempts / (p["sweep_ms"] * 1e6), 1)})
    clk = clocks.stop()
    sm_mhz = clk["sm_mhz"] or 2070.0
    peak = MULWIDE_PER_CLK_SM / MULWIDE_PER_ATTEMPT * props.multi_processor_count * sm_mhz * 1e-3
    for r in rows:
        r["frac"] = round(r["attempts_per_ns"] / peak, 3)
    line = {"metric": "spin-flip attempts/ns, multi-hit double checkerboard vs plain checkerboard",
            "workload": f"C4 shape: L={L}, R={R} geometric [{T_MIN}, {T_MAX}], exchange every {EX} sweeps; "
                        "mh black-white passes per tile visit, tiles of edge `tile` (mh = 0: plain)",
            "rows": rows, "peak_attempts_per_ns": round(peak, 1),
            "peak_basis": "Philox IMAD.WIDE limit at the sampled SM clock", "clocks": clk, "data": "synthetic"}
    print(json.dumps(line), flush=True)


def run_int_rates():
    """Builds and runs the GB300 issue-rate microbenchmark (the roofline's peak basis) and the
    instruction-mix ceiling of Philox plus the acceptance tests."""
    mb = os.path.join(ROOT, "paper_1508_06268_gb300", "microbench")
    csrc = os.path.join(ROOT, "paper_1508_06268_gb300", "csrc")
    for name in ("int_rates", "mix_rates"):
        exe = os.path.join(ROOT, "paper_1508_06268_gb300", "_lib", name)
        os.makedirs(os.path.dirname(exe), exist_ok=True)
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", csrc,
                        "-o", exe, os.path.join(mb, name + ".cu")], check=True)
        subprocess.run([exe], check=True)


def configs_measure(rf, torch):
    """The smaller benchmark configurations end to end on the device (bit layout, CUDA events on
    the context's stream): C1 L=8 Gaussian R=16 [1.5,5] 2000 sweeps / ex 10; C2 L=16 bimodal
    h=1.5 R=32 [1,5] 10^4 sweeps / ex 5; C3 L=32 Gaussian R0=64 [1,5] adapted by 3 trials of 2000
    sweeps (ex 10, 2 insertions each: R=70), then 10^5 production sweeps / ex 10.  Each run is
    preceded by a short warm-up run of the same shape.  Then 32 C3-sized realizations with the
    adapted set through the batched server."""
    from paper_1508_06268_gb300 import inputs
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1) * 1e-3

    out = {}
    for name, Lc, kind, h, T, sweeps, ex in (
            ("C1", 8, rf.FIELD_GAUSSIAN, 1.0, inputs.geometric_temps(1.5, 5.0, 16), 2000, 10),
            ("C2", 16, rf.FIELD_BIMODAL, 1.5, inputs.geometric_temps(1.0, 5.0, 32), 10_000, 5)):
        g = rf.Realization(Lc, T, h=h, field_kind=kind, field_seed=1, seed=42, layout=rf.LAYOUT_BITPACK)
        g.run(10 * ex, ex, 0)
        g.close()
        g = rf.Realization(Lc, T, h=h, field_kind=kind, field_seed=1, seed=42, layout=rf.LAYOUT_BITPACK)
        _, dt = timed(lambda: g.run(sweeps, ex, sweeps // ex // 2))
        g.observables()
        g.close()
        out[name] = {"attempts_per_ns": Lc ** 3 * len(T) * sweeps / (dt * 1e9), "seconds": dt,
                     "L": Lc, "R": len(T), "sweeps": sweeps}
    T0 = inputs.geometric_temps(1.0, 5.0, 64)
    w = rf.Realization(32, T0, field_kind=rf.FIELD_GAUSSIAN, field_seed=1, seed=42, layout=rf.LAYOUT_BITPACK,
                       R_capacity=70)
    w.adapt_temps(1, 100, 10, 2)
    w.run(1000, 10, 0)
    w.close()
    g = rf.Realization(32, T0, field_kind=rf.FIELD_GAUSSIAN, field_seed=1, seed=42, layout=rf.LAYOUT_BITPACK,
                       R_capacity=70)
    Ta, dt_a = timed(lambda: g.adapt_temps(3, 2000, 10, 2))
    _, dt_p = timed(lambda: g.run(100_000, 10, 5000))
    g.observables()
    g.close()
    trial_attempts = 32 ** 3 * (64 + 66 + 68) * 2000
    out["C3"] = {"attempts_per_ns": 32 ** 3 * len(Ta) * 100_000 / (dt_p * 1e9), "seconds": dt_p,
                 "adapt_seconds": dt_a, "adapt_attempts_per_ns": trial_attempts / (dt_a * 1e9),
                 "L": 32, "R": len(Ta), "sweeps": 100_000}
    # C3-sized work served: 32 realizations (fields 1..32) with the adapted set, 10^4 sweeps each,
    # submitted at once to the batched server (one realization alone cannot fill the GPU)
    n, sw = 32, 10_000
    with rf.Server(mem_budget_bytes=2 << 30, max_slots=n) as srv:
        warm = [srv.submit(32, Ta, 100, 10, 5, field_kind=rf.FIELD_GAUSSIAN, field_seed=1 + k, realization=k)
                for k in range(4)]
        for t in warm:
            srv.wait(t)
        t0 = time.perf_counter()
        tickets = [srv.submit(32, Ta, sw, 10, sw // 20, field_kind=rf.FIELD_GAUSSIAN, field_seed=1 + k,
                              realization=k) for k in range(n)]
        for t in tickets:
            srv.wait(t)
        dt_s = time.perf_counter() - t0
    out["C3_served"] = {"attempts_per_ns": 32 ** 3 * len(Ta) * sw * n / (dt_s * 1e9), "seconds": dt_s,
                        "realizations": n, "sweeps_each": sw, "L": 32, "R": len(Ta),
                        "timing": "wall clock from the first submit to the last result"}
    return out


def measure_layout(rf, torch, layout, args, T, real, field_seed, local, dist):
    """W untimed steps, then K timed steps (L2 flushed before each) of the C4 workload in one
    layout; returns the device time (max over ranks), wall time, kernel profile, launches, clocks."""
    g = rf.Realization(L, T, J=J, h=H, field_kind=rf.FIELD_GAUSSIAN, field_seed=field_seed, seed=42,
                       realization=real, layout=layout)
    stream = torch.cuda.current_stream()
    measure_from = args.sweeps // EX // 2
    for _ in range(max(args.warmup, 3)):
        g.run(args.sweeps, EX, measure_from)
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    launches0 = g.launch_count
    g.profile(True)
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    dev_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.run(args.sweeps, EX, measure_from)
        e1.record(stream)
        e1.synchronize()
        dev_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    prof = g.profile_read()
    g.profile(False)
    launches = g.launch_count - launches0
    plan = g.plan()
    g.close()
    del flush
    if dist is not None:
        dist.barrier()
    return {"dev_ms": max_over_ranks(dev_ms, dist, "cuda"), "dev_ms_local": dev_ms, "wall": wall, "prof": prof,
            "launches": launches, "clk": clk, "plan": plan}


def roofline_of(m, layout, rf, props, steps):
    """Dominant kernel of the layout against the Philox integer roof at the sampled SM clock:
    attempts of one launch group (one exchange interval of EX sweeps) / its CUDA-event time."""
    prof, clk = m["prof"], m["clk"]
    group_ms = prof["sweep_ms"] / max(prof["sweep_launches"], 1)
    achieved = L ** 3 * R * EX / (group_ms * 1e6)  # Gattempts/s
    sm_mhz = clk["sm_mhz"] or 2070.0
    peak = MULWIDE_PER_CLK_SM / MULWIDE_PER_ATTEMPT * props.multi_processor_count * sm_mhz * 1e-3
    # the int8 layout at L = 64 runs the same kernels with the lattice staged from bytes into bits;
    # the grid-wide kernel when the plan says S = 0
    kernel = "k_sweeps_grid" if m.get("plan", "").startswith("0,") else "k_sweeps_bits"
    if layout != rf.LAYOUT_BITPACK:
        kernel += " (int8 layout staged as bits)"
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gattempts/s", "frac": achieved / peak,
            "traffic": SWEEP_TRAFFIC_BYTES.get(kernel),
            "traffic_unit": "bytes per exchange interval (ncu, DRAM read+write of a one-interval launch)",
            "kernel": kernel, "plan": m.get("plan"),
            "peak_basis": f"Philox4x32-10 IMAD.WIDE limit: {MULWIDE_PER_CLK_SM:.0f}/clk/SM (measured) / "
                          f"{MULWIDE_PER_ATTEMPT:.0f} per attempt x {props.multi_processor_count} SMs x "
                          f"{sm_mhz:.0f} MHz (median sampled)",
            "sweep_kernel_share": prof["sweep_ms"] / max(m["dev_ms_local"], 1e-9),
            "exchange_ms_per_step": prof["exchange_ms"] / steps}


def main():
    args = parse()
    if args.int_rates:
        run_int_rates()
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "adapt":
        run_adapt(args)
        return
    if args.workload == "multihit":
        run_multihit(args)
        return
    if args.workload == "profile":
        run_profile(args)
        return
    import torch
    import paper_1508_06268_gb300 as rf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    layout = rf.LAYOUT_BITPACK if args.layout == "bitpack" else rf.LAYOUT_INT8
    T = temps()
    sh = shard_for_rank(rank)
    real = sh["realization"]
    props = torch.cuda.get_device_properties(local)
    m = measure_layout(rf, torch, layout, args, T, real, sh["field_seed"], local, dist)
    attempts_rank = L ** 3 * R * args.sweeps * args.steps
    value = aggregate_rate(attempts_rank, world, m["dev_ms"])
    roofline = roofline_of(m, layout, rf, props, args.steps)

    # the other spin layout of the C4 workload (the headline is the bit layout by default)
    other = None
    if not args.no_int8:
        olay = rf.LAYOUT_INT8 if layout == rf.LAYOUT_BITPACK else rf.LAYOUT_BITPACK
        mo = measure_layout(rf, torch, olay, args, T, real, sh["field_seed"], local, dist)
        other = {"layout": "int8" if olay == rf.LAYOUT_INT8 else "bitpack",
                 "value": aggregate_rate(attempts_rank, world, mo["dev_ms"]), "unit": "attempts/ns",
                 "ms_per_step": mo["dev_ms"] / args.steps, "gpu_launches": mo["launches"],
                 "roofline": roofline_of(mo, olay, rf, props, args.steps), "clocks": mo["clk"]}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(rf, torch, T, layout, args, real)
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        serving = serve_measure(args.serve_realizations, 1000, tune=True, with_xi=False)
    small = None
    if rank == 0 and world == 1 and not args.no_configs:
        small = configs_measure(rf, torch)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()
    if rank == 0:
        line = {
            "metric": "spin-flip attempts/ns at L=64", "value": value, "unit": "attempts/ns",
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": m["dev_ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32+f32", "data": "synthetic",
            "config": {"workload": c4_workload(args),
                       "layout": args.layout, "l2": "flushed (512 MB write) between timed steps",
                       "parallelism": f"realization per GPU x{world}",
                       "wall_s": m["wall"]},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": m["launches"],
            "clocks": m["clk"], "serving": serving, "configs": small,
        }
        if other is not None:  # the second layout of the C4 workload under its own name
            line[other["layout"]] = other
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(rf, torch, T, layout, args, real):
    """Same metric through the public API with host buffers: create from a pinned host field and
    temperature set (H2D), run, read the observables (D2H), destroy -- all inside the timing."""
    from paper_1508_06268_gb300 import inputs
    field = torch.from_numpy(inputs.gaussian_field(L, 1000 + real)).pin_memory()
    T_pin = torch.from_numpy(np.ascontiguousarray(T)).pin_memory()
    steps = max(1, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(steps):
        g = rf.Realization(L, T_pin.numpy(), J=J, h=H, field_kind=rf.FIELD_EXPLICIT, field=field.numpy(),
                           seed=42, realization=real, layout=layout)
        g.run(args.sweeps, EX, args.sweeps // EX // 2)
        ob = g.observables()
        d2h = sum(ob[k].nbytes for k in ("e", "e2", "absm", "m2", "m4", "att", "acc")) + 8
        g.close()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": L ** 3 * R * args.sweeps * steps / (dt * 1e9), "unit": "attempts/ns",
            "h2d_bytes_per_step": int(field.numel() * 4 + T_pin.numel() * 8), "d2h_bytes_per_step": int(d2h)}


if __name__ == "__main__":
    main()

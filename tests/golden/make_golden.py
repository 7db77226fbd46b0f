"""Writes the stored expected values of tests/golden/ by running the CPU oracle only.

c2_bimodal_L16_R32.json: the full C2 configuration (L=16 periodic lattice, bimodal field h=1.5,
R=32 temperatures geometric in [1, 5], 10^4 sweeps, exchange every 5 sweeps, measurements from
exchange step 1000 on; field seed 1, dynamics seed 42, realization 0).  Stored: final
temperature permutation, per-pair exchange attempts and acceptances, the per-temperature
measurement sums and a digest of the final spins.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1508_06268_gb300 import inputs  # noqa: E402

C2 = dict(L=16, R=32, h=1.5, t_min=1.0, t_max=5.0, sweeps=10_000, exchange_every=5, measure_from=1000,
          field_seed=1, seed=42, realization=0)


def spins_digest(s) -> str:
    return hashlib.sha256(s.astype("int8").tobytes()).hexdigest()


def main():
    c = C2
    temps = inputs.geometric_temps(c["t_min"], c["t_max"], c["R"])
    o = oracle.Oracle(c["L"], temps, h=c["h"], field_kind=oracle.FIELD_BIMODAL, field_seed=c["field_seed"],
                      seed=c["seed"], realization=c["realization"])
    o.run(c["sweeps"], c["exchange_every"], c["measure_from"])
    att, acc = o.exchange_stats()
    out = {"config": c, "source": "oracle/rfim_oracle.c via tests/golden/make_golden.py",
           "t2r": o.perm()[0].tolist(), "att": att.tolist(), "acc": acc.tolist(),
           "n_meas": o.n_meas, "obs_sums": o.observables().tolist(), "spins_sha256": spins_digest(o.spins())}
    with open(os.path.join(HERE, "c2_bimodal_L16_R32.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

"""Bounds-checked build (librfim_debug.so, compiled with -DRFIM_DEBUG): the small parity cases
run with every device check compiled in -- shared-memory lattice indices, decision-table slots,
cluster peer ranks, the grid-wide partition, the no-alloc scratch slots -- and no check fires,
while the results still equal the oracle bit for bit (bimodal field).  The check mechanism
itself is exercised by a self-test whose checked index is out of range on purpose: the check
records it and the kernel ends normally.

The cases run in a child process with RFIM_LIBRARY=debug, so this process keeps the release
library; the child builds the debug flavour if it is missing.
"""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
import numpy as np
sys.path.insert(0, os.environ["RFIM_ROOT"])
import torch
import oracle
import paper_1508_06268_gb300 as rf
from paper_1508_06268_gb300 import inputs

torch.cuda.set_device(0)
assert rf.debug_build(), "the debug flavour was not loaded"
assert rf.selftest_debug() == rf.OK, "an out-of-range checked index was not caught"


def pair(L, R, layout, plan=None, **kw):
    temps = inputs.geometric_temps(1.0, 5.0, R)
    if plan:
        os.environ["RFIM_BITS_PLAN"] = plan
    g = rf.Realization(L, temps, h=1.5, field_kind=rf.FIELD_BIMODAL, field_seed=3, seed=42, layout=layout, **kw)
    os.environ.pop("RFIM_BITS_PLAN", None)
    o = oracle.Oracle(L, temps, h=1.5, field_kind=oracle.FIELD_BIMODAL, field_seed=3, seed=42)
    return g, o


def same(g, o, what):
    st = g.get_state()  # raises RfimError(EBOUNDS) if a check fired
    assert np.array_equal(st["spins"], o.spins()), what
    assert np.array_equal(st["t2r"], o.perm()[0]), what
    assert np.array_equal(g.observables()["sums"], o.observables()), what


cases = [(8, 16, rf.LAYOUT_BITPACK, None), (16, 32, rf.LAYOUT_BITPACK, None), (8, 16, rf.LAYOUT_INT8, None),
         (16, 8, rf.LAYOUT_INT8, None), (32, 6, rf.LAYOUT_BITPACK, None), (64, 6, rf.LAYOUT_BITPACK, "4,4,4,512"),
         (64, 6, rf.LAYOUT_BITPACK, "0,4,4,512"), (64, 13, rf.LAYOUT_BITPACK, "0,4,1,512")]
for L, R, layout, plan in cases:
    g, o = pair(L, R, layout, plan)
    g.run(12, 3, 1)
    o.run(12, 3, 1)
    same(g, o, f"L={L} R={R} layout={layout} plan={plan}")
    g.close()

# served realizations (batched kernel), ragged replica groups
with rf.Server(mem_budget_bytes=64 << 20, max_slots=4, intervals_per_launch=2) as srv:
    mix = [(8, 5, 0), (16, 8, 1), (32, 9, 2)]
    tickets = [srv.submit(L, inputs.geometric_temps(1.0, 5.0, R), 20, 5, 1, field_kind=rf.FIELD_BIMODAL, h=1.5,
                          field_seed=10 + k, realization=k) for L, R, k in mix]
    for (L, R, k), t in zip(mix, tickets):
        res = srv.wait(t)
        o = oracle.Oracle(L, inputs.geometric_temps(1.0, 5.0, R), h=1.5, field_kind=oracle.FIELD_BIMODAL,
                          field_seed=10 + k, seed=42, realization=k)
        o.run(20, 5, 1)
        assert np.array_equal(res["sums"], o.observables()), (L, R)

# allocation-free exchange step on caller buffers (its checks synchronise in this flavour)
L, R = 16, 6
temps = inputs.geometric_temps(1.0, 5.0, R)
g = rf.Realization(L, temps, h=1.5, field_kind=rf.FIELD_BIMODAL, field_seed=3, seed=42, layout=rf.LAYOUT_BITPACK)
g.sweep(3)
st = g.get_state()
from tests.test_zz_no_alloc import pack_bits
dev = torch.device("cuda")
bufs = dict(spins=torch.from_numpy(pack_bits(st["spins"], L).view(np.int32)).to(dev),
            field=torch.from_numpy(g.field()).to(dev), beta=torch.from_numpy(1.0 / temps).to(dev),
            t2r=torch.arange(R, dtype=torch.int32, device=dev), r2t=torch.arange(R, dtype=torch.int32, device=dev),
            att=torch.zeros(R - 1, dtype=torch.int64, device=dev), acc=torch.zeros(R - 1, dtype=torch.int64, device=dev),
            obs=torch.zeros(R, 5, dtype=torch.float64, device=dev), n=torch.zeros(1, dtype=torch.int64, device=dev),
            E=torch.zeros(R, dtype=torch.float64, device=dev), M=torch.zeros(R, dtype=torch.int64, device=dev))
b = rf.ExchangeBuffers(L, R, 1.0, 1.5, rf.FIELD_BIMODAL, 42, 0, 0, *[bufs[k].data_ptr() for k in
                       ("spins", "field", "beta", "t2r", "r2t", "att", "acc", "obs", "n", "E", "M")])
rf.exchange_noalloc(b, 0, 0)
g.exchange(0)
assert np.array_equal(bufs["t2r"].cpu().numpy(), g.get_state()["t2r"])
assert np.array_equal(bufs["E"].cpu().numpy(), g.get_state(energies=True)["E"])
print("debug build ok")
'''


def test_debug_build_small_parity_cases():
    env = dict(os.environ, RFIM_LIBRARY="debug", RFIM_ROOT=ROOT)
    env.pop("RFIM_BITS_PLAN", None)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug build ok" in r.stdout

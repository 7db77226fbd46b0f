"""Small profiling driver for ncu captures of the sweep kernels.

`python -m paper_1508_06268_gb300.microbench.prof_driver [bimodal] [int8]`: the C4 shape (L=64,
R=128), four exchange intervals of 10 sweeps.
`python -m paper_1508_06268_gb300.microbench.prof_driver serve`: the batched serving kernel on a
C5-shaped mix of 16 Gaussian realizations (L = 8, 16, 32, 64 with R = 16, 32, 64, 128), 400 sweeps
each, submitted at once.
`python -m paper_1508_06268_gb300.microbench.prof_driver multihit`: the C4 shape with multi-hit
double-checkerboard sweeps (mh = 100, tiles 8^3), four launches of one sweep each."""
import sys

import torch

import paper_1508_06268_gb300 as rf
from paper_1508_06268_gb300 import inputs

if "serve" in sys.argv:
    mix = {8: 16, 16: 32, 32: 64, 64: 128}
    with rf.Server(mem_budget_bytes=2 << 30, max_slots=64, intervals_per_launch=4) as srv:
        tickets = [srv.submit(L, inputs.geometric_temps(1.0, 5.0, R), 400, 10, 20, field_kind=rf.FIELD_GAUSSIAN,
                              field_seed=1 + k, realization=k)
                   for k, (L, R) in enumerate(list(mix.items()) * 4)]
        for t in tickets:
            srv.wait(t)
    torch.cuda.synchronize()
    print("ok", len(tickets))
elif "multihit" in sys.argv:
    g = rf.Realization(64, inputs.geometric_temps(1.0, 5.0, 128), field_kind=rf.FIELD_GAUSSIAN)
    g.set_multihit(100, 8)
    g.run(4, 1, 0)
    torch.cuda.synchronize()
    print("ok", g.get_state(spins=False)["sweep"])
else:
    layout = rf.LAYOUT_INT8 if "int8" in sys.argv else rf.LAYOUT_BITPACK
    kind = rf.FIELD_BIMODAL if "bimodal" in sys.argv else rf.FIELD_GAUSSIAN
    g = rf.Realization(64, inputs.geometric_temps(1.0, 5.0, 128), field_kind=kind, layout=layout)
    g.run(40, 10, 0)
    torch.cuda.synchronize()
    print("ok", g.get_state(spins=False)["sweep"])

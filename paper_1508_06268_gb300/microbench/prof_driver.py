"""Small profiling driver for ncu captures of the sweep kernel: the C4 shape (L=64, R=128), four
exchange intervals of 10 sweeps.  `python -m paper_1508_06268_gb300.microbench.prof_driver [bimodal] [int8]`."""
import sys

import torch

import paper_1508_06268_gb300 as rf
from paper_1508_06268_gb300 import inputs

layout = rf.LAYOUT_INT8 if "int8" in sys.argv else rf.LAYOUT_BITPACK
kind = rf.FIELD_BIMODAL if "bimodal" in sys.argv else rf.FIELD_GAUSSIAN
g = rf.Realization(64, inputs.geometric_temps(1.0, 5.0, 128), field_kind=kind, layout=layout)
g.run(40, 10, 0)
torch.cuda.synchronize()
print("ok", g.get_state(spins=False)["sweep"])

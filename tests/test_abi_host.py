"""Host-side checks of the C-ABI library (no GPU): it builds, loads, exports every function that
include/rfim.h declares, and its bit-layout neighbour arithmetic matches direct lookup."""
from __future__ import annotations

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(rfim_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rfim_create", "rfim_destroy", "rfim_sweep", "rfim_exchange", "rfim_run",
                     "rfim_adapt_temps", "rfim_observables", "rfim_get_state", "rfim_set_state",
                     "rfim_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1508_06268_gb300 as rf
    lib = rf.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("L", [8, 16, 32, 64])
def test_bit_layout_neighbour_words(L):
    import paper_1508_06268_gb300 as rf
    for seed in (1, 2, 3):
        assert rf.selftest_bits(L, seed) == 0


def test_create_without_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_1508_06268_gb300 as rf
    with pytest.raises(rf.RfimError):
        rf.Realization(8, [1.0, 2.0], stream=0)


@pytest.mark.parametrize("L,R,P", [(64, 128, 152), (64, 128, 144), (64, 70, 152), (64, 8, 42), (32, 64, 152),
                                   (64, 6, 10), (16, 4, 3)])
def test_grid_partition(L, R, P):
    import paper_1508_06268_gb300 as rf
    assert rf.selftest_grid(L, R, P) == 0


def test_thermal_and_disorder_average_match_the_oracle():
    """Host-side derived observables of Sec. 7 (rfim_thermal, rfim_disorder_average) against the
    oracle's formulas on random accumulator sums."""
    import numpy as np
    import oracle
    import paper_1508_06268_gb300 as rf
    rng = np.random.default_rng(5)
    R, N, n = 6, 512, 250
    T = np.linspace(1.0, 4.0, R)
    thermals_lib, thermals_orc = [], []
    for _ in range(3):
        e = rng.normal(-1.5, 0.05, size=(n, R))
        m = rng.normal(0.3, 0.1, size=(n, R))
        F = rng.uniform(0.5, 3.0, size=(n, R))
        sums = np.stack([e.sum(0), (e * e).sum(0), np.abs(m).sum(0), (m * m).sum(0), (m ** 4).sum(0)], axis=1)
        obs = {"T": T, "e": sums[:, 0], "e2": sums[:, 1], "absm": sums[:, 2], "m2": sums[:, 3], "m4": sums[:, 4],
               "F": F.sum(0), "n_meas": n}
        thermals_lib.append(rf.thermal(obs, N))
        thermals_orc.append(oracle.thermal(sums, F.sum(0), n, N, T))
        np.testing.assert_allclose(thermals_lib[-1], thermals_orc[-1], rtol=1e-12, equal_nan=True)
    np.testing.assert_allclose(rf.disorder_average(thermals_lib), oracle.disorder_average(thermals_orc),
                               rtol=1e-12, equal_nan=True)
    no_F = dict(obs)
    no_F.pop("F")
    assert np.isnan(rf.thermal(no_F, N)[:, 5:]).all()

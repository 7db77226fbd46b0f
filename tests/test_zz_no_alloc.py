"""rfim_exchange_noalloc -- the exchange step for callers that cannot allocate device memory.

Such callers have all device memory owned by another allocator (a framework's pool, a fixed
arena), sit on a latency-critical path where cudaMalloc / cudaFree would synchronise the device,
or record their launches into a CUDA graph.  The entry point keeps its scratch in a static
device array; the caller passes every input and output.  Checked here against the allocating
entry point (rfim_exchange on a context holding the same state) on two calls in a row:
permutation, exchange counts and measurement counts exactly, energies and measurement sums to
1e-9 relative (bimodal: exactly).
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1508_06268_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_06268_gb300 as rf  # noqa: E402


def pack_bits(spins: np.ndarray, L: int) -> np.ndarray:
    """Natural-order +-1 spins [R, L^3] -> the documented bit layout uint32[R][2][L^3/64]."""
    R, N = spins.shape
    i = np.arange(N)
    x, y, z = i % L, (i // L) % L, i // (L * L)
    c = (x + y + z) % 2
    q = (x >> 1) + (L // 2) * (y + L * z)
    word, bit = q >> 5, 8 * (q & 3) + ((q & 31) >> 2)
    out = np.zeros((R, 2, N // 64), dtype=np.uint64)
    for r in range(R):
        up = (spins[r] > 0).astype(np.uint64)
        np.bitwise_or.at(out[r], (c, word), up << bit.astype(np.uint64))
    return out.astype(np.uint32)


@pytest.mark.parametrize("L,R,kind", [(16, 8, rf.FIELD_BIMODAL), (64, 16, rf.FIELD_GAUSSIAN),
                                      (32, 6, rf.FIELD_GAUSSIAN)])
def test_noalloc_exchange_matches_allocating_entry_point(L, R, kind):
    temps = inputs.geometric_temps(1.0, 5.0, R)
    h = 1.5 if kind == rf.FIELD_BIMODAL else 1.0
    g = rf.Realization(L, temps, h=h, field_kind=kind, field_seed=3, seed=42, realization=2,
                       layout=rf.LAYOUT_BITPACK)
    g.sweep(7)
    st = g.get_state()
    dev = torch.device("cuda")
    spins = torch.from_numpy(pack_bits(st["spins"], L).view(np.int32)).to(dev)
    field = torch.from_numpy(g.field()).to(dev)
    beta = torch.from_numpy(1.0 / temps).to(dev)
    t2r = torch.arange(R, dtype=torch.int32, device=dev)
    r2t = torch.arange(R, dtype=torch.int32, device=dev)
    att = torch.zeros(R - 1, dtype=torch.int64, device=dev)
    acc = torch.zeros(R - 1, dtype=torch.int64, device=dev)
    obs = torch.zeros(R, 5, dtype=torch.float64, device=dev)
    n_meas = torch.zeros(1, dtype=torch.int64, device=dev)
    E = torch.zeros(R, dtype=torch.float64, device=dev)
    M = torch.zeros(R, dtype=torch.int64, device=dev)
    b = rf.ExchangeBuffers(L, R, 1.0, h, kind, 42, 2, 0, spins.data_ptr(), field.data_ptr(),
                           beta.data_ptr(), t2r.data_ptr(), r2t.data_ptr(), att.data_ptr(),
                           acc.data_ptr(), obs.data_ptr(), n_meas.data_ptr(), E.data_ptr(), M.data_ptr())
    for j in range(2):
        rf.exchange_noalloc(b, j, 0)
        g.exchange(0)
        torch.cuda.synchronize()
        ref = g.get_state(energies=True)
        ob = g.observables()
        np.testing.assert_array_equal(t2r.cpu().numpy(), ref["t2r"])
        np.testing.assert_array_equal(att.cpu().numpy().astype(np.uint64), ob["att"])
        np.testing.assert_array_equal(acc.cpu().numpy().astype(np.uint64), ob["acc"])
        assert int(n_meas.item()) == ob["n_meas"] == j + 1
        if kind == rf.FIELD_BIMODAL:
            np.testing.assert_array_equal(E.cpu().numpy(), ref["E"])
            np.testing.assert_array_equal(obs.cpu().numpy(), ob["sums"])
        else:
            np.testing.assert_allclose(E.cpu().numpy(), ref["E"], rtol=1e-9, atol=1e-7)
            np.testing.assert_allclose(obs.cpu().numpy(), ob["sums"], rtol=1e-9, atol=1e-12)
        np.testing.assert_array_equal(M.cpu().numpy(),
                                      st["spins"].astype(np.int64).sum(axis=1))
    g.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    p = dummy.data_ptr()
    b = rf.ExchangeBuffers(8, 20000, 1.0, 1.0, rf.FIELD_GAUSSIAN, 1, 0, 0, p, p, p, p, p, p, p, p, p, p, p)
    with pytest.raises(rf.RfimError) as e:
        rf.exchange_noalloc(b, 0, 0)
    assert e.value.code == rf.EINVAL and "scratch" in str(e.value)

"""rfim_exchange_noalloc -- the exchange step for callers that cannot allocate device memory.

Such callers have all device memory owned by another allocator (a framework's pool, a fixed
arena), or sit on a latency-critical path where cudaMalloc / cudaFree would synchronise the
device.  The entry point keeps its scratch in a static
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


@pytest.mark.parametrize("L,R,kind,pre,measure_from", [
    (16, 8, rf.FIELD_BIMODAL, 0, 0),
    (64, 16, rf.FIELD_GAUSSIAN, 0, 0),
    (32, 6, rf.FIELD_GAUSSIAN, 0, 0),
    (8, 4, rf.FIELD_BIMODAL, 0, 0),       # one word per plane: the +-1 neighbour words are the word itself
    (8, 700, rf.FIELD_GAUSSIAN, 0, 0),    # more replicas than 608: one slab per replica
    (16, 8, rf.FIELD_BIMODAL, 5, 6),      # permuted start, the first calls before measure_from
])
def test_noalloc_exchange_matches_allocating_entry_point(L, R, kind, pre, measure_from):
    temps = inputs.geometric_temps(1.0, 5.0, R)
    h = 1.5 if kind == rf.FIELD_BIMODAL else 1.0
    g = rf.Realization(L, temps, h=h, field_kind=kind, field_seed=3, seed=42, realization=2,
                       layout=rf.LAYOUT_BITPACK)
    g.sweep(7)
    for _ in range(pre):  # earlier exchange steps of the allocating entry point
        g.exchange(measure_from)
        g.sweep(2)
    st = g.get_state()
    ob0 = g.observables()
    j0 = int(st["xstep"])
    assert j0 == pre
    dev = torch.device("cuda")
    spins = torch.from_numpy(pack_bits(st["spins"], L).view(np.int32)).to(dev)
    field = torch.from_numpy(g.field()).to(dev)
    beta = torch.from_numpy(1.0 / temps).to(dev)
    t2r_h = st["t2r"].astype(np.int32)
    r2t_h = np.empty_like(t2r_h)
    r2t_h[t2r_h] = np.arange(R, dtype=np.int32)
    if pre:
        assert not np.array_equal(t2r_h, np.arange(R)), "the start should be a non-identity permutation"
    t2r = torch.from_numpy(t2r_h).to(dev)
    r2t = torch.from_numpy(r2t_h).to(dev)
    att = torch.from_numpy(ob0["att"].astype(np.int64)).to(dev)
    acc = torch.from_numpy(ob0["acc"].astype(np.int64)).to(dev)
    obs = torch.from_numpy(np.ascontiguousarray(ob0["sums"], dtype=np.float64)).to(dev)
    n_meas = torch.tensor([int(ob0["n_meas"])], dtype=torch.int64, device=dev)
    E = torch.zeros(R, dtype=torch.float64, device=dev)
    M = torch.zeros(R, dtype=torch.int64, device=dev)
    b = rf.ExchangeBuffers(L, R, 1.0, h, kind, 42, 2, 0, spins.data_ptr(), field.data_ptr(),
                           beta.data_ptr(), t2r.data_ptr(), r2t.data_ptr(), att.data_ptr(),
                           acc.data_ptr(), obs.data_ptr(), n_meas.data_ptr(), E.data_ptr(), M.data_ptr())
    for j in range(j0, j0 + 2):
        rf.exchange_noalloc(b, j, measure_from)
        g.exchange(measure_from)
        torch.cuda.synchronize()
        ref = g.get_state(energies=True)
        ob = g.observables()
        np.testing.assert_array_equal(t2r.cpu().numpy(), ref["t2r"])
        np.testing.assert_array_equal(att.cpu().numpy().astype(np.uint64), ob["att"])
        np.testing.assert_array_equal(acc.cpu().numpy().astype(np.uint64), ob["acc"])
        assert int(n_meas.item()) == ob["n_meas"] == int(ob0["n_meas"]) + sum(
            1 for k in range(j0, j + 1) if k >= measure_from)
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

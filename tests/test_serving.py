"""Serving / continuous batching (GPU): each realization's result in a mixed batch equals the same
realization served alone and, for the bimodal field, the oracle bit for bit; admission control by
device-memory budget; errors reported at the boundary."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1508_06268_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_06268_gb300 as rf  # noqa: E402

MIX = [  # (L, R, field kind, realization)
    (8, 16, rf.FIELD_GAUSSIAN, 0), (16, 8, rf.FIELD_BIMODAL, 1), (32, 6, rf.FIELD_GAUSSIAN, 2),
    (64, 4, rf.FIELD_GAUSSIAN, 3), (8, 5, rf.FIELD_BIMODAL, 4), (16, 12, rf.FIELD_GAUSSIAN, 5),
    (32, 9, rf.FIELD_BIMODAL, 6), (64, 3, rf.FIELD_BIMODAL, 7),
]
SWEEPS, EX = 40, 10


def submit(srv, L, R, kind, real, sweeps=SWEEPS):
    return srv.submit(L, inputs.geometric_temps(1.0, 5.0, R), sweeps, EX, 1, field_kind=kind,
                      h=1.5 if kind == rf.FIELD_BIMODAL else 1.0, field_seed=10 + real, seed=42,
                      realization=real)


def test_results_same_alone_and_in_the_mix():
    with rf.Server(mem_budget_bytes=256 << 20, max_slots=16, intervals_per_launch=2, measure_xi=True) as srv:
        tickets = [submit(srv, *m) for m in MIX]
        mixed = [srv.wait(t) for t in tickets]
    for m, res in zip(MIX, mixed):
        with rf.Server(mem_budget_bytes=64 << 20, max_slots=1, intervals_per_launch=3, measure_xi=True) as solo:
            alone = solo.wait(submit(solo, *m))
        np.testing.assert_array_equal(res["sums"], alone["sums"], err_msg=str(m))
        np.testing.assert_array_equal(res["acc"], alone["acc"], err_msg=str(m))
        np.testing.assert_array_equal(res["F"], alone["F"], err_msg=str(m))
        assert res["n_meas"] == alone["n_meas"] == SWEEPS // EX - 1


@pytest.mark.parametrize("L,R,real", [(8, 18, 4), (16, 20, 1), (32, 9, 6), (64, 5, 7)])
def test_served_structure_factor_equals_oracle(L, R, real):
    """Structure factor of the correlation length (Sec. 7) measured inside the batched kernel,
    replica groups with a ragged last group: the per-temperature sums of F equal the oracle's
    (bimodal field, identical trajectories; only the order of the double additions differs)."""
    temps = inputs.geometric_temps(1.0, 5.0, R)
    with rf.Server(mem_budget_bytes=64 << 20, max_slots=2, measure_xi=True) as srv:
        res = srv.wait(submit(srv, L, R, rf.FIELD_BIMODAL, real))
    o = oracle.Oracle(L, temps, h=1.5, field_kind=oracle.FIELD_BIMODAL, field_seed=10 + real, seed=42,
                      realization=real)
    o.set_measure_xi(True)
    o.run(SWEEPS, EX, 1)
    np.testing.assert_array_equal(res["sums"], o.observables())
    assert res["F"].all()
    np.testing.assert_allclose(res["F"], o.observables_F(), rtol=1e-11, atol=1e-20)


def test_served_structure_factor_equals_single_realization_path():
    """Gaussian field: the fused measurement of the batched kernel and the stand-alone kernel of a
    single-realization run give the same F sums (same trajectory, both from integer marginals)."""
    L, R = 32, 6
    temps = inputs.geometric_temps(1.0, 5.0, R)
    with rf.Server(mem_budget_bytes=64 << 20, max_slots=1, measure_xi=True) as srv:
        res = srv.wait(srv.submit(L, temps, SWEEPS, EX, 1, field_kind=rf.FIELD_GAUSSIAN, field_seed=3, seed=42,
                                  realization=2))
    g = rf.Realization(L, temps, field_kind=rf.FIELD_GAUSSIAN, field_seed=3, seed=42, realization=2,
                       layout=rf.LAYOUT_BITPACK)
    g.set_measure_xi(True)
    g.run(SWEEPS, EX, 1)
    obs = g.observables()
    # energies come from differently split error-free sums: equal up to the last bits
    np.testing.assert_allclose(res["sums"], obs["sums"], rtol=1e-12)
    np.testing.assert_allclose(res["F"], obs["F"], rtol=1e-12, atol=1e-20)


@pytest.mark.parametrize("L,R,real", [(8, 5, 4), (16, 8, 1), (32, 9, 6), (64, 3, 7)])
def test_bimodal_served_equals_oracle(L, R, real):
    temps = inputs.geometric_temps(1.0, 5.0, R)
    with rf.Server(mem_budget_bytes=64 << 20, max_slots=2) as srv:
        res = srv.wait(submit(srv, L, R, rf.FIELD_BIMODAL, real))
    o = oracle.Oracle(L, temps, h=1.5, field_kind=oracle.FIELD_BIMODAL, field_seed=10 + real, seed=42,
                      realization=real)
    o.run(SWEEPS, EX, 1)
    np.testing.assert_array_equal(res["sums"], o.observables())
    assert not res["F"].any()  # not measured unless the server is asked to
    att, acc = o.exchange_stats()
    np.testing.assert_array_equal(res["att"], att)
    np.testing.assert_array_equal(res["acc"], acc)


def test_admission_by_memory_budget():
    # budget for two L=32, R=16 Gaussian realizations (about 0.67 MB each) at a time
    with rf.Server(mem_budget_bytes=1_400_000, max_slots=8, intervals_per_launch=1) as srv:
        tickets = [submit(srv, 32, 16, rf.FIELD_GAUSSIAN, r, sweeps=20) for r in range(6)]
        peak = 0
        results = {}
        while len(results) < len(tickets):
            peak = max(peak, srv.stats()["resident"])
            for t in tickets:
                if t not in results:
                    r = srv.poll(t)
                    if r is not None:
                        results[t] = r
        st = srv.stats()
    assert st["completed"] == 6 and st["queued"] == 0
    assert 1 <= peak <= 2


def test_errors_at_the_boundary():
    with rf.Server(mem_budget_bytes=2 << 20, max_slots=2) as srv:
        with pytest.raises(rf.RfimError):
            srv.submit(12, inputs.geometric_temps(1.0, 5.0, 4), 20, 10)  # unsupported L
        with pytest.raises(rf.RfimError):
            srv.submit(8, inputs.geometric_temps(1.0, 5.0, 4), 25, 10)  # not a multiple
        with pytest.raises(rf.RfimError):
            srv.poll(12345)  # unknown ticket
        t = srv.submit(64, inputs.geometric_temps(1.0, 5.0, 64), 10, 10)  # larger than the budget
        with pytest.raises(rf.RfimError) as e:
            srv.wait(t, timeout_s=60)
        assert e.value.code == rf.ENOMEM


def test_served_maximum_replica_count_equals_oracle():
    """The largest served temperature set (R = 1024, L = 8: 64 replica groups of 16) with the
    structure factor measured: observables, exchange statistics and F sums equal the oracle's."""
    L, R, real = 8, 1024, 3
    temps = inputs.geometric_temps(1.0, 5.0, R)
    with rf.Server(mem_budget_bytes=64 << 20, max_slots=2, measure_xi=True) as srv:
        res = srv.wait(submit(srv, L, R, rf.FIELD_BIMODAL, real, sweeps=20))
    o = oracle.Oracle(L, temps, h=1.5, field_kind=oracle.FIELD_BIMODAL, field_seed=10 + real, seed=42,
                      realization=real)
    o.set_measure_xi(True)
    o.run(20, EX, 1)
    np.testing.assert_array_equal(res["sums"], o.observables())
    att, acc = o.exchange_stats()
    np.testing.assert_array_equal(res["acc"], acc)
    np.testing.assert_allclose(res["F"], o.observables_F(), rtol=1e-11, atol=1e-20)


def test_served_full_size_equals_oracle():
    """A served realization of the largest C5 shape (L = 64, R = 128: 64 work items of two
    replicas) with the structure factor measured equals the oracle."""
    L, R, real = 64, 128, 5
    temps = inputs.geometric_temps(1.0, 5.0, R)
    with rf.Server(mem_budget_bytes=256 << 20, max_slots=2, measure_xi=True) as srv:
        res = srv.wait(srv.submit(L, temps, 4, 2, 1, field_kind=rf.FIELD_BIMODAL, h=1.5, field_seed=10 + real,
                                  seed=42, realization=real))
    o = oracle.Oracle(L, temps, h=1.5, field_kind=oracle.FIELD_BIMODAL, field_seed=10 + real, seed=42,
                      realization=real)
    o.set_measure_xi(True)
    o.run(4, 2, 1)
    np.testing.assert_array_equal(res["sums"], o.observables())
    np.testing.assert_array_equal(res["acc"], o.exchange_stats()[1])
    np.testing.assert_allclose(res["F"], o.observables_F(), rtol=1e-11, atol=1e-20)


DEFAULT_SHAPES = "64:2:2,32:8:2,16:16:1,8:16:1"


def test_tuned_server_gives_the_results_of_untuned_ones():
    """Batched-kernel tuner (replicas per work item and per thread for each L, intervals per graph
    replay): a server with the tuned settings, one with the built-in shapes and one with other
    shapes serve the mix with identical results; the bimodal ones equal the oracle."""
    tuned = rf.server_tune([(m[0], m[1]) for m in MIX], field_kind=rf.FIELD_GAUSSIAN, sweeps=20, exchange_every=10,
                           mem_budget_bytes=256 << 20)
    assert tuned["intervals_per_launch"] in (1, 2, 4, 8) and tuned["attempts_per_ns"] > 0
    assert [int(x.split(":")[0]) for x in tuned["batch_shapes"].split(",")] == [64, 32, 16, 8]
    runs = []
    for shapes, k in ((None, 0), (DEFAULT_SHAPES, 4), ("64:1:1,32:4:1,16:4:1,8:8:1", 3)):
        with rf.Server(mem_budget_bytes=256 << 20, max_slots=16, intervals_per_launch=k, measure_xi=True,
                       batch_shapes=shapes) as srv:
            st = srv.stats()
            if shapes is None:  # the defaults are the tuner's choice
                assert st["batch_shapes"] == tuned["batch_shapes"]
                assert st["intervals_per_launch"] == tuned["intervals_per_launch"]
            else:
                assert st["batch_shapes"] == shapes and st["intervals_per_launch"] == k
            tickets = [submit(srv, *m) for m in MIX]
            runs.append([srv.wait(t) for t in tickets])
    for other in runs[1:]:
        for m, a, b in zip(MIX, runs[0], other):
            for key in ("sums", "att", "acc", "F"):
                np.testing.assert_array_equal(a[key], b[key], err_msg=f"{m} {key}")
    for m, res in zip(MIX, runs[0]):
        L, R, kind, real = m
        if kind != rf.FIELD_BIMODAL:
            continue
        o = oracle.Oracle(L, inputs.geometric_temps(1.0, 5.0, R), h=1.5, field_kind=oracle.FIELD_BIMODAL,
                          field_seed=10 + real, seed=42, realization=real)
        o.run(SWEEPS, EX, 1)
        np.testing.assert_array_equal(res["sums"], o.observables(), err_msg=str(m))


@pytest.mark.parametrize("shapes", ["64:3:2", "64:2:4", "12:4:1", "64:2", "64:2:2;32:8:2", "64:16:2"])
def test_invalid_batch_shapes_rejected(shapes):
    with pytest.raises(rf.RfimError) as e:
        rf.Server(mem_budget_bytes=16 << 20, max_slots=2, batch_shapes=shapes)
    assert e.value.code == rf.EINVAL


def test_servers_of_different_shapes_coexist():
    """The batched kernel is shared by all servers: creating a server with smaller shapes must not
    shrink the shared-memory limit that an earlier server's captured launches need."""
    big = rf.Server(mem_budget_bytes=64 << 20, max_slots=2, batch_shapes="64:4:2")
    small = rf.Server(mem_budget_bytes=64 << 20, max_slots=2, batch_shapes="64:1:1,32:4:1,16:4:1,8:8:1")
    try:
        a = big.wait(submit(big, 64, 8, rf.FIELD_BIMODAL, 7))
        b = small.wait(submit(small, 64, 8, rf.FIELD_BIMODAL, 7))
        for key in ("sums", "att", "acc"):
            np.testing.assert_array_equal(a[key], b[key])
    finally:
        big.close()
        small.close()

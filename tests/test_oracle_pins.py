"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Every test here runs on the CPU only.  Pins used: an independent Philox4x32-10 implementation
(triton's, run by its CPU interpreter), brute-force energies by periodic array shifts, exact
enumeration of the 2x2x2 lattice (Boltzmann averages and the exact one-sweep transition matrix),
closed forms (J = 0 independent spins, h = 0 low- and high-temperature expansions of the 3D
Ising model), the exact stationary law of the exchange-only permutation chain, a sort-based
reference for the min-heap selection of Sec. 4, recomputation of the Sec. 7 accumulators, and
for the multi-hit double checkerboard of Sec. 3.2 its reduction to the plain checkerboard, its
flip count at infinite temperature and a numpy zero-temperature sweep.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from oracle import Oracle, FIELD_BIMODAL, FIELD_GAUSSIAN, FIELD_EXPLICIT
from paper_1508_06268_gb300 import inputs
from tests import brute

TAG_INIT, TAG_METRO, TAG_EXCH, TAG_FIELD = 1, 2, 3, 4


def c3(tag, stage, colour):
    return (tag << 28) | (stage << 1) | colour


# ------------------------------------------------------------------ Philox (Salmon et al.)
_TRITON_KERNEL = None


def _triton_kernel():
    """Builds a kernel around triton's own Philox4x32-10, run by triton's CPU interpreter."""
    global _TRITON_KERNEL, tphilox, tl
    if _TRITON_KERNEL is None:
        os.environ["TRITON_INTERPRET"] = "1"
        pytest.importorskip("torch")
        triton = pytest.importorskip("triton")
        import triton.language as tl
        from triton.language.random import philox as tphilox

        @triton.jit
        def _k(cp, outp, seed, n, BLOCK: tl.constexpr):
            offs = tl.arange(0, BLOCK)
            m = offs < n
            c0 = tl.load(cp + offs * 4 + 0, mask=m).to(tl.uint32, bitcast=True)
            c1 = tl.load(cp + offs * 4 + 1, mask=m).to(tl.uint32, bitcast=True)
            c2 = tl.load(cp + offs * 4 + 2, mask=m).to(tl.uint32, bitcast=True)
            c3_ = tl.load(cp + offs * 4 + 3, mask=m).to(tl.uint32, bitcast=True)
            a, b, c, d = tphilox(seed, c0, c1, c2, c3_)
            tl.store(outp + offs * 4 + 0, a.to(tl.int32, bitcast=True), mask=m)
            tl.store(outp + offs * 4 + 1, b.to(tl.int32, bitcast=True), mask=m)
            tl.store(outp + offs * 4 + 2, c.to(tl.int32, bitcast=True), mask=m)
            tl.store(outp + offs * 4 + 3, d.to(tl.int32, bitcast=True), mask=m)

        _TRITON_KERNEL = _k
    return _TRITON_KERNEL


def _triton_philox(key, ctrs):
    """triton's Philox4x32-10 on an [n, 4] uint32 counter array with key (k0, k1)."""
    import torch
    k = _triton_kernel()
    ctrs = np.ascontiguousarray(ctrs, dtype=np.uint32)
    n = ctrs.shape[0]
    block = 1 << max(4, (n - 1).bit_length())
    out = torch.zeros(n * 4, dtype=torch.int32)
    k[(1,)](torch.from_numpy(ctrs.view(np.int32).reshape(-1).copy()), out,
            int(key[0]) | (int(key[1]) << 32), n, BLOCK=block)
    return out.numpy().view(np.uint32).reshape(n, 4)


@pytest.mark.parametrize("key", [(0, 0), (42, 7), (0xFFFFFFFF, 0xFFFFFFFF), (0x9E3779B9, 1)])
def test_philox_matches_independent_implementation(key):
    rng = np.random.default_rng(key[0] ^ 1234)
    ctrs = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    ctrs[0] = 0
    ctrs[1] = 0xFFFFFFFF
    ref = _triton_philox(key, ctrs)
    mine = np.array([oracle.philox4x32_10(key, c) for c in ctrs])
    np.testing.assert_array_equal(mine, ref)


def test_philox_uniformity():
    words = np.concatenate([oracle.philox4x32_10((42, 3), (i, 5, 9, c3(TAG_METRO, 0, 1)))
                            for i in range(4096)]).astype(np.float64)
    u = words / 2 ** 32
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    counts = np.histogram(u, bins=16, range=(0, 1))[0]
    exp = u.size / 16
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 45.0  # chi^2 with 15 dof: p ~ 1e-4


# ------------------------------------------------------------------ field (Sec. 3.1 step 2)
def test_bimodal_field_stream_and_balance():
    L, fs, real = 8, 11, 3
    h = oracle.make_field(L, FIELD_BIMODAL, fs, real)
    N = L ** 3
    ctrs = np.array([(i >> 2, 0, 0, c3(TAG_FIELD, 0, 0)) for i in range(0, N, 4)], dtype=np.uint32)
    words = _triton_philox((fs, real), ctrs).reshape(-1)
    np.testing.assert_array_equal(h, np.where(words >> 31, -1.0, 1.0).astype(np.float32))
    big = oracle.make_field(32, FIELD_BIMODAL, 1, 0)
    assert set(np.unique(big)) == {-1.0, 1.0}
    assert abs(big.mean()) < 5 / math.sqrt(big.size)


def test_gaussian_field_distribution():
    from scipy import stats
    h = oracle.make_field(32, FIELD_GAUSSIAN, 1, 0).astype(np.float64)
    assert abs(h.mean()) < 5 / math.sqrt(h.size)
    assert abs(h.var() - 1.0) < 5 * math.sqrt(2 / h.size)
    assert stats.kstest(h, "norm").pvalue > 1e-3


def test_gaussian_field_stream():
    L, fs, real = 4, 5, 9
    h = oracle.make_field(L, FIELD_GAUSSIAN, fs, real)
    N = L ** 3
    ctrs = np.array([(i >> 1, 1, 0, c3(TAG_FIELD, 0, 0)) for i in range(0, N, 2)], dtype=np.uint32)
    w = _triton_philox((fs, real), ctrs).astype(np.float64)
    ref = np.empty(N)
    for i in range(N):
        a, b = w[i >> 1, 2 * (i & 1)], w[i >> 1, 2 * (i & 1) + 1]
        u1, u2 = (a + 0.5) / 2 ** 32, (b + 0.5) / 2 ** 32
        ref[i] = math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2)
    # same double-precision transform, rounded to float: at most one float ulp apart
    assert np.max(np.abs(h.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1e-30)) < 2 ** -23


# ------------------------------------------------------------------ energy (Eq. 1)
@pytest.mark.parametrize("L,kind", [(2, FIELD_BIMODAL), (2, FIELD_GAUSSIAN), (4, FIELD_BIMODAL),
                                    (4, FIELD_GAUSSIAN), (6, FIELD_GAUSSIAN)])
def test_energy_brute_force(L, kind):
    J, h = 0.75, 1.3
    temps = inputs.geometric_temps(1.0, 4.0, 3)
    o = Oracle(L, temps, J=J, h=h, field_kind=kind, field_seed=3, seed=9)
    s = inputs.random_spins(3, L, seed=L * 10 + kind)
    o.set_spins(s)
    hraw, hh = o.field()
    np.testing.assert_array_equal(hh, brute.scaled_field(h, hraw))
    for r in range(3):
        E, B, F, M = o.energy(r)
        ref = brute.energy(s[r], L, J, hh)
        assert abs(E - ref) <= 1e-9 * max(1.0, abs(ref))
        assert M == int(s[r].astype(np.int64).sum())


@pytest.mark.parametrize("L,kind", [(2, FIELD_BIMODAL), (2, FIELD_GAUSSIAN), (4, FIELD_BIMODAL),
                                    (4, FIELD_EXPLICIT)])
def test_single_flip_delta_equals_energy_difference(L, kind):
    J, h = 1.0, 1.5
    temps = inputs.geometric_temps(1.0, 4.0, 2)
    field = inputs.gaussian_field(L, 77) if kind == FIELD_EXPLICIT else None
    o = Oracle(L, temps, J=J, h=h, field_kind=kind, field=field, field_seed=2, seed=5)
    _, hh = o.field()
    rng = np.random.default_rng(L)
    for trial in range(4):
        s = inputs.random_spins(2, L, seed=100 + trial)
        o.set_spins(s)
        for site in range(L ** 3):
            x, y, z = site % L, (site // L) % L, site // (L * L)
            dE = o.delta_e(0, x, y, z)
            s2 = s.copy()
            s2[0, site] = -s2[0, site]
            ref = brute.energy(s2[0], L, J, hh) - brute.energy(s[0], L, J, hh)
            if kind == FIELD_BIMODAL:
                assert dE == ref  # exact integers times h
            else:
                assert abs(dE - ref) <= 4e-6 * max(1.0, abs(ref))
    # exhaustive over all 2x2x2 states for one site
    if L == 2:
        for st in brute.all_states(8)[::7]:
            o.set_spins(np.stack([st, st]))
            dE = o.delta_e(0, 1, 0, 1)
            st2 = st.copy()
            st2[1 + 2 * (0 + 2 * 1)] *= -1
            ref = brute.energy(st2, 2, J, hh) - brute.energy(st, 2, J, hh)
            assert abs(dE - ref) <= 4e-6 * max(1.0, abs(ref))


def test_bimodal_threshold_properties():
    assert oracle.bimodal_threshold(1.0, 0.0) == 2 ** 32
    assert oracle.bimodal_threshold(1.0, -4.0) == 2 ** 32
    assert oracle.bimodal_threshold(10.0, 40.0) == 1  # clamped to the smallest probability
    prev = 2 ** 32
    for dE in (0.5, 1.0, 2.0, 4.0, 8.0, 12.0, 20.0):
        t = oracle.bimodal_threshold(0.7, dE)
        assert t < prev
        assert abs(t / 2 ** 32 - math.exp(-0.7 * dE)) <= 2 ** -32
        prev = t


# ------------------------------------------------------------------ Metropolis + checkerboard
def test_exact_transition_matrix_2x2x2_has_boltzmann_stationary_law():
    """One checkerboard sweep (Eq. 3 colours) built from the oracle's own acceptance
    probabilities leaves the exact Boltzmann distribution invariant (global balance)."""
    L, J, h, beta = 2, 1.0, 1.5, 0.45
    o = Oracle(L, np.array([1 / beta, 2 / beta]), J=J, h=h, field_kind=FIELD_BIMODAL, field_seed=4)
    _, hh = o.field()
    states = brute.all_states(8)
    colour = brute.colour_of(L)
    E = np.array([brute.energy(s, L, J, hh) for s in states])
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    flip_p = np.zeros((256, 8))
    for a, st in enumerate(states):
        o.set_spins(np.stack([st, st]))
        for site in range(8):
            x, y, z = site % 2, (site // 2) % 2, site // 4
            flip_p[a, site] = oracle.bimodal_threshold(beta, o.delta_e(0, x, y, z)) / 2 ** 32
    P = np.eye(256)
    for c in (0, 1):
        Pc = np.zeros((256, 256))
        sites = [i for i in range(8) if colour[i] == c]
        for a in range(256):
            for mask in range(1 << len(sites)):
                b, p = a, 1.0
                for t, site in enumerate(sites):
                    if (mask >> t) & 1:
                        b ^= 1 << site
                        p *= flip_p[a, site]
                    else:
                        p *= 1.0 - flip_p[a, site]
                Pc[a, b] += p
        P = P @ Pc
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(pi @ P, pi, atol=1e-8)


def _binned(o, n_bins, sweeps_per_bin, ex):
    means, prev, prev_n = [], o.observables(), o.n_meas
    for _ in range(n_bins):
        o.run(sweeps_per_bin, ex, 0)
        cur, n = o.observables(), o.n_meas
        means.append((cur - prev) / (n - prev_n))
        prev, prev_n = cur, n
    means = np.array(means)
    return means.mean(axis=0), means.std(axis=0, ddof=1) / math.sqrt(n_bins)


@pytest.mark.parametrize("kind", [FIELD_BIMODAL, FIELD_GAUSSIAN])
def test_mcmc_2x2x2_matches_exact_enumeration(kind):
    L, J, h = 2, 1.0, 1.0
    temps = np.array([1.0, 1.6, 2.6, 4.0])
    o = Oracle(L, temps, J=J, h=h, field_kind=kind, field_seed=6, seed=17)
    _, hh = o.field()
    o.run(200, 1, 10 ** 9)  # burn-in, no measurement
    mean, err = _binned(o, 20, 5000, 1)
    for k, T in enumerate(temps):
        exact = brute.exact_averages(L, J, hh, 1.0 / T)
        for col in (0, 2, 3):
            assert abs(mean[k, col] - exact[col]) < 5 * err[k, col] + 1e-12, (k, col)


def test_zero_coupling_closed_form():
    """J = 0: independent spins, <s_i> = tanh(beta hh_i), <e> = -(1/N) sum hh_i tanh(beta hh_i)."""
    L = 8
    temps = np.array([0.8, 1.5, 3.0])
    o = Oracle(L, temps, J=0.0, h=1.0, field_kind=FIELD_GAUSSIAN, field_seed=8, seed=3)
    _, hh = o.field()
    hh = hh.astype(np.float64)
    o.run(100, 1, 10 ** 9)
    mean, err = _binned(o, 20, 300, 1)
    for k, T in enumerate(temps):
        exact = -np.mean(hh * np.tanh(hh / T))
        assert abs(mean[k, 0] - exact) < 5 * err[k, 0] + 1e-9, k


def test_zero_field_low_temperature_expansion():
    """h = 0, ordered start: e = -3 + 12 exp(-12 beta) + O(exp(-20 beta)) (single-spin excitations)."""
    L = 8
    temps = np.array([1.1, 1.25])
    o = Oracle(L, temps, J=1.0, h=0.0, field_kind=FIELD_BIMODAL, seed=21)
    o.set_spins(np.ones((2, L ** 3), dtype=np.int8))
    o.run(200, 1, 10 ** 9)
    mean, err = _binned(o, 20, 500, 1)
    for k, T in enumerate(temps):
        b = 1.0 / T
        exact = -3.0 + 12.0 * math.exp(-12 * b)
        corr = 60.0 * math.exp(-20 * b)  # bound on the next order
        assert abs(mean[k, 0] - exact) < 5 * err[k, 0] + corr, (k, mean[k, 0], exact, err[k, 0])
        assert mean[k, 2] > 0.99  # stays magnetised


def test_zero_field_high_temperature_expansion():
    """h = 0: nearest-neighbour correlation t + 4 t^3 + O(t^5), t = tanh(beta): e = -3 (t + 4 t^3)."""
    L = 8
    temps = np.array([16.0, 25.0])
    o = Oracle(L, temps, J=1.0, h=0.0, field_kind=FIELD_BIMODAL, seed=23)
    o.run(100, 1, 10 ** 9)
    mean, err = _binned(o, 20, 400, 1)
    for k, T in enumerate(temps):
        t = math.tanh(1.0 / T)
        exact = -3.0 * (t + 4 * t ** 3)
        assert abs(mean[k, 0] - exact) < 5 * err[k, 0] + 3 * 30 * t ** 5, (k, mean[k, 0], exact)


# ------------------------------------------------------------------ exchange (Eq. 2, Sec. 3.3)
def test_exchange_only_chain_has_exact_stationary_law():
    L, J, h = 2, 1.0, 0.5
    temps = np.array([2.0, 2.6, 3.4])
    o = Oracle(L, temps, J=J, h=h, field_kind=FIELD_BIMODAL, field_seed=1, seed=31)
    st = brute.all_states(8)
    o.set_spins(np.stack([st[255], st[90], st[21]]))
    _, hh = o.field()
    E = np.array([brute.energy(o.spins()[r], L, J, hh) for r in range(3)])
    assert len(set(E.tolist())) == 3
    perms = brute.permutations_of(3)
    beta = 1.0 / temps
    w = np.array([math.exp(-sum(beta[k] * E[p[k]] for k in range(3))) for p in perms])
    w /= w.sum()
    n_steps, n_bins = 60000, 20
    visits = np.zeros((n_bins, len(perms)))
    flux = np.zeros((len(perms), len(perms)))
    cur = perms.index(tuple(o.perm()[0]))
    for step in range(n_steps):
        o.exchange(10 ** 9)
        nxt = perms.index(tuple(o.perm()[0]))
        visits[step * n_bins // n_steps, nxt] += 1
        flux[cur, nxt] += 1
        cur = nxt
    freq = visits / visits.sum(axis=1, keepdims=True)
    mean = freq.mean(axis=0)
    err = freq.std(axis=0, ddof=1) / math.sqrt(n_bins)
    assert np.all(np.abs(mean - w) < 5 * err + 1e-3), (mean, w)
    # detailed balance of the pair moves: flux a->b equals flux b->a
    for a in range(6):
        for b in range(a + 1, 6):
            tot = flux[a, b] + flux[b, a]
            if tot > 0:
                assert abs(flux[a, b] - flux[b, a]) < 5 * math.sqrt(tot) + 2
    att, acc = o.exchange_stats()
    assert att[0] == n_steps // 2 and att[1] == n_steps // 2  # odd xor even alternation


def test_exchange_counter_semantics():
    temps = inputs.geometric_temps(1.0, 5.0, 4)
    o = Oracle(4, temps, field_kind=FIELD_BIMODAL)
    o.run(25, 10, 0)
    assert o.sweep_count == 25 and o.xstep_count == 2 and o.n_meas == 2
    o.run(5, 10, 0)
    assert o.sweep_count == 30 and o.xstep_count == 3
    att, _ = o.exchange_stats()
    assert att.tolist() == [2, 1, 2]  # steps 0, 2 use even pairs; step 1 odd pairs


def test_measurement_accumulators_match_recomputation():
    L, J, h = 4, 1.0, 1.0
    temps = inputs.geometric_temps(1.5, 4.0, 3)
    o = Oracle(L, temps, J=J, h=h, field_kind=FIELD_GAUSSIAN, field_seed=2, seed=8)
    _, hh = o.field()
    acc = np.zeros((3, 5))
    for step in range(12):
        o.run(1, 1, 3)
        if step >= 3:
            s = o.spins()
            t2r, _ = o.perm()
            for k in range(3):
                e = brute.energy(s[t2r[k]], L, J, hh) / L ** 3
                m = s[t2r[k]].astype(np.float64).sum() / L ** 3
                acc[k] += [e, e * e, abs(m), m * m, m ** 4]
    assert o.n_meas == 9
    np.testing.assert_allclose(o.observables(), acc, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ adaptation (Sec. 4)
def test_heap_selection_equals_sort():
    rng = np.random.default_rng(5)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        rates = np.round(rng.random(n), 1)
        a = int(rng.integers(0, n + 1))
        ref = [k for _, k in sorted((r, k) for k, r in enumerate(rates))][:a]
        assert oracle.select_lowest(rates, a).tolist() == ref


def test_adaptation_inserts_midpoints_at_lowest_rates():
    L, R0, trials, a = 4, 5, 3, 2
    temps = inputs.geometric_temps(1.0, 5.0, R0)
    o = Oracle(L, temps, J=1.0, h=1.0, field_kind=FIELD_BIMODAL, R_capacity=R0 + trials * a)
    R, rates = o.adapt(trials, 400, 5, a, return_rates=True)
    assert R == R0 + trials * a
    cur = list(temps)
    for t in range(trials):
        rt = rates[t, :len(cur) - 1]
        assert np.all((rt >= 0) & (rt <= 1))
        pick = [k for _, k in sorted((r, k) for k, r in enumerate(rt))][:a]
        cur = sorted(cur + [0.5 * (cur[k] + cur[k + 1]) for k in pick])
    final = o.temps()
    np.testing.assert_array_equal(final, np.array(cur))
    assert np.all(np.diff(final) > 0)
    # reset to stage 0 afterwards
    assert o.sweep_count == 0 and o.xstep_count == 0 and o.n_meas == 0
    np.testing.assert_array_equal(o.perm()[0], np.arange(R))


def test_adaptation_rejects_over_capacity():
    temps = inputs.geometric_temps(1.0, 5.0, 4)
    o = Oracle(4, temps, field_kind=FIELD_BIMODAL, R_capacity=6)
    with pytest.raises(ValueError):
        o.adapt(2, 10, 5, 2)


# ------------------------------------------------------------ Sec. 7 observables beyond e and m
@pytest.mark.parametrize("L", [2, 4, 6, 8])
def test_structure_factor_matches_fft_of_marginals(L):
    rng = np.random.default_rng(L)
    R = 3
    o = Oracle(L, inputs.geometric_temps(1.0, 3.0, R), field_kind=FIELD_BIMODAL, seed=5)
    s = rng.choice(np.array([-1, 1], dtype=np.int8), size=(R, L ** 3))
    o.set_spins(s)
    for r in range(R):
        assert o.structure_F(r) == pytest.approx(brute.structure_factor_fft(s[r], L), rel=1e-12, abs=1e-12)


def test_structure_factor_of_uniform_and_staggered_lattices():
    L = 8
    o = Oracle(L, [1.0, 2.0], field_kind=FIELD_BIMODAL)
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    up = np.ones(L ** 3, dtype=np.int8)
    stripes = np.where(np.cos(2 * np.pi * x / L) >= 0, 1, -1).astype(np.int8).reshape(-1)  # half-period slabs in x
    o.set_spins(np.stack([up, stripes]))
    assert abs(o.structure_F(0)) < 1e-20  # a full period of cos and sin sums to zero
    xi = oracle.thermal(np.array([[0.0, 0.0, 1.0, 1.0, 1.0]]), np.array([o.structure_F(0)]), 1, L ** 3,
                        np.array([1.0]))[0, 6]
    assert xi == np.inf  # an ordered lattice: the second-moment length diverges
    # slabs along x: only the x axis contributes, |sum_x s(x) e^{iKx}|^2 L^4 / (3 L^3)
    sx = np.where(np.cos(2 * np.pi * np.arange(L) / L) >= 0, 1.0, -1.0)
    want = abs(np.sum(sx * np.exp(2j * np.pi * np.arange(L) / L))) ** 2 * L ** 4 / (3 * L ** 3)
    assert o.structure_F(1) == pytest.approx(want, rel=1e-12)


def test_structure_factor_accumulates_lattice_at_each_temperature():
    L, R = 4, 3
    o = Oracle(L, inputs.geometric_temps(1.0, 4.0, R), field_kind=FIELD_BIMODAL, h=1.2, seed=9)
    o.set_measure_xi(True)
    want = np.zeros(R)
    for _ in range(12):
        o.run(1, 1, 0)  # one sweep, then an exchange step with its measurement
        t2r, _ = o.perm()
        s = o.spins()
        want += [brute.structure_factor_fft(s[t2r[k]], L) for k in range(R)]
    np.testing.assert_allclose(o.observables_F(), want, rtol=1e-12)
    assert o.n_meas == 12


def test_specific_heat_equals_temperature_derivative_of_energy():
    """C = (N / T^2)(<e^2> - <e>^2) from accumulator sums equals d<e>/dT, the specific heat per
    site (fluctuation-dissipation; exact 2x2x2 enumeration)."""
    L, J = 2, 1.0
    hh = brute.scaled_field(1.0, np.where(np.arange(8) % 3 == 0, 1.0, -1.0))
    N = L ** 3
    for T in (1.5, 3.0, 6.0):
        E1, E2 = brute.exact_energy_moments(L, J, hh, 1.0 / T)
        n = 1000
        obs = np.array([[n * E1 / N, n * E2 / N ** 2, 0.0, 0.0, 0.0]])
        C = oracle.thermal(obs, None, n, N, np.array([T]))[0, 1]
        dT = 1e-4 * T
        ep = brute.exact_energy_moments(L, J, hh, 1.0 / (T + dT))[0] / N
        em = brute.exact_energy_moments(L, J, hh, 1.0 / (T - dT))[0] / N
        assert C == pytest.approx((ep - em) / (2 * dT), rel=1e-6)


def test_binder_factor_limits():
    """g = 1 for a magnetisation of fixed modulus, g -> 0 for a Gaussian one (textbook limits)."""
    rng = np.random.default_rng(3)
    n, N = 20000, 64
    T = np.array([1.0])

    def sums(m):
        return np.array([[0.0, 0.0, np.abs(m).sum(), (m ** 2).sum(), (m ** 4).sum()]])

    ordered = oracle.thermal(sums(rng.choice([-1.0, 1.0], size=n)), None, n, N, T)
    gauss = oracle.thermal(sums(rng.normal(0.0, 0.1, size=n)), None, n, N, T)
    avg = oracle.disorder_average([ordered, ordered])
    assert avg[0, 4] == pytest.approx(1.0, abs=1e-12)
    assert abs(oracle.disorder_average([gauss])[0, 4]) < 0.05


def test_correlation_length_vanishes_for_independent_spins():
    """Independent +-1 spins (beta = 0): N <m^2> = <F> = 1, so xi = 0; measured on sampled
    lattices through the oracle's own F and magnetisation."""
    rng = np.random.default_rng(11)
    L, R, n = 6, 2, 400
    o = Oracle(L, [1.0, 2.0], field_kind=FIELD_BIMODAL)
    m2 = F = 0.0
    for _ in range(n):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=(R, L ** 3))
        o.set_spins(s)
        m2 += (s[0].astype(np.float64).mean()) ** 2
        F += o.structure_F(0)
    N = L ** 3
    assert N * m2 / n == pytest.approx(1.0, abs=0.15)
    assert F / n == pytest.approx(1.0, abs=0.15)
    xi = oracle.thermal(np.array([[0.0, 0.0, 0.0, m2, 0.0]]), np.array([F]), n, N, np.array([1.0]))[0, 6]
    assert np.isnan(xi) or xi < 0.5


@pytest.mark.parametrize("L", [4, 8, 12])
def test_correlation_length_of_plane_defects_closed_form(L):
    """xi of Sec. 7 from two hand-built lattices measured through the oracle's exchange step
    (frozen spins, both replicas alike so a swap changes nothing).  A: all up but the plane x = 0;
    B: all up but the planes x = 0 and y = 0.  With sum_t e^{iKt} = 0 over a period, by hand:
      A: m = 1 - 2/L, S_x = (-L^2 at t = 0, L^2 else) -> F = |2 L^2|^2 / (3N) = 4L/3;
      B: m = 1 - 2(2L^2 - L)/N, S_x = S_y = (-L^2 at 0, L^2 - 2L else) -> F = 2 (2L(L-1))^2 / (3N).
    xi = sqrt(N <m^2> / <F> - 1) over the two measurements: a dropped root, a dropped -1 or a
    wrong normalisation of F or <m^2> each changes it by far more than the tolerance."""
    N = L ** 3
    o = Oracle(L, [1.0, 2.0], field_kind=FIELD_BIMODAL, h=1.0)
    o.set_measure_xi(True)
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    a = np.where(x == 0, -1, 1).astype(np.int8).reshape(-1)
    b = np.where((x == 0) | (y == 0), -1, 1).astype(np.int8).reshape(-1)
    for s in (a, b):
        o.set_spins(np.stack([s, s]))
        o.exchange(0)
    assert o.n_meas == 2
    mA, mB = 1.0 - 2.0 / L, 1.0 - 2.0 * (2 * L * L - L) / N
    FA, FB = 4.0 * L / 3.0, 2.0 * (2.0 * L * (L - 1)) ** 2 / (3.0 * N)
    want = math.sqrt(N * (mA ** 2 + mB ** 2) / (FA + FB) - 1.0)
    th = oracle.thermal(o.observables(), o.observables_F(), o.n_meas, N, o.temps())
    np.testing.assert_allclose(th[:, 5], 0.5 * (FA + FB), rtol=1e-12)
    np.testing.assert_allclose(th[:, 3], 0.5 * (mA ** 2 + mB ** 2), rtol=1e-12)
    np.testing.assert_allclose(th[:, 6], want, rtol=1e-12)
    assert want > 0.5  # nonzero, so neither the root nor the -1 can be dropped unnoticed


# ------------------------------------------------------------------ multi-hit double checkerboard
@pytest.mark.parametrize("kind", [FIELD_BIMODAL, FIELD_GAUSSIAN])
def test_multihit_single_site_tiles_single_pass_is_the_plain_checkerboard(kind):
    """Tiles of one site and one pass per visit: the coarse colour of a tile is its site's colour,
    so a sweep updates colour 0 then colour 1 with the plain counters (word 2 = sweep)."""
    temps = inputs.geometric_temps(1.0, 5.0, 4)
    a = Oracle(6, temps, h=1.5, field_kind=kind, field_seed=3, seed=11)
    b = Oracle(6, temps, h=1.5, field_kind=kind, field_seed=3, seed=11)
    a.set_multihit(1, 1)
    a.run(12, 3, 1)
    b.run(12, 3, 1)
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.observables(), b.observables())


@pytest.mark.parametrize("tile,mh", [(1, 3), (2, 1), (2, 2), (4, 3)])
def test_multihit_every_site_flips_mh_times_at_infinite_temperature(tile, mh):
    """beta -> 0 (T = 1e30): every attempt is accepted, so after n sweeps every spin has flipped
    n mh times: s = s0 (-1)^(n mh).  Fails if a tile is visited twice or never, or a pass misses a
    fine colour."""
    o = Oracle(8, np.array([1e30, 2e30]), h=1.0, field_kind=FIELD_GAUSSIAN, field_seed=5, seed=2)
    s0 = o.spins().astype(np.int64)
    o.set_multihit(mh, tile)
    for n in (1, 2, 3):
        o.sweep(1)
        np.testing.assert_array_equal(o.spins(), s0 * (-1) ** (n * mh))


@pytest.mark.parametrize("tile,mh", [(2, 3), (4, 2), (1, 4)])
def test_multihit_zero_temperature_matches_numpy_sweep(tile, mh):
    """T -> 0 (T = 1e-30): a flip is accepted iff it does not raise the energy, so the dynamics is
    deterministic; the oracle equals an independent numpy sweep in the tile / pass / colour order
    of the double checkerboard."""
    L = 8
    o = Oracle(L, np.array([1e-30, 2e-30]), J=1.0, h=1.3, field_kind=FIELD_GAUSSIAN, field_seed=8, seed=4)
    _, hh = o.field()
    s = o.spins()
    o.set_multihit(mh, tile)
    changed_after_first_pass = False
    for _ in range(3):
        want = [brute.zero_temperature_multihit_sweep(s[r], L, 1.0, hh, tile, mh) for r in range(2)]
        once = brute.zero_temperature_multihit_sweep(s[0], L, 1.0, hh, tile, 1)
        changed_after_first_pass |= bool((once != want[0]).any())
        o.sweep(1)
        s = o.spins()
        np.testing.assert_array_equal(s, np.stack(want))
    if mh > 1 and tile > 1:
        # the later passes change spins (with single-site tiles they cannot at zero temperature:
        # the neighbours of a site stay frozen during its visit), so the order is tested
        assert changed_after_first_pass


def test_multihit_2x2x2_matches_exact_enumeration():
    """Multi-hit sweeps keep the Boltzmann law: averages over a long chain with three hits per
    visit equal the exact enumeration of the 2x2x2 lattice."""
    L, J, h = 2, 1.0, 1.0
    temps = np.array([1.0, 1.6, 2.6, 4.0])
    o = Oracle(L, temps, J=J, h=h, field_kind=FIELD_BIMODAL, field_seed=6, seed=23)
    o.set_multihit(3, 1)
    _, hh = o.field()
    o.run(200, 1, 10 ** 9)
    mean, err = _binned(o, 20, 3000, 1)
    for k, T in enumerate(temps):
        exact = brute.exact_averages(L, J, hh, 1.0 / T)
        for col in (0, 2, 3):
            assert abs(mean[k, col] - exact[col]) < 5 * err[k, col] + 1e-12, (k, col)


def test_multihit_rejects_tiles_that_do_not_tile_the_lattice():
    o = Oracle(8, np.array([1.0, 2.0]))
    for mh, tile in ((1, 3), (1, 8), (1, 0), (-1, 2)):
        with pytest.raises(ValueError):
            o.set_multihit(mh, tile)
    o.set_multihit(0, 0)

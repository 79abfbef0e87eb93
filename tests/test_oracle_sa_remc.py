"""Pins of the oracle's simulated annealing and replica-exchange Monte Carlo
(SI: Simulated annealing; Replica Exchange Monte Carlo)."""
import math

import numpy as np
import pytest

import goac_synth as synth
import oracle


@pytest.fixture(scope="module")
def tiny():
    prob = synth.tiny_rocksalt_problem()
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    return prob, J


def test_sa_constant_schedule_is_mc(tiny):
    prob, J = tiny
    start = synth.random_population(prob, 3, 2)
    a = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, 0.4, 3000, seed=5)
    b = oracle.sa_run(J, prob.site_class, prob.fixed_q, prob.z, start, 0.4, 0.4, 3000, 3000, seed=5)
    assert np.array_equal(a["species"], b["species"])
    assert np.array_equal(a["n_accept"], b["n_accept"])


def test_sa_anneals_to_ground_state(tiny):
    """Exponential cooling from a hot start to ~0 finds the brute-forced minimum."""
    prob, J = tiny
    emin = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts)["Emin"]
    start = synth.random_population(prob, 16, 3)
    r = oracle.sa_run(J, prob.site_class, prob.fixed_q, prob.z, start, 5.0, 1e-4, 20000, 20000, seed=11)
    assert np.all(r["bestE"] >= emin - 1e-9)
    assert np.mean(np.abs(r["E"] - emin) < 1e-9 * abs(emin)) >= 0.75


def test_remc_single_replica_is_mc(tiny):
    prob, J = tiny
    start = synth.random_population(prob, 4, 6)
    r = oracle.remc_run(J, prob.site_class, prob.fixed_q, prob.z, start, 4, 1, [0.3], 5, 200, seed=8)
    m = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, 0.3, 1000, seed=8)
    assert np.array_equal(r["species"], m["species"])
    assert r["n_exchanges"] == 0 and np.array_equal(r["perm"], np.arange(4))


def test_remc_exchange_acceptance(tiny):
    """No moves (0 steps per round), one exchange attempt per group between a
    low-energy configuration at the cold rank and a high-energy one at the hot
    rank: accepted with probability exp(dE (1/kT0 - 1/kT1)) < 1."""
    prob, J = tiny
    import itertools
    pop = []
    for pos in itertools.combinations(range(8), 4):
        sp = np.zeros(8, dtype=np.int8)
        sp[list(pos)] = 1
        pop.append(sp)
    pop = np.array(pop)
    E = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, pop)
    levels = np.unique(np.round(E, 6))
    lo = pop[int(np.argmin(E))]
    hi = pop[int(np.argmin(np.abs(E - levels[1])))]          # second-lowest level
    G = 4000
    start = np.stack([lo, hi] * G)
    kT = np.array([0.8, 1.6])
    r = oracle.remc_run(J, prob.site_class, prob.fixed_q, prob.z, start, G, 2, kT, 1, 0, seed=21)
    dE = E.min() - E[int(np.argmin(np.abs(E - levels[1])))]
    p = math.exp(dE * (1 / kT[0] - 1 / kT[1]))
    assert 0.05 < p < 0.95
    frac = r["n_exchanges"] / G
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / G)
    perm = r["perm"].reshape(G, 2)
    assert np.all(np.sort(perm, axis=1) == np.arange(G * 2).reshape(G, 2))


def test_gd_reaches_local_minimum(tiny):
    """Every swap from the descent's end point raises the energy (checked by
    fresh q^T J q evaluations); energies never increase; the brute-forced
    ground state is a fixed point."""
    prob, J = tiny
    start = synth.random_population(prob, 6, 14)
    E0 = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, start)
    r = oracle.gd_run(J, prob.site_class, prob.fixed_q, prob.z, start, 100)
    assert np.all(r["E"] <= E0 + 1e-9) and np.all(r["steps"] < 100)
    assert np.allclose(r["E"], oracle.score(J, prob.site_class, prob.fixed_q, prob.z, r["species"]), rtol=1e-12)
    for c in range(6):
        base = r["species"][c]
        Eb = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, base[None])[0]
        for a in range(8):
            for b in range(a + 1, 8):
                if base[a] == base[b]:
                    continue
                t = base.copy()
                t[a], t[b] = base[b], base[a]
                assert oracle.score(J, prob.site_class, prob.fixed_q, prob.z, t[None])[0] >= Eb - 1e-9
    gs = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts, max_argmin=1)["argmin"][0]
    r2 = oracle.gd_run(J, prob.site_class, prob.fixed_q, prob.z, gs[None], 10)
    assert r2["steps"][0] == 0 and np.array_equal(r2["species"][0], gs)


def test_hybrid_is_remc_then_ga(tiny):
    prob, J = tiny
    start = synth.random_population(prob, 8, 31)
    lad = [0.1, 0.3, 0.6, 1.2]
    h = oracle.hybrid_run(J, prob.site_class, prob.fixed_q, prob.z, start, 2, 4, lad, 2, 3, 50, 4, 1, 0.2, seed=5)
    sp = start.copy()
    for c in range(2):
        r = oracle.remc_run(J, prob.site_class, prob.fixed_q, prob.z, sp, 2, 4, lad, 3, 50, seed=5 + 2 * c)
        sp, E = oracle.ga_run(J, prob.site_class, prob.fixed_q, prob.z, r["species"], 4, 1, 0.2, seed=5 + 2 * c + 1,
                              gen0=c * 4)
    assert np.array_equal(h["species"], sp) and np.allclose(h["E"], E, rtol=1e-13)
    emin = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts)["Emin"]
    assert h["E"].min() == pytest.approx(emin, rel=1e-12)

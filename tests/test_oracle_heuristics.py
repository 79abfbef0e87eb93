"""Pins of the oracle's heuristics (SI: Random, Monte Carlo, Genetic
Algorithm) and of the relaxed-occupation gradient and rounding.

The heuristics are stochastic, so they are pinned through properties the
paper's definitions fix: Metropolis sampling reaches the Boltzmann
distribution over brute-forced levels, swaps preserve counts, roulette
selects in proportion to fitness, crossover takes half of the difference
swaps, the random generator is uniform, and the gradient matches finite
differences.
"""
import math
from collections import Counter

import numpy as np
import pytest

import goac_synth as synth
import oracle


@pytest.fixture(scope="module")
def tiny():
    prob = synth.tiny_rocksalt_problem()
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    return prob, J


def _class_counts(prob, sp):
    vclass = prob.site_class[prob.site_class >= 0]
    out = np.zeros((prob.n_class, prob.S), dtype=np.int64)
    for k in range(prob.n_class):
        for s in range(prob.S):
            out[k, s] = int(((vclass == k) & (sp == s)).sum())
    return out


def test_random_configs_counts_and_uniformity():
    prob = synth.layered_problem(reps=(2, 2, 1))
    pop = oracle.random_configs(prob.site_class, prob.counts, 16, seed=99)
    for b in range(16):
        assert np.array_equal(_class_counts(prob, pop[b]), prob.counts)
    # 4 positions holding 2 + 2: six arrangements, each with probability 1/6
    sc = np.array([0, 0, 0, 0], dtype=np.int32)
    B = 60000
    pop = oracle.random_configs(sc, np.array([[2, 2]]), B, seed=5)
    c = Counter(map(bytes, pop))
    assert len(c) == 6
    exp = B / 6
    chi2 = sum((v - exp) ** 2 / exp for v in c.values())
    assert chi2 < 25.0      # 5 dof, p ~ 1e-4


def test_mc_boltzmann_visits(tiny):
    """Single-swap Metropolis with a symmetric proposal samples exp(-E/kT):
    visit frequencies of the brute-forced energy levels must match."""
    prob, J = tiny
    allE = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts, max_all=100)["all_E"]
    kT = 0.5 * float(np.std(allE))
    levels = {}
    for e in allE:
        key = round(e, 6)
        levels[key] = levels.get(key, 0) + 1
    keys = np.array(sorted(levels))
    g = np.array([levels[k] for k in keys], dtype=float)
    w = g * np.exp(-(keys - keys.min()) / kT)
    p_exp = w / w.sum()
    start = synth.random_population(prob, 4, 21)
    res = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, kT, 200000, seed=1234, trace=True)
    tr = res["E_trace"][:, 1000::5].ravel()
    idx = np.searchsorted(keys, np.round(tr, 6))
    assert np.all(keys[idx] == np.round(tr, 6))
    freq = np.bincount(idx, minlength=len(keys)) / tr.size
    big = p_exp > 0.02
    assert np.all(np.abs(freq[big] - p_exp[big]) < 0.1 * p_exp[big] + 0.005)
    # counts preserved and the tracked E equals a fresh evaluation
    for c in range(4):
        assert np.array_equal(_class_counts(prob, res["species"][c]), prob.counts)
    E_fresh = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, res["species"])
    assert np.allclose(res["E"], E_fresh, rtol=1e-12)
    E_best = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, res["best_species"])
    assert np.allclose(res["bestE"], E_best, rtol=1e-12)


def test_mc_zero_temperature_is_descent(tiny):
    prob, J = tiny
    start = synth.random_population(prob, 3, 4)
    res = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, 0.0, 3000, seed=7, trace=True)
    d = np.diff(res["E_trace"], axis=1)
    assert np.all(d <= 1e-12)
    emin = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts)["Emin"]
    assert np.all(res["bestE"] >= emin - 1e-9)


def test_mc_resume_is_exact(tiny):
    """Counter-based draws: 2 x 500 steps equal 1000 steps."""
    prob, J = tiny
    start = synth.random_population(prob, 2, 8)
    a = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, 0.3, 1000, seed=3)
    b1 = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, 0.3, 500, seed=3)
    b2 = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, b1["species"], 0.3, 500, seed=3, step0=500)
    assert np.array_equal(a["species"], b2["species"])


def test_mc_multi_class_counts():
    prob = synth.layered_problem(reps=(2, 2, 1))
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    start = oracle.random_configs(prob.site_class, prob.counts, 3, seed=2)
    res = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, 0.1, 2000, seed=11)
    for c in range(3):
        assert np.array_equal(_class_counts(prob, res["species"][c]), prob.counts)
    assert res["n_accept"].min() > 0


def test_ga_generation_properties():
    prob = synth.layered_problem(reps=(2, 2, 1))
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    P = 512
    pop = oracle.random_configs(prob.site_class, prob.counts, P, seed=17)
    E = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, pop)
    n_elite = 10
    kids, parents, nsw = oracle.ga_generation(prob.site_class, pop, E, n_elite, 0.0, gen=3, seed=42)
    order = np.lexsort((np.arange(P), E))
    assert np.array_equal(kids[:n_elite], pop[order[:n_elite]])
    for c in range(P):
        assert np.array_equal(_class_counts(prob, kids[c]), prob.counts)
    # without mutation, a site where both parents agree keeps that species
    for c in range(n_elite, P):
        A, B = parents[c]
        same = pop[A] == pop[B]
        assert np.array_equal(kids[c][same], pop[A][same])
    # half of the candidate swaps are taken
    taken, cand = nsw[n_elite:, 0].sum(), nsw[n_elite:, 1].sum()
    assert cand > 1000
    assert abs(taken / cand - 0.5) < 4 * 0.5 / math.sqrt(cand)
    # roulette: mean fitness of selected parents = sum F^2 / sum F
    emin, emax = E.min(), E.max()
    F = np.floor((emax - E) / (emax - emin) * 2 ** 24)
    sel = F[parents[n_elite:].ravel()]
    expect = (F ** 2).sum() / F.sum()
    var = (F ** 3).sum() / F.sum() - expect ** 2
    assert abs(sel.mean() - expect) < 4 * math.sqrt(var / sel.size)


def test_ga_mutation_rate():
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    P = 2048
    pop = oracle.random_configs(prob.site_class, prob.counts, P, seed=23)
    E = np.zeros(P)
    # identical parents (all fitness equal) -> children differ from parent only by mutation
    pop[:] = pop[0]
    kids, parents, nsw = oracle.ga_generation(prob.site_class, pop, E, 0, 0.25, gen=0, seed=5)
    changed = np.any(kids != pop, axis=1)
    # a mutation swap of equal species is a no-op: P(change | mutate) = 2*16*16/(32*31)
    p = 0.25 * (2 * 16 * 16) / (32 * 31)
    assert abs(changed.mean() - p) < 4 * math.sqrt(p * (1 - p) / P)


def test_ga_run_improves(tiny):
    prob, J = tiny
    pop = synth.random_population(prob, 32, 3)
    final, E = oracle.ga_run(J, prob.site_class, prob.fixed_q, prob.z, pop, 30, 2, 0.1, seed=9)
    E0 = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, pop)
    assert E.min() <= E0.min() + 1e-12
    emin = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts)["Emin"]
    assert E.min() >= emin - 1e-9
    assert np.allclose(E, oracle.score(J, prob.site_class, prob.fixed_q, prob.z, final), rtol=1e-13)


def _relaxed_problem():
    prob = synth.layered_problem(reps=(1, 1, 1))
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    return prob, J


def test_gradient_finite_differences():
    prob, J = _relaxed_problem()
    rng = np.random.default_rng(4)
    L = rng.standard_normal((prob.Nv, prob.S))
    lam = 0.7
    E, g = oracle.energy_grad(J, prob.site_class, prob.fixed_q, prob.z, prob.counts, L, lam)
    allowed = np.zeros((prob.Nv, prob.S), dtype=bool)
    vclass = prob.site_class[prob.site_class >= 0]
    for v in range(prob.Nv):
        allowed[v] = prob.counts[vclass[v]] > 0
    h = 1e-4
    for v in range(prob.Nv):
        for s in range(prob.S):
            Lp, Lm = L.copy(), L.copy()
            Lp[v, s] += h
            Lm[v, s] -= h
            fd = (oracle.energy_grad(J, prob.site_class, prob.fixed_q, prob.z, prob.counts, Lp, lam)[0]
                  - oracle.energy_grad(J, prob.site_class, prob.fixed_q, prob.z, prob.counts, Lm, lam)[0]) / (2 * h)
            if not allowed[v, s]:
                assert g[v, s] == 0.0 and abs(fd) < 1e-9
            else:
                assert g[v, s] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(g).max())


def test_gradient_one_hot_limit():
    """Sharp logits: p is one-hot, q equals the configuration's charges and
    E equals q^T J q (the counts penalty vanishes at exact counts)."""
    prob, J = _relaxed_problem()
    sp = oracle.random_configs(prob.site_class, prob.counts, 1, seed=1)[0]
    L = np.full((prob.Nv, prob.S), -60.0)
    L[np.arange(prob.Nv), sp] = 60.0
    E, g = oracle.energy_grad(J, prob.site_class, prob.fixed_q, prob.z, prob.counts, L, 1.0)
    E_ref = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, sp[None])[0]
    assert E == pytest.approx(E_ref, rel=1e-12)
    assert np.abs(g).max() < 1e-40


def test_round_to_counts():
    prob = synth.layered_problem(reps=(2, 2, 1))
    sp = oracle.random_configs(prob.site_class, prob.counts, 1, seed=31)[0]
    onehot = np.zeros((prob.Nv, prob.S), dtype=np.float32)
    onehot[np.arange(prob.Nv), sp] = 1.0
    assert np.array_equal(oracle.round_to_counts(prob.site_class, prob.counts, onehot), sp)
    rng = np.random.default_rng(3)
    p = rng.dirichlet(np.ones(prob.S), size=prob.Nv).astype(np.float32)
    out = oracle.round_to_counts(prob.site_class, prob.counts, p)
    assert np.array_equal(_class_counts(prob, out), prob.counts)
    # the globally largest allowed p is always honoured
    vclass = prob.site_class[prob.site_class >= 0]
    masked = np.where(prob.counts[vclass] > 0, p, -1)
    v, s = np.unravel_index(np.argmax(masked), masked.shape)
    assert out[v] == s


def test_round_to_counts_bruteforce_small():
    """On tiny inputs the greedy rule equals an explicit brute-force search
    for the lexicographically greatest sorted assignment."""
    import itertools
    rng = np.random.default_rng(8)
    sc = np.zeros(5, dtype=np.int32)
    counts = np.array([[2, 3]], dtype=np.int32)
    for _ in range(20):
        p = rng.uniform(0, 1, (5, 2)).astype(np.float32)
        out = oracle.round_to_counts(sc, counts, p)
        best = None
        for pos in itertools.combinations(range(5), 2):
            sp = np.ones(5, dtype=np.int8)
            sp[list(pos)] = 0
            key = sorted([float(p[v, sp[v]]) for v in range(5)], reverse=True)
            if best is None or key > best[0]:
                best = (key, sp)
        assert np.array_equal(out, best[1])

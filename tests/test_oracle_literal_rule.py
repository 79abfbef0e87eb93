"""The oracle's Metropolis and descent rules against the paper's rules taken
literally (SI, Monte Carlo: accept with probability min[1, exp(-dE/kT)];
SI, Gradient Descent: take the lowest neighbour while it is lower).

orc_mc_run reads |dE| <= 1e-9 eV as dE = 0 (accepted), tests the event
u < exp(-dE/kT) as dE < -kT ln u, and updates phi with one fma.  Its twin
orc_mc_run_literal accepts iff dE <= 0 or u < exp(-dE/kT) and updates phi with
a separately rounded product and sum.  On the workloads the GPU parity tests
use, and at every kT > 0, the two take the same decision at every step
(identical configurations, acceptance counts and energies), although hundreds
of proposals fall in the tie band; no proposal lies within 1e-9 of the exp/log
boundary.  At kT = 0 the literal rule rejects symmetric swaps whose dE is
+1e-14 eV of rounding and accepts their -1e-14 eV mirror images, so its
trajectory follows rounding noise: that case is where the band is needed.

orc_gd_run takes the lowest pair within 1e-9 eV of the minimum and stops once
no swap lowers E by more than 1e-9 eV; orc_gd_run_literal takes the exact
argmin and stops at dE >= 0.  From every configuration of the brute-forced
1x1x2 cell both end at the same energy, and from random starts of the 2x2x2
rocksalt cell both reach the exhaustively enumerated ground state."""
import itertools
import os

import numpy as np
import pytest

import goac_synth as synth
import oracle

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rocksalt222_ground_state.txt")


def _J(prob):
    return oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)


@pytest.mark.parametrize("cell,C,steps,kT,seed,step0", [
    ("rocksalt222", 8, 20000, 0.05, 0x600AC, 0),     # the 2x2x2 rocksalt parity workload
    ("layered221", 5, 6000, 0.1, 77, 123),            # the multi-class parity workload
    ("layered221", 8, 20000, 0.05, 0x600AC, 0),
    ("layered221", 8, 20000, 0.002, 0x600AD, 0),      # the coldest temperature of the annealing runs
])
def test_mc_rule_equals_literal_metropolis(cell, C, steps, kT, seed, step0):
    prob = synth.rocksalt_problem((2, 2, 2), 4.2) if cell == "rocksalt222" else synth.layered_problem(reps=(2, 2, 1))
    J = _J(prob)
    start = synth.random_population(prob, C, 5)
    a = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, kT, steps, seed, step0=step0)
    b = oracle.mc_run_literal(J, prob.site_class, prob.fixed_q, prob.z, start, kT, steps, seed, step0=step0)
    assert np.array_equal(a["species"], b["species"])
    assert np.array_equal(a["n_accept"], b["n_accept"])
    assert np.array_equal(a["E"], b["E"]) and np.array_equal(a["bestE"], b["bestE"])
    assert b["n_close"].sum() == 0
    assert b["n_band"].sum() > 0          # the band was exercised, and decided as the literal rule did
    assert a["n_accept"].sum() > 0


def test_mc_rules_part_at_zero_temperature():
    """kT = 0: the literal rule takes symmetric swaps by the sign of their
    rounding error, so the trajectories part (the reason for the band)."""
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    J = _J(prob)
    start = synth.random_population(prob, 8, 5)
    a = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, 0.0, 20000, 0x600AC)
    b = oracle.mc_run_literal(J, prob.site_class, prob.fixed_q, prob.z, start, 0.0, 20000, 0x600AC)
    assert b["n_band"].sum() > 0
    assert not np.array_equal(a["species"], b["species"])


def test_literal_twin_samples_boltzmann():
    """The twin is pinned by its own definition: on the brute-forced 1x1x2
    cell its visit frequencies of the energy levels follow exp(-E/kT)."""
    prob = synth.tiny_rocksalt_problem()
    J = _J(prob)
    res = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts, max_all=100)
    allE = np.sort(res["all_E"])
    kT = 0.5 * float(np.std(allE))
    start = synth.random_population(prob, 1, 1)
    steps = 200000
    # the energy after every step, from the twin's state at step prefixes of one long run
    n_blocks, blk = 200, steps // 200
    visits = []
    sp = start
    for r in range(n_blocks):
        out = oracle.mc_run_literal(J, prob.site_class, prob.fixed_q, prob.z, sp, kT, blk, 17, step0=r * blk)
        sp = out["species"]
        visits.append(out["E"][0])
    visits = np.array(visits)
    levels = np.unique(np.round(allE, 6))
    w = np.array([np.sum(np.isclose(allE, e, atol=1e-6)) * np.exp(-(e - allE[0]) / kT) for e in levels])
    p = w / w.sum()
    obs = np.array([np.sum(np.isclose(visits, e, atol=1e-6)) for e in levels])
    assert obs.sum() == n_blocks
    keep = p * n_blocks >= 5
    exp_ = p[keep] * n_blocks
    chi2 = (((obs[keep] - exp_) ** 2) / exp_).sum() + ((obs[~keep].sum() - (p[~keep] * n_blocks).sum()) ** 2
                                                        / max((p[~keep] * n_blocks).sum(), 1e-9))
    assert chi2 < 30.0


def _all_halves(nv):
    out = []
    for comb in itertools.combinations(range(nv), nv // 2):
        s = np.zeros(nv, np.int8)
        s[list(comb)] = 1
        out.append(s)
    return np.array(out)


def _is_local_min(J, prob, sp, E):
    """Every same-class swap, rescored from scratch, lowers E by at most 1e-9 eV."""
    vclass = prob.site_class[prob.site_class >= 0]
    cand = []
    for a in range(sp.size):
        for b in range(a + 1, sp.size):
            if vclass[a] == vclass[b] and sp[a] != sp[b]:
                t = sp.copy()
                t[a], t[b] = t[b], t[a]
                cand.append(t)
    Es = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, np.array(cand))
    return Es.min() >= E - 1e-9


def test_gd_band_changes_no_end_energy_on_brute_forced_cell():
    prob = synth.tiny_rocksalt_problem()
    J = _J(prob)
    pop = _all_halves(prob.Nv)
    assert pop.shape[0] == 70
    a = oracle.gd_run(J, prob.site_class, prob.fixed_q, prob.z, pop, 1000)
    b = oracle.gd_run_literal(J, prob.site_class, prob.fixed_q, prob.z, pop, 1000)
    assert np.all(np.abs(a["E"] - b["E"]) <= 1e-9)
    assert np.array_equal(a["steps"], b["steps"])
    Emin = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts)["Emin"]
    assert abs(a["E"].min() - Emin) <= 1e-9 and abs(b["E"].min() - Emin) <= 1e-9
    for r in range(70):
        assert _is_local_min(J, prob, b["species"][r], b["E"][r])
        assert _is_local_min(J, prob, a["species"][r], a["E"][r])


def test_gd_band_reaches_the_exhaustive_ground_state():
    """2x2x2 rocksalt cell (32 cations, 16 + 16): from 256 random starts the
    banded and the literal descent both reach the enumerated minimum."""
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    J = _J(prob)
    E_gold = None
    for line in open(GOLD):
        if line.startswith("E_min_eV"):
            E_gold = float(line.split()[1])
    assert E_gold is not None
    pop = synth.random_population(prob, 256, 3)
    a = oracle.gd_run(J, prob.site_class, prob.fixed_q, prob.z, pop, 1000)
    b = oracle.gd_run_literal(J, prob.site_class, prob.fixed_q, prob.z, pop, 1000)
    assert abs(a["E"].min() - E_gold) <= 1e-9 * abs(E_gold)
    assert abs(b["E"].min() - E_gold) <= 1e-9 * abs(E_gold)
    same = np.abs(a["E"] - b["E"]) <= 1e-9
    assert same.mean() >= 0.9

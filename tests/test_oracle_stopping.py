"""Pins of the oracle's run-level stops and statistics (Section "Internal
Fortran Heuristics in GOAC": a run ends after a number of steps or
generations, or of steps or generations without improvement).

The statistics and the stop point are recomputed here from the definition,
by replaying the run one step (or one generation) at a time through the plain
entry points, whose resumption is itself pinned: the pair each step proposes
comes from the published Philox4x32-10 (pinned by its known-answer vectors)
and the multiply-high map, no-ops are the steps whose pair holds one species,
and the stop is the first step t with t - t_imp >= patience."""
import numpy as np
import pytest

import goac_synth as synth
import oracle


def _J(prob):
    return oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)


def _pair(seed, t, chain, n):
    x = oracle.philox4x32_10([t & 0xFFFFFFFF, t >> 32, chain, 0], [seed & 0xFFFFFFFF, seed >> 32])
    a = (int(x[0]) * n) >> 32
    bb = (int(x[1]) * (n - 1)) >> 32
    return a, bb + (bb >= a)


def _replay(J, prob, start, kT, nsteps, seed):
    """Per chain: whether each step's pair held one species (single movable
    class; the species before every step by running the chain one step at a
    time), and the energy after every step as the run tracks it (its trace of
    the energy before each step, shifted by one)."""
    pos = np.nonzero(prob.site_class[prob.site_class >= 0] == 0)[0]
    full = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, kT, nsteps, seed, trace=True)
    out = []
    for c in range(start.shape[0]):
        sp = start[c:c + 1].copy()
        noop = []
        for t in range(nsteps):
            a, b = _pair(seed, t, c, pos.size)
            noop.append(sp[0, pos[a]] == sp[0, pos[b]])
            # chain index c (the draw counter): pad with copies in front
            block = np.repeat(sp, c + 1, axis=0)
            r = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, block, kT, 1, seed, step0=t)
            sp = r["species"][c:c + 1]
        assert np.array_equal(sp[0], full["species"][c])
        E_after = np.append(full["E_trace"][c, 1:], full["E"][c])
        out.append((np.array(noop), E_after))
    return out


def test_mc_statistics_and_patience_from_replay():
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    J = _J(prob)
    start = synth.random_population(prob, 3, 5)
    kT, nsteps, seed, patience = 0.05, 1500, 0x600AC, 150
    E0 = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, start)
    full = oracle.mc_run_ex(J, prob.site_class, prob.fixed_q, prob.z, start, kT, nsteps, seed, patience=0)
    plain = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start, kT, nsteps, seed)
    assert np.array_equal(full["species"], plain["species"]) and np.array_equal(full["n_accept"], plain["n_accept"])
    assert np.all(full["steps_done"] == nsteps)
    stop = oracle.mc_run_ex(J, prob.site_class, prob.fixed_q, prob.z, start, kT, nsteps, seed, patience=patience)
    rep = _replay(J, prob, start, kT, nsteps, seed)
    for c, (noop, E_after) in enumerate(rep):
        assert full["n_noop"][c] == noop.sum()
        # best step: the last step whose energy undercut every earlier one (and the start) by more than
        # the 1e-9 eV tie
        run_min, t_best = E0[c], -1
        for t, e in enumerate(E_after):
            if e < run_min - 1e-9:
                run_min, t_best = e, t
        assert full["best_step"][c] == t_best and full["bestE"][c] == run_min
        # patience: improvements by more than 1e-9 eV; stop after the first t with t - t_imp >= patience
        E_imp, t_imp, done = E0[c], -1, nsteps
        for t, e in enumerate(E_after):
            if e < E_imp - 1e-9:
                E_imp, t_imp = e, t
            if t - t_imp >= patience:
                done = t + 1
                break
        assert done < nsteps                    # the rule stopped this chain
        assert stop["steps_done"][c] == done
        assert stop["n_noop"][c] == noop[:done].sum()
        assert stop["E"][c] == E_after[done - 1]
    # the stopped chains are the plain chains run for their own number of steps
    for c in range(3):
        r = oracle.mc_run(J, prob.site_class, prob.fixed_q, prob.z, start[:c + 1], kT, int(stop["steps_done"][c]), seed)
        assert np.array_equal(r["species"][c], stop["species"][c])


def test_ga_patience_from_replay():
    prob = synth.layered_problem(reps=(2, 2, 1))
    J = _J(prob)
    pop0 = synth.random_population(prob, 64, 8)
    patience = 4
    fin, E, gens, best_gen, stopped = oracle.ga_run_ex(J, prob.site_class, prob.fixed_q, prob.z, pop0, 60, 2, 0.1, 5,
                                                       patience=patience)
    # one generation at a time (a GA run resumes from its population and generation number)
    pop = pop0.copy()
    Eg = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, pop)
    b_ref, stall, want_best, want_gens = Eg.min(), 0, 0, 60
    for g in range(1, 61):
        pop, Eg = oracle.ga_run(J, prob.site_class, prob.fixed_q, prob.z, pop, 1, 2, 0.1, seed=5, gen0=g - 1)
        if Eg.min() < b_ref - 1e-9:
            b_ref, stall, want_best = Eg.min(), 0, g
        else:
            stall += 1
        if stall >= patience:
            want_gens = g
            break
    assert stopped and gens == want_gens < 60 and best_gen == want_best
    assert np.array_equal(fin, pop) and np.array_equal(E, Eg)
    # no patience: the plain run
    fin0, E0, g0, _, st0 = oracle.ga_run_ex(J, prob.site_class, prob.fixed_q, prob.z, pop0, 7, 2, 0.1, 5)
    ref, Eref = oracle.ga_run(J, prob.site_class, prob.fixed_q, prob.z, pop0, 7, 2, 0.1, seed=5)
    assert g0 == 7 and not st0 and np.array_equal(fin0, ref) and np.array_equal(E0, Eref)

"""Pins of the oracle's configuration energies: Eq. 2 cluster expansion,
fixed-site split, single-swap energy change, brute force and Eq. 1 counts."""
import math
import os

import numpy as np
import pytest

import goac_synth as synth
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tiny():
    prob = synth.tiny_rocksalt_problem()
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    return prob, J


def test_score_equals_direct_ewald(tiny):
    prob, J = tiny
    pop = synth.random_population(prob, 6, 11)
    E = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, pop)
    for b in range(pop.shape[0]):
        q = oracle.config_charges(prob.site_class, prob.fixed_q, prob.z, pop[b])
        Ed = oracle.ewald_energy(prob.lattice, prob.frac, q, prob.alpha, prob.nimg, prob.kcut)
        assert E[b] == pytest.approx(Ed, rel=1e-12)


def test_fixed_split(tiny):
    prob, J = tiny
    phi_fix, E_const = oracle.fixed_split(J, prob.site_class, prob.fixed_q)
    pop = synth.random_population(prob, 4, 12)
    E = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, pop)
    vidx = np.nonzero(prob.site_class >= 0)[0]
    Jvv = J[np.ix_(vidx, vidx)]
    for b in range(4):
        qv = prob.z[pop[b]]
        e = qv @ Jvv @ qv + 2 * qv @ phi_fix + E_const
        assert e == pytest.approx(E[b], rel=1e-13)


def test_eq2_cluster_expansion(tiny):
    """Eq. 2 with coefficients from sub-structure Ewald energies (as the paper
    builds them) equals the direct Ewald energy, and equals the coefficients
    read off J: the second-order expansion is exact for point charges."""
    prob, J = tiny
    ec_j, al_j, be_j = oracle.ce_from_J(J, prob.site_class, prob.fixed_q, prob.z)
    ec_s, al_s, be_s = oracle.ce_from_substructures(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut,
                                                     prob.site_class, prob.fixed_q, prob.z)
    scale = abs(ec_j)
    assert ec_s == pytest.approx(ec_j, rel=1e-12)
    assert np.max(np.abs(al_s - al_j)) <= 1e-11 * scale
    assert np.max(np.abs(be_s - be_j)) <= 1e-11 * scale
    pop = synth.random_population(prob, 5, 13)
    for b in range(5):
        q = oracle.config_charges(prob.site_class, prob.fixed_q, prob.z, pop[b])
        Ed = oracle.ewald_energy(prob.lattice, prob.frac, q, prob.alpha, prob.nimg, prob.kcut)
        e2 = oracle.ce_energy(prob.Nv, prob.S, ec_s, al_s, be_s, pop[b])
        assert e2 == pytest.approx(Ed, rel=1e-11)


def test_delta_E_identity():
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    rng = np.random.default_rng(5)
    pop = synth.random_population(prob, 1, 6)[0]
    vidx = np.nonzero(prob.site_class >= 0)[0]
    E0 = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, pop[None])[0]
    q = oracle.config_charges(prob.site_class, prob.fixed_q, prob.z, pop)
    phi = J @ q
    for _ in range(40):
        a, b = rng.choice(prob.Nv, 2, replace=False)
        after = pop.copy()
        after[a], after[b] = pop[b], pop[a]
        E1 = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, after[None])[0]
        dE = oracle.delta_E(J, phi, vidx[a], vidx[b], prob.z[pop[a]], prob.z[pop[b]])
        assert dE == pytest.approx(E1 - E0, abs=1e-10 * abs(E0))


def test_brute_force_tiny(tiny):
    """1x1x2 rocksalt cell, 8 cations 4 x +1 / 4 x +3: C(8,4) = 70 configs.
    The minimum from the enumeration equals the minimum of independent direct
    Ewald energies of every configuration."""
    prob, J = tiny
    res = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts, max_all=100)
    assert res["n_configs"] == math.comb(8, 4)
    assert 10 ** oracle.log10_configurations([8], [[4, 4]]) == pytest.approx(70, rel=1e-12)
    # enumerate the 70 independently (itertools) with the direct Ewald energy
    import itertools
    direct = []
    for pos in itertools.combinations(range(8), 4):
        sp = np.zeros(8, dtype=np.int8)
        sp[list(pos)] = 1
        q = oracle.config_charges(prob.site_class, prob.fixed_q, prob.z, sp)
        direct.append(oracle.ewald_energy(prob.lattice, prob.frac, q, prob.alpha, prob.nimg, prob.kcut))
    direct = np.array(direct)
    assert res["Emin"] == pytest.approx(direct.min(), rel=1e-12)
    assert np.allclose(np.sort(res["all_E"]), np.sort(direct), rtol=1e-12)
    n_min = int((np.abs(direct - direct.min()) <= 1e-9 * abs(direct.min())).sum())
    assert res["n_argmin"] == n_min


def _gold_nconf():
    rows, single = [], []
    for line in open(os.path.join(GOLD, "table1_nconf.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = line.split()
        if w[0] == "single":
            single.append((w[1], int(w[2]), [int(x) for x in w[3].split(",")], int(w[4])))
        else:
            rows.append((w[0], int(w[1]), int(w[2])))
    return rows, single


def test_eq1_counts_table1():
    rows, single = _gold_nconf()
    assert len(rows) == 8
    for _name, n, expo in rows:
        na = [6 * n, 3 * n] + [0] * 5
        h = 3 * n // 2
        tm = [0, 0, h, h, h, h, 3 * n]
        l10 = oracle.log10_configurations([9 * n, 9 * n], [na, tm])
        assert round(l10) == expo
    for _name, pos, cnt, expo in single:
        assert round(oracle.log10_configurations([pos], [cnt])) == expo


def test_enumeration_count_two_classes():
    """Eq. 1 for two classes equals the number of enumerated configurations."""
    prob = synth.tiny_rocksalt_problem()
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    sc = prob.site_class.copy()
    cat = np.nonzero(sc >= 0)[0]
    an = np.nonzero(sc < 0)[0]
    sc[an[:4]] = 1
    z = np.array([1.0, 3.0, -2.0, -1.0])
    counts = np.array([[4, 4, 0, 0], [0, 0, 2, 2]], dtype=np.int32)
    fq = np.where(sc < 0, -2.0, 0.0)
    # neutralise: anion class carries -2 -2 -1 -1 = -6 instead of -8 -> adjust fixed
    fq[an[4]] = -2.0
    res = oracle.enumerate_all(J, sc, fq, z, counts, max_all=0)
    assert res["n_configs"] == math.comb(8, 4) * math.comb(4, 2)
    assert cat.shape[0] == 8

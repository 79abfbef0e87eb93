"""Exhaustive ground states (brute force) as pins: the two-species
enumeration against the generic multiset enumeration on small cells, and the
stored ground state of the rocksalt 2x2x2 cation problem (601,080,390
configurations, tests/golden/rocksalt222_ground_state.txt) re-checked by
scoring."""
import math
import os

import numpy as np
import pytest

import goac_synth as synth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rocksalt222_ground_state.txt")


def _two_species_cell(n_pos, k, seed):
    """Random cell: one class of n_pos positions holding (n_pos - k) x +1 and
    k x +3, neutralised by fixed anions at -2."""
    rng = np.random.default_rng(seed)
    n_an = (n_pos - k + 3 * k) // 2
    N = n_pos + n_an
    A = np.diag([6.0, 6.5, 7.0]) + rng.uniform(-0.5, 0.5, (3, 3))
    frac = rng.uniform(0, 1, (N, 3))
    site_class = np.array([0] * n_pos + [-1] * n_an, dtype=np.int32)
    fixed_q = np.array([0.0] * n_pos + [-2.0] * n_an)
    p = synth.Problem(name="two", lattice=A, frac=frac, site_class=site_class, fixed_q=fixed_q,
                      z=np.array([1.0, 3.0]), counts=np.array([[n_pos - k, k]], np.int32), alpha=0.0,
                      nimg=(0, 0, 0), kcut=0.0)
    p.alpha, p.nimg, p.kcut = synth.default_cutoffs(A)
    return p


@pytest.mark.parametrize("n_pos,k,seed", [(8, 4, 1), (10, 2, 2), (12, 6, 3), (13, 5, 4)])
def test_two_species_enumeration_matches_brute_force(n_pos, k, seed):
    prob = _two_species_cell(n_pos, k, seed)
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    a = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts)
    b = oracle.enumerate_two_species(J, prob.site_class, prob.fixed_q, prob.z, prob.counts)
    assert a["n_configs"] == b["n_configs"] == math.comb(n_pos, k)
    assert b["Emin"] == pytest.approx(a["Emin"], rel=1e-12, abs=1e-12)
    assert a["n_argmin"] == b["n_argmin"]
    assert sorted(map(tuple, a["argmin"].tolist())) == sorted(map(tuple, b["argmin"].tolist()))


def test_tiny_rocksalt_two_species_enumeration():
    prob = synth.tiny_rocksalt_problem()
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    a = oracle.enumerate_all(J, prob.site_class, prob.fixed_q, prob.z, prob.counts)
    b = oracle.enumerate_two_species(J, prob.site_class, prob.fixed_q, prob.z, prob.counts)
    assert b["n_configs"] == 70 and b["Emin"] == pytest.approx(a["Emin"], rel=1e-12)
    assert sorted(map(tuple, a["argmin"].tolist())) == sorted(map(tuple, b["argmin"].tolist()))


def read_golden():
    vals, arg = {}, []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        key, val = line.split()
        if key == "argmin":
            arg.append([int(c) for c in val])
        else:
            vals[key] = float(val)
    return vals, np.array(arg, dtype=np.int8)


def test_rocksalt222_ground_state_file():
    """Every stored minimiser scores E_min, keeps the counts, and no single swap
    from it lowers the energy; the count is C(32, 16)."""
    vals, arg = read_golden()
    assert int(vals["n_configs"]) == math.comb(32, 16)
    assert len(arg) == int(vals["n_argmin"]) > 0
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    E = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, arg)
    assert np.allclose(E, vals["E_min_eV"], rtol=0, atol=1e-9)
    assert np.all(arg.sum(axis=1) == 16)
    sp = arg[0]
    swapped = []
    for a in np.nonzero(sp == 1)[0]:
        for b in np.nonzero(sp == 0)[0]:
            t = sp.copy()
            t[a], t[b] = 0, 1
            swapped.append(t)
    Es = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, np.array(swapped))
    assert Es.min() >= vals["E_min_eV"] - 1e-9
    rnd = synth.random_population(prob, 2000, 11)
    assert oracle.score(J, prob.site_class, prob.fixed_q, prob.z, rnd).min() > vals["E_min_eV"]

"""Pins of the oracle's Ewald pair matrix J and direct Ewald energy.

Each test checks the oracle against something other than itself: textbook
Madelung constants (the paper prints the rocksalt one, Eq. 3), the exact
alpha-independence of the Ewald split, symmetry / translation invariance, and
an independent structure-factor evaluation of the energy.
"""
import math
import os

import numpy as np
import pytest

import goac_synth as synth
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _madelung_table():
    rows = {}
    for line in open(os.path.join(GOLD, "madelung.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, r0a, m = line.split()
        rows[name] = (float(r0a), float(m))
    return rows


def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = oracle.philox4x32_10(w[0:4], w[4:6])
        assert [int(x) for x in out] == w[6:10]


def test_geometry_reciprocal_basis():
    rng = np.random.default_rng(1)
    A = np.eye(3) * 4.0 + rng.uniform(-0.5, 0.5, (3, 3))
    B, V = oracle.cell_geometry(A)
    assert np.allclose(A @ B.T, 2 * math.pi * np.eye(3), atol=1e-12)
    assert V == pytest.approx(abs(np.linalg.det(A)), rel=1e-14)
    lat, frac, _ = synth.layered_problem().lattice, synth.layered_problem().frac, None
    cart = oracle.frac_to_cart(lat, frac[:10])
    assert np.allclose(cart, frac[:10] @ lat, atol=1e-12)


@pytest.mark.parametrize("structure", ["rocksalt", "cscl", "zincblende"])
def test_madelung_constants(structure):
    r0a, M_ref = _madelung_table()[structure]
    a = 5.62 if structure == "rocksalt" else 3.0
    cell = {"rocksalt": synth.rocksalt_cell((1, 1, 1), a), "cscl": synth.cscl_cell(a),
            "zincblende": synth.zincblende_cell(a)}[structure]
    lat, frac, is_anion = cell
    q = np.where(is_anion, -1.0, 1.0)
    alpha, kcut = 5.0 / a, 8 * 2 * math.pi / a
    J = oracle.ewald_J(lat, frac, alpha, (3, 3, 3), kcut)
    E = oracle.qJq(J, q)
    r0 = r0a * a
    M = abs(E) * r0 / ((len(q) / 2) * oracle.KE)
    assert M == pytest.approx(M_ref, rel=1e-9)
    # charge scaling +-z gives z^2 times the energy
    Ez = oracle.qJq(J, 2.0 * q)
    assert Ez == pytest.approx(4.0 * E, rel=1e-13)
    # the structure-factor evaluation, independent of J, agrees
    Ed = oracle.ewald_energy(lat, frac, q, alpha, (3, 3, 3), kcut)
    assert Ed == pytest.approx(E, rel=1e-12)


def test_nacl_3x3x3_closed_form():
    """Paper's NaCl benchmark: 216 ions, r = 2.81 A; perfect alternation has
    E = -(N/2) M ke / r (Eq. 3 solved for E)."""
    lat, frac, is_anion = synth.rocksalt_cell((3, 3, 3), 5.62)
    q = np.where(is_anion, -1.0, 1.0)
    L = 3 * 5.62
    E = oracle.ewald_energy(lat, frac, q, 5.0 / L, (2, 2, 2), 8 * 2 * math.pi / L)
    M_ref = _madelung_table()["rocksalt"][1]
    assert E == pytest.approx(-108 * M_ref * oracle.KE / 2.81, rel=1e-9)


def _random_cell(n, seed):
    rng = np.random.default_rng(seed)
    A = np.diag([6.0, 6.5, 7.0]) + rng.uniform(-0.6, 0.6, (3, 3))
    frac = rng.uniform(0, 1, (n, 3))
    return A, frac


def test_alpha_independence():
    A, frac = _random_cell(12, 7)
    L = abs(np.linalg.det(A)) ** (1 / 3)
    a1 = 5.0 / L
    a2 = 1.3 * a1
    J1 = oracle.ewald_J(A, frac, a1, (4, 4, 4), 14 * a1)
    J2 = oracle.ewald_J(A, frac, a2, (4, 4, 4), 14 * a2)
    assert np.max(np.abs(J1 - J2)) <= 1e-10 * np.max(np.abs(J1))


def test_symmetry_and_translation():
    A, frac = _random_cell(10, 3)
    L = abs(np.linalg.det(A)) ** (1 / 3)
    J = oracle.ewald_J(A, frac, 5.0 / L, (3, 3, 3), 60.0 / L)
    assert np.max(np.abs(J - J.T)) <= 1e-13 * np.max(np.abs(J))
    Js = oracle.ewald_J(A, (frac + np.array([0.137, 0.71, 0.29])) % 1.0, 5.0 / L, (3, 3, 3), 60.0 / L)
    assert np.max(np.abs(J - Js)) <= 1e-12 * np.max(np.abs(J))


def test_entries_match_full_matrix():
    A, frac = _random_cell(9, 5)
    L = abs(np.linalg.det(A)) ** (1 / 3)
    J = oracle.ewald_J(A, frac, 5.0 / L, (3, 3, 3), 60.0 / L)
    pairs = np.array([[0, 0], [1, 5], [8, 2], [4, 4]])
    e = oracle.ewald_J_entries(A, frac, 5.0 / L, (3, 3, 3), 60.0 / L, pairs)
    assert np.array_equal(e, J[pairs[:, 0], pairs[:, 1]])


def test_direct_energy_matches_quadratic_form():
    """Random non-neutral charges: the neutralising background makes both
    sides defined and they must agree."""
    A, frac = _random_cell(14, 11)
    L = abs(np.linalg.det(A)) ** (1 / 3)
    rng = np.random.default_rng(2)
    for neutral in (True, False):
        q = rng.integers(-3, 4, 14).astype(float)
        if neutral:
            q[-1] -= q.sum()
        J = oracle.ewald_J(A, frac, 5.0 / L, (3, 3, 3), 60.0 / L)
        E1 = oracle.qJq(J, q)
        E2 = oracle.ewald_energy(A, frac, q, 5.0 / L, (3, 3, 3), 60.0 / L)
        assert E1 == pytest.approx(E2, rel=1e-12, abs=1e-11)


def test_neutral_shift_invariance():
    """J + c 11^T leaves every neutral energy unchanged; J + c I shifts it by
    c sum q^2 (fixed counts => a constant)."""
    prob = synth.tiny_rocksalt_problem()
    J = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    pop = synth.random_population(prob, 5, 3)
    E = oracle.score(J, prob.site_class, prob.fixed_q, prob.z, pop)
    E1 = oracle.score(J + 0.37, prob.site_class, prob.fixed_q, prob.z, pop)
    assert np.allclose(E, E1, rtol=1e-12, atol=1e-10)
    E2 = oracle.score(J + 0.5 * np.eye(prob.N), prob.site_class, prob.fixed_q, prob.z, pop)
    q2 = (prob.fixed_q ** 2).sum() + (prob.counts[0] * prob.z ** 2).sum()
    assert np.allclose(E2 - E, 0.5 * q2, rtol=1e-12)

"""The seeded synthetic workloads have the sizes, counts and charges their
recipe states (the inputs both sides of every parity test are built from)."""
import numpy as np
import pytest

import goac_synth as synth


def _total_charge(p):
    return float(p.fixed_q[p.site_class < 0].sum() + (p.counts @ p.z).sum())


def _check_common(p):
    vclass = p.site_class[p.site_class >= 0]
    for k in range(p.n_class):
        assert int(p.counts[k].sum()) == int((vclass == k).sum())
    assert np.all(p.frac >= 0.0) and np.all(p.frac < 1.0)
    assert p.alpha > 0 and p.kcut > 0 and all(n >= 1 for n in p.nimg)


def test_rocksalt_parity_cell():
    p = synth.rocksalt_problem((2, 2, 2), 4.2)
    _check_common(p)
    assert p.N == 64 and p.Nv == 32
    assert np.all(p.fixed_q[p.site_class < 0] == -2.0)
    assert sorted(zip(p.z.tolist(), p.counts[0].tolist())) == [(1.0, 16), (3.0, 16)]
    assert abs(_total_charge(p)) < 1e-12
    assert np.allclose(np.diag(p.lattice), 8.4)


def test_layered_r3m_cell():
    """12x12x1 R-3m: 432 O (the +z member of each 6c pair) carrying the
    neutralising charge, Li 346 / vacancy 86, Ni2+/Ni3+/Mn4+/Co3+ 108 each."""
    p = synth.layered_problem()
    _check_common(p)
    assert p.N == 1296 and p.Nv == 864
    qo = p.fixed_q[p.site_class < 0]
    assert qo.size == 432 and np.allclose(qo, -(346 + 1296) / 432)
    li, tm = p.counts
    assert (li[0], li[1]) == (346, 86) and list(tm[2:6]) == [108, 108, 108, 108]
    assert abs(_total_charge(p)) < 1e-9


def test_random_cubic_benchmark_cell():
    p = synth.random_cubic_problem()
    _check_common(p)
    assert p.N == p.Nv == 4096
    assert list(p.counts[0]) == [512, 1024, 512, 2048] and list(p.z) == [1.0, 2.0, 3.0, -2.0]
    assert abs(_total_charge(p)) < 1e-12
    assert np.allclose(np.diag(p.lattice), 40.0)
    again = synth.random_cubic_problem()
    assert np.array_equal(again.frac, p.frac)          # seeded


def test_bcc_relaxed_cell():
    p = synth.bcc_relaxed_problem()
    _check_common(p)
    assert p.N == p.Nv == 8192 and list(p.z) == [1.0, 2.0, 3.0, 4.0, 0.0]
    assert sorted(p.counts[0].tolist()) == [1638, 1638, 1638, 1639, 1639]


def test_batch_cells():
    """Targets log-uniform in [64, 2048], each realised as the nearest rocksalt
    (8 abc sites) or spinel (56 abc sites) supercell."""
    cells = synth.batch_problems(256)
    assert len(cells) == 256
    Ns = np.array([c.N for c in cells])
    assert np.all(Ns % 8 == 0) and Ns.min() >= 56 and Ns.max() <= 2 * 2048
    assert Ns.min() <= 96 and Ns.max() >= 1024 and len(set(Ns.tolist())) > 20
    for c in cells:
        _check_common(c)
        assert np.all(c.fixed_q[c.site_class < 0] == -2.0)
        assert 2 <= c.S <= 5 and np.all((c.z >= 1) & (c.z <= 4))
        assert abs(_total_charge(c)) < 1e-9
        assert 0.01 <= c.kT <= 0.2


def test_population_generator_keeps_counts():
    p = synth.layered_problem(reps=(2, 2, 1))
    pop = synth.random_population(p, 50, 3)
    vclass = p.site_class[p.site_class >= 0]
    for b in range(50):
        for k in range(p.n_class):
            assert np.array_equal(np.bincount(pop[b][vclass == k], minlength=p.S), p.counts[k])
    assert np.array_equal(pop, synth.random_population(p, 50, 3))


@pytest.mark.parametrize("reps", synth.TABLE1_CELLS[:3])
def test_o3_table1_cells(reps):
    """O3 Na2/3[Li1/6 Fe1/6 Co1/6 Ni1/6 Mn1/3]O2: per sqrt3 cell 9 Na positions
    (6 Na + 3 vacancies), 9 TM positions, 18 O at -1.75; neutral."""
    p = synth.o3_layered_problem(reps)
    _check_common(p)
    ncell = reps[0] * reps[1] * reps[2]
    assert p.N == 36 * ncell and p.Nv == 18 * ncell
    assert np.allclose(p.fixed_q[p.site_class < 0], -1.75)
    assert abs(_total_charge(p)) < 1e-9

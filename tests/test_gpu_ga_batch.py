"""GA populations of several cells of different sizes in one launch per step
(goac_batch_ga_run, the batching form): every cell's population evolves
exactly as the oracle's GA run with its own key, and as the single-cell GPU run
with that key; the energies stay consistent with a full FP64 rescoring."""
import numpy as np
import pytest
import torch

import goac_synth as synth
import oracle
from gpu_common import build_pair, gpu_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2409_08808_gb300 as g
    return g.Context(0)


def _cells():
    return [(synth.layered_problem(reps=(2, 2, 1)), 48, 8), (synth.layered_problem(reps=(3, 3, 1)), 40, 9),
            (synth.o3_layered_problem((2, 2, 1)), 33, 10)]


def test_batch_ga_equals_oracle_per_cell(ctx):
    import paper_2409_08808_gb300 as g
    cells = _cells()
    seed, n_gen, n_elite, p_mut = 4, 5, 2, 0.1
    probs, pops, refs = [], [], []
    for i, (prob, P, ps) in enumerate(cells):
        Jg, Jo = build_pair(ctx, prob)
        probs.append(gpu_problem(ctx, prob, Jg))
        pop = synth.random_population(prob, P, ps)
        pops.append(torch.tensor(pop, device="cuda"))
        refs.append(oracle.ga_run(Jo, prob.site_class, prob.fixed_q, prob.z, pop, n_gen, n_elite, p_mut,
                                  seed=seed + i))
    E = g.batch_ga_run(ctx, probs, pops, n_gen, n_elite, oracle.p_mut_to_u32(p_mut), seed)
    for i in range(len(cells)):
        assert np.array_equal(pops[i].cpu().numpy(), refs[i][0]), i
        assert np.allclose(E[i].cpu().numpy(), refs[i][1], rtol=1e-10), i


def test_batch_ga_equals_single_cell_runs(ctx):
    """16 cells of the uneven batch (rocksalt / spinel-like, 56 .. 2016 sites),
    populations of 64 .. 256: each equals its own single-cell incremental run,
    counts are preserved and the energies match a full FP64 rescoring."""
    import paper_2409_08808_gb300 as g
    cells = synth.batch_problems(16)
    probs, pops, alone = [], [], []
    seed, n_gen = 77, 12
    for i, pr in enumerate(cells):
        frac = torch.tensor(pr.frac, device="cuda")
        J = g.build_ewald(ctx, pr.lattice, frac, pr.alpha, pr.nimg, pr.kcut)
        gp = g.Problem(ctx, J, pr.site_class, pr.fixed_q, pr.z, pr.counts)
        probs.append(gp)
        P = 64 * (1 + i % 4)
        start = gp.random_configs(P, 100 + i)
        pops.append(start.clone())
        one = start.clone()
        E1 = gp.ga_run(one, n_gen, 3, oracle.p_mut_to_u32(0.2), seed + i, precision="f64_incr")
        alone.append((one, E1))
    E = g.batch_ga_run(ctx, probs, pops, n_gen, 3, oracle.p_mut_to_u32(0.2), seed)
    for i, gp in enumerate(probs):
        assert torch.equal(pops[i], alone[i][0]), i
        assert torch.equal(E[i], alone[i][1]), i
        E64 = gp.score(pops[i], "f64")
        assert ((E[i] - E64).abs() / E64.abs()).max().item() <= 1e-10
        vclass = cells[i].site_class[cells[i].site_class >= 0]
        fin = pops[i].cpu().numpy()
        for k in range(cells[i].n_class):
            for s in range(cells[i].S):
                assert np.all(((vclass == k)[None, :] & (fin == s)).sum(1) == cells[i].counts[k, s])


def test_batch_ga_rejects_bad_arguments(ctx):
    import paper_2409_08808_gb300 as g
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, _ = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = gp.random_configs(16, 1)
    with pytest.raises(g.GoacError):
        g.batch_ga_run(ctx, [gp], [pop], 2, 1, 0, 1, precision="f64")
    with pytest.raises(g.GoacError):
        g.batch_ga_run(ctx, [gp, gp], [pop, pop.clone()], 2, 1, 0, 1)
    with pytest.raises(g.GoacError):
        g.batch_ga_run(ctx, [gp], [pop], 2, 17, 0, 1)

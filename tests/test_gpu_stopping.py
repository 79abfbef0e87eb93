"""Run-level stops and statistics on the GPU against the oracle (Section
"Internal Fortran Heuristics in GOAC": a run ends after a number of steps or
generations, or of steps / generations without improvement, or a time
budget; the n lowest structures are the output): the chains and populations
stop at the oracle's step / generation, with the oracle's configurations,
energies and statistics."""
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


@pytest.mark.parametrize("cell,C,steps,kT,patience,W", [
    ("rocksalt222", 8, 20000, 0.05, 500, 0),     # the 2x2x2 rocksalt parity workload, stopped early
    ("rocksalt222", 8, 20000, 0.05, 0, 0),       # no patience: every step, statistics only
    ("layered661", 6, 4000, 0.1, 300, 4),        # two classes, 4 warps per chain
    ("layered661", 6, 4000, 0.1, 300, 2),
])
def test_mc_patience_and_statistics(ctx, cell, C, steps, kT, patience, W):
    prob = synth.rocksalt_problem((2, 2, 2), 4.2) if cell == "rocksalt222" else synth.layered_problem((6, 6, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, C, 5)
    ref = oracle.mc_run_ex(Jo, prob.site_class, prob.fixed_q, prob.z, start, kT, steps, 0x600AC, step0=64,
                           patience=patience)
    gp.mc_set_shape(W, 0, "f64")
    try:
        got = gp.mc_run_ex(torch.tensor(start, device="cuda"), kT, steps, 0x600AC, step0=64, patience=patience)
        torch.cuda.synchronize()
    finally:
        gp.mc_set_shape(0, 0, "f64")
    g = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in got.items()}
    assert np.array_equal(g["species"], ref["species"])
    assert np.array_equal(g["best_species"], ref["best_species"])
    for k_got, k_ref in [("n_accept", "n_accept"), ("n_noop", "n_noop"), ("best_step", "best_step"),
                         ("steps", "steps_done")]:
        assert np.array_equal(g[k_got], ref[k_ref]), k_got
    assert np.allclose(g["E"], ref["E"], rtol=1e-10, atol=0)
    assert np.allclose(g["bestE"], ref["bestE"], rtol=1e-10, atol=0)
    if patience:
        assert np.all(ref["steps_done"] < steps)      # the rule stopped every chain
    else:
        assert np.all(ref["steps_done"] == steps)


def test_mc_ex_without_patience_equals_mc_run(ctx):
    prob = synth.layered_problem((3, 3, 1))
    Jg, _ = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, 20, 9)
    a = gp.mc_run(torch.tensor(start, device="cuda"), 0.1, 3000, 3, precision="f32")
    b = gp.mc_run_ex(torch.tensor(start, device="cuda"), 0.1, 3000, 3, precision="f32")
    assert torch.equal(a["species"], b["species"]) and torch.equal(a["E"], b["E"])
    assert torch.equal(a["n_accept"], b["n_accept"]) and torch.all(b["steps"] == 3000)


@pytest.mark.parametrize("precision", ["f64", "f64_incr"])
@pytest.mark.parametrize("P,patience,seed", [(48, 3, 4), (64, 4, 5)])
def test_ga_patience_parity(ctx, precision, P, patience, seed):
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, P, 8)
    fin_o, E_o, gens_o, best_o, stop_o = oracle.ga_run_ex(Jo, prob.site_class, prob.fixed_q, prob.z, pop, 60, 2, 0.1,
                                                          seed, patience=patience)
    assert stop_o and gens_o < 60
    sp = torch.tensor(pop, device="cuda")
    out = gp.ga_run_ex(sp, 60, 2, oracle.p_mut_to_u32(0.1), seed, precision=precision, patience=patience, topk=8)
    st = out["stats"][0]
    assert (st["generations"], st["best_generation"], st["stop_reason"]) == (gens_o, best_o, 1)
    assert np.array_equal(sp.cpu().numpy(), fin_o)
    E = out["E"].cpu().numpy()
    assert np.allclose(E, E_o, rtol=1e-10)
    assert abs(st["best_E"] - E_o.min()) <= 1e-10 * abs(E_o.min())
    # the n lowest structures: the oracle's 8 lowest (E, index), FP64 energies sorted
    order = np.lexsort((np.arange(P), E_o))[:8]
    idx = out["top_idx"][0].cpu().numpy()
    assert sorted(idx.tolist()) == sorted(order.tolist())
    assert np.allclose(out["top_E"][0].cpu().numpy(), np.sort(E_o[order]), rtol=1e-10)


def test_ga_populations_stop_independently(ctx):
    """Two populations, patience per population: each ends at the generation
    (and with the population) that the oracle's run with its key gives."""
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    P, R, seed = 48, 2, 4
    pops = [synth.random_population(prob, P, 8 + r) for r in range(R)]
    ref = [oracle.ga_run_ex(Jo, prob.site_class, prob.fixed_q, prob.z, pops[r], 60, 2, 0.1, seed + r, patience=3)
           for r in range(R)]
    sp = torch.tensor(np.concatenate(pops), device="cuda")
    out = gp.ga_run_ex(sp, 60, 2, oracle.p_mut_to_u32(0.1), seed, precision="f64", patience=3, R=R)
    fin = sp.cpu().numpy()
    for r in range(R):
        assert np.array_equal(fin[r * P:(r + 1) * P], ref[r][0])
        assert out["stats"][r]["generations"] == ref[r][2] and out["stats"][r]["stop_reason"] == 1


def test_ga_time_budget_and_plain_run(ctx):
    prob = synth.layered_problem(reps=(3, 3, 1))
    Jg, _ = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = gp.random_configs(256, 3)
    a = pop.clone()
    out = gp.ga_run_ex(a, 100, 4, oracle.p_mut_to_u32(0.1), 7, precision="bf16x3", time_budget_s=1e-9)
    st = out["stats"][0]
    assert st["stop_reason"] == 2 and st["generations"] == 8        # the first check, after 8 generations
    b = pop.clone()
    E8 = gp.ga_run(b, 8, 4, oracle.p_mut_to_u32(0.1), 7, precision="bf16x3")
    assert torch.equal(a, b) and torch.equal(out["E"], E8)
    c = pop.clone()
    out = gp.ga_run_ex(c, 12, 4, oracle.p_mut_to_u32(0.1), 7, precision="bf16x3")
    assert out["stats"][0] == {"generations": 12, "best_generation": out["stats"][0]["best_generation"],
                               "stop_reason": 0, "best_E": out["stats"][0]["best_E"]}
    d = pop.clone()
    gp.ga_run(d, 12, 4, oracle.p_mut_to_u32(0.1), 7, precision="bf16x3")
    assert torch.equal(c, d)


def test_ga_ex_rejects_bad_parameters(ctx):
    import paper_2409_08808_gb300 as g
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, _ = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = gp.random_configs(16, 3)
    for kw in [dict(patience=-1), dict(topk=17), dict(time_budget_s=-1.0)]:
        with pytest.raises(g.GoacError):
            gp.ga_run_ex(pop, 3, 1, 0, 1, **kw)
    with pytest.raises(g.GoacError):
        gp.mc_run_ex(pop[:2].clone(), 0.1, 10, 1, patience=-5)

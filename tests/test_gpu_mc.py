"""GPU parity of parallel-chain Metropolis swap MC against the oracle, with a
shared Philox stream: configurations bit-exact, energies within 1e-10."""
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


def _run_both(ctx, prob, C, steps, kT, seed, step0=0, init_seed=5):
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, C, init_seed)
    ref = oracle.mc_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, kT, steps, seed, step0=step0)
    sp = torch.tensor(start, device="cuda")
    got = gp.mc_run(sp, kT, steps, seed, step0=step0, precision="f64")
    torch.cuda.synchronize()
    return ref, {k: (v.cpu().numpy() if v is not None else None) for k, v in got.items()}, gp, start


def test_mc_rocksalt_trajectory_parity(ctx):
    """Rocksalt 2x2x2 (a = 4.2 A): 32 anions fixed at -2, 16 x +1 / 16 x +3
    cations; 8 chains x 20,000 swaps at kT = 0.05 eV."""
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    ref, got, _, _ = _run_both(ctx, prob, 8, 20000, 0.05, seed=0x600AC)
    assert np.array_equal(got["species"], ref["species"])
    assert np.array_equal(got["n_accept"], ref["n_accept"])
    assert np.array_equal(got["best_species"], ref["best_species"])
    assert np.allclose(got["E"], ref["E"], rtol=1e-10, atol=0)
    assert np.allclose(got["bestE"], ref["bestE"], rtol=1e-10, atol=0)


def test_mc_multiclass_trajectory_parity(ctx):
    prob = synth.layered_problem(reps=(2, 2, 1))
    ref, got, _, _ = _run_both(ctx, prob, 5, 6000, 0.1, seed=77, step0=123)
    assert np.array_equal(got["species"], ref["species"])
    assert np.array_equal(got["n_accept"], ref["n_accept"])
    assert np.allclose(got["E"], ref["E"], rtol=1e-10)


def test_mc_ragged_steps_and_resume(ctx):
    prob = synth.tiny_rocksalt_problem()
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, 3, 9)
    a = torch.tensor(start, device="cuda")
    gp.mc_run(a, 0.3, 1001, 3)
    b = torch.tensor(start, device="cuda")
    gp.mc_run(b, 0.3, 501, 3)
    gp.mc_run(b, 0.3, 500, 3, step0=501)
    assert torch.equal(a, b)
    ref = oracle.mc_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, 0.3, 1001, 3)
    assert np.array_equal(a.cpu().numpy(), ref["species"])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_mc_autotune_keeps_trajectories(ctx, prec):
    """The autotuned launch shape (warps per chain, chains per CTA) changes no
    trajectory: the same chains as with the size-based shape, and in FP64 the
    oracle's."""
    prob = synth.layered_problem(reps=(3, 3, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, 40, 12)
    before = torch.tensor(start, device="cuda")
    out0 = gp.mc_run(before, 0.1, 3000, 5, precision=prec)
    W, cpc, ms = gp.mc_autotune(torch.tensor(start, device="cuda"), 0.1, 200, prec)
    assert W in (1, 2, 4) and cpc in (1, 2, 4, 8, 15) and ms > 0
    after = torch.tensor(start, device="cuda")
    out1 = gp.mc_run(after, 0.1, 3000, 5, precision=prec)
    assert torch.equal(before, after)
    assert torch.equal(out0["n_accept"], out1["n_accept"])
    assert torch.equal(out0["E"], out1["E"])
    if prec == "f64":
        ref = oracle.mc_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, 0.1, 3000, 5)
        assert np.array_equal(after.cpu().numpy(), ref["species"])


def test_mc_zero_steps_and_zero_temperature(ctx):
    prob = synth.tiny_rocksalt_problem()
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, 2, 4)
    sp = torch.tensor(start, device="cuda")
    out = gp.mc_run(sp, 0.0, 0, 1)
    assert np.array_equal(sp.cpu().numpy(), start)
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, start)
    assert np.allclose(out["E"].cpu().numpy(), Eo, rtol=1e-10)
    ref = oracle.mc_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, 0.0, 700, 11)
    gp.mc_run(sp, 0.0, 700, 11)
    assert np.array_equal(sp.cpu().numpy(), ref["species"])


def test_mc_f32_variant_invariants(ctx):
    prob = synth.layered_problem(reps=(3, 3, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, 16, 8)
    sp = torch.tensor(start, device="cuda")
    out = gp.mc_run(sp, 0.05, 4000, 21, precision="f32")
    fin = sp.cpu().numpy()
    vclass = prob.site_class[prob.site_class >= 0]
    for c in range(16):
        for k in range(prob.n_class):
            for s in range(prob.S):
                assert ((vclass == k) & (fin[c] == s)).sum() == prob.counts[k, s]
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, fin)
    # FP32 phi drifts by ~1e-6 relative per accepted swap at most
    assert np.allclose(out["E"].cpu().numpy(), Eo, rtol=2e-5)
    assert np.all(out["E"].cpu().numpy() < oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, start))


def test_batch_mc_matches_single_runs(ctx):
    """Persistent work-queue launch (and its CUDA-graph replay) gives the same
    chains as one launch per problem with key seed + p; problem 0 also
    matches the oracle."""
    import paper_2409_08808_gb300 as g
    probs = synth.batch_problems(n_cells=5, n_min=16, n_max=160, seed=99)
    gps, starts, kts, Jos = [], [], [], []
    for i, pr in enumerate(probs):
        Jg, Jo = build_pair(ctx, pr)
        gps.append(gpu_problem(ctx, pr, Jg))
        Jos.append(Jo)
        starts.append(synth.random_population(pr, 3 + i, 40 + i))
        kts.append(torch.full((3 + i,), pr.kT, dtype=torch.float64, device="cuda"))
    results = {}
    for mode in (0, 1, 2, 2):
        sps = [torch.tensor(s, device="cuda") for s in starts]
        E, bE = g.batch_mc_run(ctx, gps, sps, kts, 3000, seed=1000, mode=mode, chains_per_cta=2)
        torch.cuda.synchronize()
        results.setdefault(mode, []).append(([s.cpu().numpy() for s in sps], [e.cpu().numpy() for e in E]))
    base_sp, base_E = results[0][0]
    for mode in (1, 2):
        for sp, E in results[mode]:
            for i in range(len(probs)):
                assert np.array_equal(sp[i], base_sp[i])
                assert np.array_equal(E[i], base_E[i])
    ref = oracle.mc_run(Jos[0], probs[0].site_class, probs[0].fixed_q, probs[0].z, starts[0], probs[0].kT, 3000, 1000)
    assert np.array_equal(base_sp[0], ref["species"])
    assert np.allclose(base_E[0], ref["E"], rtol=1e-10)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_mc_multiwarp_chain_equals_single_warp_chain(ctx, prec):
    """N = 4096 (the benchmark cell): goac_mc_run runs each chain with 4 warps
    and GEMM-built potentials; the batched kernel runs the same chain with one
    warp and its own potential build.  With the same Philox key both must take
    the same swaps (the one-warp chain matches the oracle in the tests above)."""
    import paper_2409_08808_gb300 as g
    prob = synth.random_cubic_problem()
    J = g.build_ewald(ctx, prob.lattice, torch.tensor(prob.frac, device="cuda"), prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, J)
    start = synth.random_population(prob, 6, 3)
    a = torch.tensor(start, device="cuda")
    out = gp.mc_run(a, 0.05, 3000, 77, step0=10, precision=prec)
    b = torch.tensor(start, device="cuda")
    kT = [torch.full((6,), 0.05, dtype=torch.float64, device="cuda")]
    E, _ = g.batch_mc_run(ctx, [gp], [b], kT, 3000, 77, step0=10, precision=prec, chains_per_cta=2, mode=1)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert out["n_accept"].min().item() > 50
    E64 = gp.score(a, "f64")
    tol = 1e-9 if prec == "f64" else 2e-5
    assert torch.allclose(out["E"], E64, rtol=tol, atol=0)
    assert torch.allclose(E[0], E64, rtol=tol, atol=0)


def test_sa_trajectory_parity(ctx):
    """Simulated annealing, kT 1.0 -> 0.01 eV over 5000 steps: same swaps as the oracle."""
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, 8, 12)
    ref = oracle.sa_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, 1.0, 0.01, 5000, 5000, seed=33)
    sp = torch.tensor(start, device="cuda")
    out = gp.sa_run(sp, 1.0, 0.01, 5000, 5000, 33)
    assert np.array_equal(sp.cpu().numpy(), ref["species"])
    assert np.array_equal(out["n_accept"].cpu().numpy(), ref["n_accept"])
    assert np.allclose(out["E"].cpu().numpy(), ref["E"], rtol=1e-10)


def test_remc_parity(ctx):
    """Replica exchange, 3 groups x 4 temperatures, 6 rounds of 400 steps: same
    configurations, temperature permutation and number of exchanges."""
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    G, R = 3, 4
    ladder = [0.05, 0.15, 0.4, 1.0]
    start = synth.random_population(prob, G * R, 13)
    ref = oracle.remc_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, G, R, ladder, 6, 400, seed=44)
    sp = torch.tensor(start, device="cuda")
    E, perm, nex = gp.remc_run(sp, G, R, ladder, 6, 400, 44)
    assert ref["n_exchanges"] > 0
    assert nex == ref["n_exchanges"]
    assert np.array_equal(perm.cpu().numpy(), ref["perm"])
    assert np.array_equal(sp.cpu().numpy(), ref["species"])
    assert np.allclose(E.cpu().numpy(), ref["E"], rtol=1e-10)


@pytest.mark.parametrize("which,B", [("rocksalt", 8), ("layered", 5), ("o3_quarter", 4)])
def test_gd_parity(ctx, which, B):
    """All-pairs steepest descent: same end configurations, steps and energies
    as the oracle (ties within 1e-9 eV resolve to the lowest pair on both sides).
    The kernel filters pairs in FP32 and decides in FP64: the symmetric rocksalt
    cell has many exactly tied pairs (tie sets overflow, the FP64 second pass
    decides), the layered cell few, and the O3 cell's charges are quarters
    (2d and d^2 not integers)."""
    prob = {"rocksalt": lambda: synth.rocksalt_problem((2, 2, 2), 4.2),
            "layered": lambda: synth.layered_problem(reps=(2, 2, 1)),
            "o3_quarter": lambda: synth.o3_layered_problem()}[which]()
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, B, 19)
    ref = oracle.gd_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, 500)
    sp = torch.tensor(start, device="cuda")
    E, steps = gp.gd_run(sp, 500)
    assert np.array_equal(steps.cpu().numpy(), ref["steps"])
    assert np.array_equal(sp.cpu().numpy(), ref["species"])
    assert np.allclose(E.cpu().numpy(), ref["E"], rtol=1e-10)
    assert ref["steps"].max() > 3


def test_hybrid_parity(ctx):
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    start = synth.random_population(prob, 8, 23)
    lad = [0.05, 0.15, 0.4, 1.0]
    ref = oracle.hybrid_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, 2, 4, lad, 2, 3, 300, 3, 1, 0.2, seed=7)
    sp = torch.tensor(start, device="cuda")
    E = gp.hybrid_run(sp, 2, 4, lad, 2, 3, 300, 3, 1, oracle.p_mut_to_u32(0.2), 7)
    assert np.array_equal(sp.cpu().numpy(), ref["species"])
    assert np.allclose(E.cpu().numpy(), ref["E"], rtol=1e-10)


def test_mc_exact_potentials_quarter_charges(ctx):
    """O3 layered oxide 2x2x1 (charges in quarters: O 1.75-, Fe 2.5+, Co 3.5+),
    whose FP64 chains start from the integer-digit tensor-core potentials:
    trajectories identical to the oracle's."""
    prob = synth.o3_layered_problem((2, 2, 1))
    ref, got, _, _ = _run_both(ctx, prob, 6, 5000, 0.1, seed=31)
    assert np.array_equal(got["species"], ref["species"])
    assert np.array_equal(got["n_accept"], ref["n_accept"])
    assert np.allclose(got["E"], ref["E"], rtol=1e-10, atol=0)


def test_mc_exact_potentials_full_size(ctx):
    """N = 4096, 300 chains: the starting energies from the integer-digit
    potentials equal the FP64 scoring path, and after 64 swaps per chain the
    running energies equal FP64 rescoring of the final configurations."""
    import paper_2409_08808_gb300 as g
    prob = synth.random_cubic_problem()
    J = g.build_ewald(ctx, prob.lattice, torch.tensor(prob.frac, device="cuda"), prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, J)
    sp = gp.random_configs(300, 5)
    E64 = gp.score(sp, "f64")
    out = gp.mc_run(sp.clone(), 0.05, 0, 1)
    assert ((out["E"] - E64).abs() / E64.abs()).max().item() <= 1e-11
    out = gp.mc_run(sp, 0.05, 64, 1)
    E64 = gp.score(sp, "f64")
    assert ((out["E"] - E64).abs() / E64.abs()).max().item() <= 1e-10


def test_batch_full_size_sampled(ctx):
    """The uneven batch at full size (256 cells, N 64..2048, 512 chains each)
    in the graph-captured persistent launch: counts preserved in every chain,
    all 512 chains of the three smallest cells identical to the oracle's, and
    the chains of the three largest cells with running energies equal to FP64
    rescoring."""
    import paper_2409_08808_gb300 as g
    cells = synth.batch_problems(256)
    C, steps = 512, 64
    gps, sps, kts, starts = [], [], [], []
    for i, pr in enumerate(cells):
        J = g.build_ewald(ctx, pr.lattice, torch.tensor(pr.frac, device="cuda"), pr.alpha, pr.nimg, pr.kcut)
        gps.append(gpu_problem(ctx, pr, J))
        sps.append(gps[-1].random_configs(C, 100 + i))
        starts.append(sps[-1].clone())
        kts.append(torch.full((C,), pr.kT, dtype=torch.float64, device="cuda"))
    E, _ = g.batch_mc_run(ctx, gps, sps, kts, steps, 7, mode=2)
    torch.cuda.synchronize()
    for pr, sp in zip(cells, sps):
        vclass = pr.site_class[pr.site_class >= 0]
        fin = sp.cpu().numpy()
        for k in range(pr.n_class):
            for s in range(pr.S):
                assert np.all(((vclass[None, :] == k) & (fin == s)).sum(axis=1) == pr.counts[k, s])
    order = np.argsort([pr.N for pr in cells])
    for i in order[:3]:
        pr = cells[i]
        Jo = oracle.ewald_J(pr.lattice, pr.frac, pr.alpha, pr.nimg, pr.kcut)
        ref = oracle.mc_run(Jo, pr.site_class, pr.fixed_q, pr.z, starts[i].cpu().numpy(), pr.kT, steps, 7 + int(i))
        assert np.array_equal(sps[i].cpu().numpy(), ref["species"]), (i, pr.N)
        assert np.allclose(E[i].cpu().numpy(), ref["E"], rtol=1e-10)
    for i in order[-3:]:
        E64 = gps[i].score(sps[i], "f64")
        assert torch.allclose(E[i], E64, rtol=1e-10, atol=0)


def test_sa_finds_exhaustive_ground_state(ctx):
    """Rocksalt 2x2x2 cation problem (N = 64, C(32, 16) = 601,080,390
    configurations): simulated annealing on the GPU (1,024 chains x 20,000
    swaps, kT 1.0 -> 0.002 eV, FP64) reaches the oracle's exhaustive minimum,
    and the best configurations it returns are among the stored minimisers."""
    from test_oracle_ground_state import read_golden
    vals, arg = read_golden()
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    import paper_2409_08808_gb300 as g
    Jg = g.build_ewald(ctx, prob.lattice, torch.tensor(prob.frac, device="cuda"), prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, Jg)
    sp = gp.random_configs(1024, 3)
    out = gp.sa_run(sp, 1.0, 0.002, 20000, 20000, 17)
    bestE = out["bestE"].cpu().numpy()
    assert bestE.min() == pytest.approx(vals["E_min_eV"], rel=1e-10, abs=0)
    assert np.all(bestE >= vals["E_min_eV"] - 1e-9)
    minimisers = set(map(tuple, arg.tolist()))
    hits = np.nonzero(bestE <= vals["E_min_eV"] + 1e-9)[0]
    best_sp = out["best_species"].cpu().numpy()
    assert all(tuple(best_sp[i].tolist()) in minimisers for i in hits)

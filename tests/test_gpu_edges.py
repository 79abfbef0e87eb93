"""Edge cases on the GPU: empty batches through every entry point, single
configurations in every scoring form, a problem with degenerate site classes
(a class holding one species only, a class of one position, species shared by
two classes), and a population whose species array passes 2^31 bytes."""
import dataclasses

import numpy as np
import pytest
import torch

import goac_synth as synth
import oracle
from gpu_common import build_pair, form_tolerance, gpu_problem, quad_scale

pytestmark = pytest.mark.gpu

FORMS = ["f64", "f32", "tf32", "tf32x2", "bf16x2", "bf16x3", "exact"]


@pytest.fixture(scope="module")
def ctx():
    import paper_2409_08808_gb300 as g
    return g.Context(0)


def _counts_ok(prob, pop):
    vclass = prob.site_class[prob.site_class >= 0]
    for b in range(pop.shape[0]):
        for k in range(prob.n_class):
            for s in range(prob.S):
                if ((vclass == k) & (pop[b] == s)).sum() != prob.counts[k, s]:
                    return False
    return True


def _exact_bound(prob, Jo, pop, Eo):
    """|E_exact - E| <= (sum_i |q_i|)^2 2^-46 max|J_vv| (six 8-bit digits per
    128-row panel) plus FP64 rounding of the sums."""
    vidx = np.nonzero(prob.site_class >= 0)[0]
    qabs = np.abs(prob.z[pop]).sum(axis=1)
    return qabs ** 2 * 2.0 ** -46 * np.abs(Jo[np.ix_(vidx, vidx)]).max() + 1e-10 * np.abs(Eo)


def test_empty_batches_are_noops(ctx):
    """B = C = P = G = 0 through every entry point: GOAC_OK and empty outputs
    (torch gives NULL data pointers for empty tensors), and the context stays
    usable afterwards."""
    import paper_2409_08808_gb300 as g
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    Nv, S = gp.Nv, prob.S
    none = torch.empty((0, Nv), dtype=torch.int8, device="cuda")
    for form in FORMS:
        assert gp.score(none, form).shape == (0,)
    assert gp.score_host(np.empty((0, Nv), np.int8)).shape == (0,)
    assert gp.score_host_async(torch.empty((0, Nv), dtype=torch.int8).pin_memory(), "bf16x2").shape == (0,)
    assert gp.random_configs(0, 1).shape == (0, Nv)
    out = gp.mc_run(none, 0.1, 100, 1)
    assert out["E"].shape == (0,) and out["species"].shape == (0, Nv)
    assert gp.mc_run(none, 0.1, 100, 1, precision="f32")["bestE"].shape == (0,)
    assert gp.sa_run(none, 0.5, 0.01, 100, 100, 1)["E"].shape == (0,)
    E, steps = gp.gd_run(none, 10)
    assert E.shape == (0,) and steps.shape == (0,)
    L0 = torch.empty((0, Nv, S), dtype=torch.float32, device="cuda")
    for prec in ("f64", "tf32x2"):
        E, dL = gp.energy_grad(L0, 1.0, prec)
        assert E.shape == (0,) and dL.shape == (0, Nv, S)
    assert gp.relaxed_descent(L0, 1.0, 0.01, 5).shape == (0,)
    assert gp.occupations(L0).shape == (0, Nv, S)
    assert gp.round_to_counts(L0).shape == (0, Nv)
    kids, _, _ = gp.ga_generation(none, torch.empty(0, dtype=torch.float64, device="cuda"), 0, 0, 0, 1)
    assert kids.shape == (0, Nv)
    assert gp.ga_run(none, 3, 0, 0, 1).shape == (0,)
    E, perm, nex = gp.remc_run(none, 0, 4, [0.05, 0.1, 0.2, 0.4], 2, 10, 1)
    assert E.shape == (0,) and nex == 0
    assert gp.hybrid_run(none, 0, 4, [0.05, 0.1, 0.2, 0.4], 1, 2, 10, 2, 0, 0, 1).shape == (0,)
    # a batch in which one problem has no chains (NULL buffers) and one has three
    start = synth.random_population(prob, 3, 8)
    sps = [torch.tensor(start, device="cuda"), none.clone()]
    kts = [torch.full((3,), 0.1, dtype=torch.float64, device="cuda"), torch.empty(0, dtype=torch.float64, device="cuda")]
    gp2 = gpu_problem(ctx, prob, Jg)
    for mode in (0, 1):
        sps[0] = torch.tensor(start, device="cuda")
        Eb, _ = g.batch_mc_run(ctx, [gp, gp2], sps, kts, 500, seed=40, mode=mode, chains_per_cta=2)
        assert Eb[1].shape == (0,)
        ref = oracle.mc_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, 0.1, 500, 40)
        assert np.array_equal(sps[0].cpu().numpy(), ref["species"])
        assert np.allclose(Eb[0].cpu().numpy(), ref["E"], rtol=1e-10)
    ctx.synchronize()
    pop = synth.random_population(prob, 5, 2)
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, pop)
    assert np.allclose(gp.score(torch.tensor(pop, device="cuda")).cpu().numpy(), Eo, rtol=1e-10)


def test_negative_and_oversized_counts_are_rejected(ctx):
    import paper_2409_08808_gb300 as g
    from paper_2409_08808_gb300 import _lib
    L = _lib.lib
    prob = synth.tiny_rocksalt_problem()
    Jg, _ = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    h = gp.handle
    e = torch.empty(4, dtype=torch.float64, device="cuda")
    sp = torch.zeros((4, gp.Nv), dtype=torch.int8, device="cuda")
    big = 2 ** 31 - 255            # GOAC_MAX_BATCH + 1
    for B in (-1, big):
        assert L.goac_score(h, sp.data_ptr(), B, 3, e.data_ptr()) == -1
        assert L.goac_random_configs(h, B, 1, sp.data_ptr()) == -1
    assert L.goac_score(h, sp.data_ptr(), 2 ** 31 - 1, 6, e.data_ptr()) == -1
    ctx.synchronize()
    assert torch.isfinite(gp.score(gp.random_configs(4, 2), "bf16x2")).all()
    # G R = 2^32 replicas > GOAC_MAX_BATCH, rejected before any buffer is used
    assert L.goac_remc_run(h, sp.data_ptr(), 2 ** 20, 2 ** 12, None, 1, 1, 1, 0, e.data_ptr(), None, None) == -1


@pytest.mark.parametrize("which", ["layered", "random300"])
def test_single_configuration_every_form(ctx, which):
    """B = 1: one configuration in a 256-wide tile of padding, every form
    against the oracle within its bound; top-1 FP64 rescoring."""
    if which == "layered":
        prob = synth.layered_problem(reps=(3, 3, 1))
    else:
        rng = np.random.default_rng(12)
        A = np.diag([8.0, 8.5, 9.0]) + rng.uniform(-0.5, 0.5, (3, 3))
        n = 300
        prob = synth.Problem(name="rand", lattice=A, frac=rng.uniform(0, 1, (n, 3)),
                             site_class=np.zeros(n, np.int32), fixed_q=np.zeros(n), z=np.array([2.0, -1.0]),
                             counts=np.array([[100, 200]], np.int32), alpha=0.0, nimg=(0, 0, 0), kcut=0.0)
        prob.alpha, prob.nimg, prob.kcut = synth.default_cutoffs(A)
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, 1, 77)
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, pop)
    sp = torch.tensor(pop, device="cuda")
    R = quad_scale(Jo, prob, pop)
    for form in FORMS:
        E = gp.score(sp, form).cpu().numpy()
        if form == "f64":
            assert abs(E[0] - Eo[0]) <= 1e-10 * abs(Eo[0])
        elif form == "exact":
            assert abs(E[0] - Eo[0]) <= _exact_bound(prob, Jo, pop, Eo)[0]
        elif form == "f32":
            # J_vv rounded to FP32 (2^-24 per entry) and Nv FP32 multiply-adds per site
            vidx = np.nonzero(prob.site_class >= 0)[0]
            qv = np.abs(prob.z[pop[0]])
            mass = qv @ np.abs(Jo[np.ix_(vidx, vidx)]) @ qv
            assert abs(E[0] - Eo[0]) <= (prob.Nv + 2) * 2.0 ** -24 * mass
        else:
            assert abs(E[0] - Eo[0]) <= form_tolerance(form, R, prob.Nv)[0]
    idx, E1 = gp.topk_rescore(sp, gp.score(sp, "bf16x2"), 1)
    assert idx.cpu().numpy().tolist() == [0]
    assert E1.cpu().numpy()[0] == pytest.approx(Eo[0], rel=1e-10)


def _degenerate_problem():
    """The 1x1x2 rocksalt cell with its 8 cations split into two classes of 4
    sharing species +1, +3, +2 (counts 2/1/1 and 1/2/1) and its 8 anions made
    variable: 7 in a class holding species -2 only (every swap a no-op) and 1
    in a class of its own (never picked).  Neutral: 7 + 9 - 16 = 0."""
    base = synth.tiny_rocksalt_problem()
    sc = base.site_class.copy()
    cat = np.nonzero(sc >= 0)[0]
    an = np.nonzero(sc < 0)[0]
    sc[cat[:4]] = 0
    sc[cat[4:]] = 1
    sc[an[:-1]] = 2
    sc[an[-1]] = 3
    z = np.array([1.0, 3.0, 2.0, -2.0])
    counts = np.array([[2, 1, 1, 0], [1, 2, 1, 0], [0, 0, 0, len(an) - 1], [0, 0, 0, 1]], np.int32)
    return dataclasses.replace(base, name="degenerate", site_class=sc.astype(np.int32), fixed_q=np.zeros(base.N),
                               z=z, counts=counts)


def test_degenerate_classes(ctx):
    prob = _degenerate_problem()
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    assert gp.Nv == 16 and gp.E_const == 0.0
    # random structures, scoring
    pop = gp.random_configs(60, 5).cpu().numpy()
    assert np.array_equal(pop, oracle.random_configs(prob.site_class, prob.counts, 60, 5))
    assert _counts_ok(prob, pop)
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, pop)
    sp = torch.tensor(pop, device="cuda")
    assert np.allclose(gp.score(sp, "f64").cpu().numpy(), Eo, rtol=1e-10, atol=0)
    assert np.all(np.abs(gp.score(sp, "exact").cpu().numpy() - Eo) <= _exact_bound(prob, Jo, pop, Eo))
    # Monte Carlo: same trajectory as the oracle (no-op proposals in class 2 consume their draws)
    start = pop[:8]
    ref = oracle.mc_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, 0.3, 5000, 91)
    a = torch.tensor(start, device="cuda")
    got = gp.mc_run(a, 0.3, 5000, 91)
    assert np.array_equal(a.cpu().numpy(), ref["species"])
    assert np.array_equal(got["n_accept"].cpu().numpy(), ref["n_accept"])
    assert np.allclose(got["E"].cpu().numpy(), ref["E"], rtol=1e-10)
    assert _counts_ok(prob, a.cpu().numpy())
    # GA generation: crossover partners stay inside the class although species are shared
    kids_o, par_o, nsw_o = oracle.ga_generation(prob.site_class, pop, Eo, 2, 0.5, gen=3, seed=17)
    kids, par, nsw = gp.ga_generation(sp, torch.tensor(Eo, device="cuda"), 2, oracle.p_mut_to_u32(0.5), 3, 17,
                                      record=True)
    assert np.array_equal(kids.cpu().numpy(), kids_o)
    assert np.array_equal(par.cpu().numpy(), par_o)
    assert np.array_equal(nsw.cpu().numpy(), nsw_o)
    assert _counts_ok(prob, kids_o)
    # steepest descent
    refg = oracle.gd_run(Jo, prob.site_class, prob.fixed_q, prob.z, pop[:6], 100)
    b = torch.tensor(pop[:6], device="cuda")
    Eg, steps = gp.gd_run(b, 100)
    assert np.array_equal(b.cpu().numpy(), refg["species"])
    assert np.array_equal(steps.cpu().numpy(), refg["steps"])
    assert np.allclose(Eg.cpu().numpy(), refg["E"], rtol=1e-10)
    # relaxed occupations: the one-species classes are pinned at p = 1
    Lg = synth.random_logits(prob, 2, 4)
    E2, dL = gp.energy_grad(torch.tensor(Lg, device="cuda"), 0.2, "f64")
    E2, dL = E2.cpu().numpy(), dL.cpu().numpy()
    for r in range(2):
        e_o, g_o = oracle.energy_grad(Jo, prob.site_class, prob.fixed_q, prob.z, prob.counts,
                                      Lg[r].astype(np.float64), 0.2)
        assert E2[r] == pytest.approx(e_o, rel=1e-10, abs=1e-10)
        assert np.max(np.abs(dL[r] - g_o)) <= 1e-6 * np.abs(g_o).max()
    vclass = prob.site_class[prob.site_class >= 0]
    p_gpu = gp.occupations(torch.tensor(Lg, device="cuda")).cpu().numpy()
    assert np.all(p_gpu[:, vclass >= 2, 3] == 1.0) and np.all(p_gpu[:, vclass >= 2, :3] == 0.0)
    rng = np.random.default_rng(6)
    allowed = (prob.counts[vclass] > 0).astype(np.float32)
    p = rng.dirichlet(np.ones(prob.S), size=(3, prob.Nv)).astype(np.float32) * allowed
    p /= p.sum(axis=2, keepdims=True)
    rounded = gp.round_to_counts(torch.tensor(p, device="cuda")).cpu().numpy()
    for r in range(3):
        assert np.array_equal(rounded[r], oracle.round_to_counts(prob.site_class, prob.counts, p[r]))
    assert _counts_ok(prob, rounded)
    # exhaustive: 12 x 12 configurations; simulated annealing reaches the minimum
    ex = oracle.enumerate_all(Jo, prob.site_class, prob.fixed_q, prob.z, prob.counts)
    assert ex["n_configs"] == 144
    out = gp.sa_run(gp.random_configs(256, 9), 1.0, 0.005, 4000, 4000, 23)
    assert out["bestE"].min().item() == pytest.approx(ex["Emin"], rel=1e-10)


def test_population_over_2gib(ctx):
    """Layered 5x5x1 (Nv = 150, padded to 256 sites) and B = 14,316,700
    configurations: the species array holds 2,147,505,000 bytes (> 2^31) and B
    is not a multiple of the 256-configuration tile.  The population is 4,096
    oracle-scored configurations repeated; every copy, up to the last, must
    score exactly as its original does in a 4,096 batch (the arithmetic of a
    configuration does not depend on which tile it sits in when the offset is a
    multiple of 256), and the originals match the oracle."""
    prob = synth.layered_problem(reps=(5, 5, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    K, B = 4096, 14_316_700
    assert B * gp.Nv > 2 ** 31 and B % 256 != 0
    small = synth.random_population(prob, K, 101)
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, small)
    sm = torch.tensor(small, device="cuda")
    big = sm.repeat((B + K - 1) // K, 1)[:B].contiguous()
    last = torch.arange(B - 300, B, device="cuda")
    R = quad_scale(Jo, prob, small[:64])
    for form in ("f64", "bf16x2", "exact"):
        Es = gp.score(sm, form)
        Eb = gp.score(big, form)
        torch.cuda.synchronize()
        head = Eb[: (B // K) * K].view(-1, K)
        assert torch.equal(head, Es.expand_as(head)), form
        assert torch.equal(Eb[last], Es[last % K]), form
        es = Es.cpu().numpy()
        if form == "f64":
            assert np.max(np.abs(es - Eo) / np.abs(Eo)) <= 1e-10
        elif form == "exact":
            assert np.all(np.abs(es - Eo) <= _exact_bound(prob, Jo, small, Eo))
        else:
            assert np.all(np.abs(es[:64] - Eo[:64]) <= form_tolerance(form, R, prob.Nv))
        del Eb, head
    # random structures at the same size: every sampled row is a valid structure
    del big
    torch.cuda.empty_cache()
    rc = gp.random_configs(B, 6)
    rows = torch.cat([torch.arange(0, 200, device="cuda"), last]).long()
    assert _counts_ok(prob, rc[rows].cpu().numpy())


@pytest.mark.parametrize("B,k", [(513, 64), (1025, 1024), (16385, 64), (250_000, 1024), (40_000, 1)])
def test_topk_radix_select(ctx, B, k):
    """Above 512 configurations the top-k selection is a radix select: the
    same set as the k smallest (E, index) of the given approximate energies,
    here integers and halves with many ties at and across the k-th place, and
    -0 / +0 together; the rescored energies are the oracle's."""
    prob = synth.tiny_rocksalt_problem()
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, B, 3)
    rng = np.random.default_rng(B + k)
    Ea = rng.integers(0, 400, B).astype(np.float64) * 0.5 - 100.0
    Ea[rng.integers(0, B, 50)] = -0.0
    Ea[rng.integers(0, B, 50)] = 0.0
    Ea[rng.integers(0, B, 3 * k)] = -250.0          # a block of ties at the smallest value
    want = np.lexsort((np.arange(B), Ea))[:k]
    idx, E = gp.topk_rescore(torch.tensor(pop, device="cuda"), torch.tensor(Ea, device="cuda"), k)
    idx, E = idx.cpu().numpy(), E.cpu().numpy()
    assert sorted(idx.tolist()) == sorted(want.tolist())
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, pop[np.sort(want)])
    Eo_by = dict(zip(np.sort(want).tolist(), Eo.tolist()))
    assert np.allclose(E, [Eo_by[i] for i in idx.tolist()], rtol=1e-10)
    assert np.all(np.diff(E) >= 0)


def test_context_close_returns_device_memory():
    """50 contexts, each with a problem that has built its lazily allocated
    operands (FP64 and BF16x2 scoring, an MC run), are created and closed: the
    device's free memory returns to its starting level (no handle or buffer
    leaks), and a closed context or problem raises GoacError when used."""
    import paper_2409_08808_gb300 as g
    prob = synth.layered_problem(reps=(2, 2, 1))
    frac = torch.tensor(prob.frac, device="cuda")
    pop = torch.tensor(synth.random_population(prob, 64, 3), device="cuda")

    def one_round():
        c = g.Context(0)
        J = g.build_ewald(c, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
        p = g.Problem(c, J, prob.site_class, prob.fixed_q, prob.z, prob.counts)
        E64 = p.score(pop, "f64")
        Ebf = p.score(pop, "bf16x2")
        p.mc_run(pop[:8].clone(), 0.1, 64, 1)
        c.synchronize()
        out = (E64.cpu(), Ebf.cpu())
        c.close()
        del J, E64, Ebf
        return c, p, out

    one_round()                     # module loading and torch's own caches first
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    first = None
    for _ in range(50):
        c, p, out = one_round()
        if first is None:
            first = out
        assert torch.equal(out[0], first[0]) and torch.equal(out[1], first[1])
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 <= 4 << 20, (free0, free1)
    assert c.closed
    with pytest.raises(g.GoacError):
        c.synchronize()
    with pytest.raises(g.GoacError):
        p.score(pop, "f64")
    c.close()                       # a second close is a no-op

"""GPU parity of the genetic algorithm, the relaxed-occupation energy and its
adjoint, and rounding to counts, against the oracle."""
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


def _counts_ok(prob, pop):
    vclass = prob.site_class[prob.site_class >= 0]
    for b in range(pop.shape[0]):
        for k in range(prob.n_class):
            for s in range(prob.S):
                if ((vclass == k) & (pop[b] == s)).sum() != prob.counts[k, s]:
                    return False
    return True


@pytest.mark.parametrize("P,n_elite,p_mut", [(200, 4, 0.3), (64, 0, 0.0), (33, 33, 1.0)])
def test_ga_generation_bit_exact(ctx, P, n_elite, p_mut):
    """Same population and (oracle) energies in: identical children, parents
    and swap counts out."""
    prob = synth.layered_problem(reps=(3, 3, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, P, 5)
    E = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, pop)
    kids_o, par_o, nsw_o = oracle.ga_generation(prob.site_class, pop, E, n_elite, p_mut, gen=7, seed=99)
    kids, par, nsw = gp.ga_generation(torch.tensor(pop, device="cuda"), torch.tensor(E, device="cuda"), n_elite,
                                      oracle.p_mut_to_u32(p_mut), 7, 99, record=True)
    assert np.array_equal(kids.cpu().numpy(), kids_o)
    assert np.array_equal(par.cpu().numpy(), par_o)
    assert np.array_equal(nsw.cpu().numpy(), nsw_o)


def test_ga_generation_equal_energies(ctx):
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, 50, 3)
    E = np.full(50, -123.0)
    kids_o, par_o, _ = oracle.ga_generation(prob.site_class, pop, E, 2, 0.2, gen=0, seed=1)
    kids, par, _ = gp.ga_generation(torch.tensor(pop, device="cuda"), torch.tensor(E, device="cuda"), 2,
                                    oracle.p_mut_to_u32(0.2), 0, 1, record=True)
    assert np.array_equal(kids.cpu().numpy(), kids_o)
    assert np.array_equal(par.cpu().numpy(), par_o)


def test_ga_run_parity(ctx):
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, 48, 8)
    fin_o, E_o = oracle.ga_run(Jo, prob.site_class, prob.fixed_q, prob.z, pop, 6, 2, 0.1, seed=4)
    sp = torch.tensor(pop, device="cuda")
    E = gp.ga_run(sp, 6, 2, oracle.p_mut_to_u32(0.1), 4, precision="f64").cpu().numpy()
    assert np.array_equal(sp.cpu().numpy(), fin_o)
    assert np.allclose(E, E_o, rtol=1e-10)


def test_ga_run_incremental_parity(ctx):
    """Incremental FP64 rescoring (each child's potential from its nearer
    parent's plus the J rows of the changed sites): the same populations as the
    oracle's GA with full q^T J q rescoring, energies within 1e-10."""
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, 48, 8)
    fin_o, E_o = oracle.ga_run(Jo, prob.site_class, prob.fixed_q, prob.z, pop, 6, 2, 0.1, seed=4)
    sp = torch.tensor(pop, device="cuda")
    E = gp.ga_run(sp, 6, 2, oracle.p_mut_to_u32(0.1), 4, precision="f64_incr").cpu().numpy()
    assert np.array_equal(sp.cpu().numpy(), fin_o)
    assert np.max(np.abs(E - E_o) / np.abs(E_o)) <= 1e-10


@pytest.mark.parametrize("prec", ["f64", "f64_incr"])
def test_ga_populations_equal_separate_runs(ctx, prec):
    """Three populations of 40 in one run (children of all from one launch,
    one rescoring call): each equals goac_ga_run on it alone with key seed + r,
    bit for bit, and population 1 equals the oracle's GA with that key."""
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    R, P, n_gen, n_elite, seed = 3, 40, 5, 3, 11
    pops = [synth.random_population(prob, P, 100 + r) for r in range(R)]
    sp = torch.tensor(np.concatenate(pops), device="cuda")
    E = gp.ga_run_populations(sp, R, n_gen, n_elite, oracle.p_mut_to_u32(0.2), seed, precision=prec)
    for r in range(R):
        spr = torch.tensor(pops[r], device="cuda")
        Er = gp.ga_run(spr, n_gen, n_elite, oracle.p_mut_to_u32(0.2), seed + r, precision=prec)
        assert torch.equal(sp[r * P:(r + 1) * P], spr)
        assert torch.equal(E[r * P:(r + 1) * P], Er)
    fin_o, E_o = oracle.ga_run(Jo, prob.site_class, prob.fixed_q, prob.z, pops[1], n_gen, n_elite, 0.2, seed=seed + 1)
    assert np.array_equal(sp[P:2 * P].cpu().numpy(), fin_o)
    assert np.max(np.abs(E[P:2 * P].cpu().numpy() - E_o) / np.abs(E_o)) <= 1e-10


def test_ga_incremental_degenerate_cell(ctx):
    """Rocksalt 2x2x2: symmetry and duplicated individuals make many energies
    equal, so the GA's rank and fitness decisions sit on ties that FP64 rounding
    (a different summation order, or the path of an incremental update) breaks
    differently from the oracle; both the dense and the incremental FP64 paths
    leave the oracle's trajectory after such a tie.  The run is checked by what
    holds on any trajectory: counts preserved, every energy equal to the full
    FP64 rescoring of its configuration within 1e-10, and elitism never losing
    the best energy."""
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    Jg, _ = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    sp = torch.tensor(synth.random_population(prob, 64, 8), device="cuda")
    best = []
    for gen in range(4):
        E = gp.ga_run(sp, 3, 2, oracle.p_mut_to_u32(0.1), 4, gen0=3 * gen, precision="f64_incr")
        best.append(E.min().item())
        E64 = gp.score(sp, "f64")
        assert ((E - E64).abs() / E64.abs()).max().item() <= 1e-10
    assert all(best[i] >= best[i + 1] - 1e-9 for i in range(3))
    assert _counts_ok(prob, sp.cpu().numpy())


def test_ga_incremental_full_size(ctx):
    """Layered 12x12x1 (Nv = 864), population 1024, 25 generations with
    incremental FP64 rescoring: every energy equals the FP64 path's full
    rescoring of the final population within 1e-10, counts are preserved, and
    sampled configurations match the oracle's energies."""
    import paper_2409_08808_gb300 as g
    prob = synth.layered_problem()
    Jg = g.build_ewald(ctx, prob.lattice, torch.tensor(prob.frac, device="cuda"), prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, Jg)
    pop = gp.random_configs(1024, 13)
    E = gp.ga_run(pop, 25, 20, oracle.p_mut_to_u32(0.1), 7, precision="f64_incr")
    E64 = gp.score(pop, "f64")
    assert ((E - E64).abs() / E64.abs()).max().item() <= 1e-10
    fin = pop.cpu().numpy()
    assert _counts_ok(prob, fin[:64])
    En = E.cpu().numpy()
    for b in (0, 1023):        # the oracle's direct Ewald energy of two final configurations
        q = oracle.config_charges(prob.site_class, prob.fixed_q, prob.z, fin[b])
        Eo = oracle.ewald_energy(prob.lattice, prob.frac, q, prob.alpha, prob.nimg, prob.kcut)
        assert abs(En[b] - Eo) <= 1e-10 * abs(Eo)


def test_ga_layered_full_size(ctx):
    """Layered 12x12x1 cell, N = 1296, population 1024: counts preserved,
    elitism keeps the best energy non-increasing, FP64 and split scoring."""
    prob = synth.layered_problem()
    import paper_2409_08808_gb300 as g
    frac = torch.tensor(prob.frac, device="cuda")
    Jg = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, Jg)
    pop = gp.random_configs(1024, 11)
    best = []
    for gen in range(3):
        E = gp.ga_run(pop, 1, 20, oracle.p_mut_to_u32(0.1), 5, gen0=gen, precision="f64")
        best.append(E.min().item())
    assert best[0] >= best[1] >= best[2]
    assert _counts_ok(prob, pop.cpu().numpy()[:64])
    E64 = gp.score(pop, "f64")
    E32 = gp.score(pop, "f32")
    Ebf = gp.score(pop, "bf16x3")
    assert torch.allclose(E, E64, rtol=0, atol=0)
    assert (E32 - E64).abs().max().item() < 1e-3 * E64.abs().max().item()
    assert (Ebf - E64).abs().max().item() < 1e-4 * E64.abs().max().item()
    # the oracle's q^T J q on the GPU-built J for elites, the middle and the last children
    fin = pop.cpu().numpy()
    rows = np.array([0, 1, 19, 20, 511, 1022, 1023])
    Eo = oracle.score(Jg.cpu().numpy(), prob.site_class, prob.fixed_q, prob.z, fin[rows])
    assert np.max(np.abs(E.cpu().numpy()[rows] - Eo) / np.abs(Eo)) <= 1e-10


@pytest.mark.parametrize("which,B", [("layered", 3), ("bcc", 5)])
def test_energy_grad_parity(ctx, which, B):
    prob = {"layered": lambda: synth.layered_problem(reps=(2, 1, 1)),
            "bcc": lambda: synth.bcc_relaxed_problem(n_side=4)}[which]()
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg) if which != "bcc" else None
    if gp is None:
        import paper_2409_08808_gb300 as g
        gp = g.Problem(ctx, Jg, prob.site_class, prob.fixed_q, prob.z, prob.counts, allow_charged=True)
    L = synth.random_logits(prob, B, 3)
    lam = 0.05
    E, dL = gp.energy_grad(torch.tensor(L, device="cuda"), lam, "f64")
    E, dL = E.cpu().numpy(), dL.cpu().numpy()
    for b in range(B):
        Eo, go = oracle.energy_grad(Jo, prob.site_class, prob.fixed_q, prob.z, prob.counts, L[b].astype(np.float64), lam)
        assert E[b] == pytest.approx(Eo, rel=1e-10, abs=1e-10)
        scale = np.abs(go).max()
        assert np.max(np.abs(dL[b] - go)) <= 1e-6 * scale + 1e-30


def _many_species_problem():
    """120 random sites in one class holding 10 species (more than the
    register path of the column sums takes), charged."""
    rng = np.random.default_rng(21)
    A = np.diag([9.0, 9.5, 10.0]) + rng.uniform(-0.5, 0.5, (3, 3))
    n = 120
    prob = synth.Problem(name="s10", lattice=A, frac=rng.uniform(0, 1, (n, 3)), site_class=np.zeros(n, np.int32),
                         fixed_q=np.zeros(n), z=np.array([1.0, 2.0, 3.0, -1.0, -2.0, 0.0, 1.5, -0.5, 4.0, -3.0]),
                         counts=np.full((1, 10), 12, np.int32), alpha=0.0, nimg=(0, 0, 0), kcut=0.0)
    prob.alpha, prob.nimg, prob.kcut = synth.default_cutoffs(A)
    return prob


@pytest.mark.parametrize("form", ["tf32x2", "f16x2"])
@pytest.mark.parametrize("which,B", [("layered", 3), ("bcc", 5), ("s10", 4), ("layered864", 3)])
def test_energy_grad_tensor_core_tf32x2(ctx, which, B, form):
    """J.Q on tcgen05 with J and the real Q split in hi/lo parts of 11-bit
    significands (TF32, or FP16 with J scaled per 128-row panel and q scaled
    by powers of two into FP16's range): within the deterministic bound of
    the form.  Per site, |dPhi_v| <= (gamma_K + 2^-20) sum_w |J_vw q_w|
    (K = 3 Nv products accumulated in FP32; the three kept products miss at
    most 2^-20 relative; an FP16 lo part below the normal range is off by at
    most 2^-39 of its panel's largest |J| or of max|z|, far inside that
    margin), so |dE| <= sum_v |q_v| that bound and |d(dE/dL_vs)| <=
    4 max|z| p_vs that bound (+ FP32 output rounding).
    Cases: one 256-site chunk of the elementwise kernels (layered 2x1x1, bcc
    4^3), more than 8 species (the general kernels), and several classes over
    Nv = 864 = 3 x 256 + 96 sites (chunk partials of every class, a ragged
    last chunk)."""
    import paper_2409_08808_gb300 as g
    prob = {"layered": lambda: synth.layered_problem(reps=(2, 1, 1)),
            "bcc": lambda: synth.bcc_relaxed_problem(n_side=4),
            "s10": _many_species_problem,
            "layered864": lambda: synth.layered_problem()}[which]()
    Jg, Jo = build_pair(ctx, prob)
    gp = g.Problem(ctx, Jg, prob.site_class, prob.fixed_q, prob.z, prob.counts, allow_charged=True)
    L = synth.random_logits(prob, B, 13)
    lam = 0.05
    E, dL = gp.energy_grad(torch.tensor(L, device="cuda"), lam, form)
    E, dL = E.cpu().numpy(), dL.cpu().numpy()
    K = 3 * gp.Nv
    eps = K * 2.0 ** -24 + 2.0 ** -20
    vidx = np.nonzero(prob.site_class >= 0)[0]
    zmax = np.abs(prob.z).max()
    for b in range(B):
        Eo, go = oracle.energy_grad(Jo, prob.site_class, prob.fixed_q, prob.z, prob.counts, L[b].astype(np.float64), lam)
        Lb = L[b].astype(np.float64)
        allowed = prob.counts[prob.site_class[vidx]] > 0
        ex = np.where(allowed, np.exp(Lb - np.where(allowed, Lb, -np.inf).max(axis=1, keepdims=True)), 0.0)
        pb = ex / ex.sum(axis=1, keepdims=True)
        q = prob.fixed_q.copy()
        q[vidx] = pb @ prob.z
        mass = (np.abs(Jo) @ np.abs(q))[vidx]
        assert abs(E[b] - Eo) <= eps * float(np.abs(q[vidx]) @ mass) + 1e-9
        bound = 4 * zmax * pb * (eps * mass)[:, None] + 2.0 ** -23 * np.abs(go)
        assert np.all(np.abs(dL[b] - go) <= bound + 1e-30)


def test_autograd_function(ctx):
    import paper_2409_08808_gb300 as g
    prob = synth.layered_problem(reps=(2, 1, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    L = torch.tensor(synth.random_logits(prob, 2, 9), device="cuda", requires_grad=True)
    E = g.RelaxedEnergy.apply(L, gp, 0.1, "f64")
    E.sum().backward()
    _, dL = gp.energy_grad(L.detach(), 0.1, "f64")
    assert torch.equal(L.grad, dL)


@pytest.mark.parametrize("B", [1, 6])
def test_round_to_counts_parity(ctx, B):
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, _ = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    rng = np.random.default_rng(B)
    p = rng.dirichlet(np.ones(prob.S), size=(B, prob.Nv)).astype(np.float32)
    p[0, 3, :] = p[0, 4, :]           # exact ties between sites
    got = gp.round_to_counts(torch.tensor(p, device="cuda")).cpu().numpy()
    for b in range(B):
        ref = oracle.round_to_counts(prob.site_class, prob.counts, p[b])
        assert np.array_equal(got[b], ref)
    assert _counts_ok(prob, got)


def test_energy_grad_full_size(ctx):
    """bcc N = 8192, 5 species (the differentiation workload): the TF32x2 path
    within the form's bound of the FP64 path (pinned to the oracle above), and
    the FP64 adjoint against central differences of the FP64 energy on sampled
    logits (h = 1e-4, the actual FP32 step taken)."""
    import paper_2409_08808_gb300 as g
    prob = synth.bcc_relaxed_problem()
    J = g.build_ewald(ctx, prob.lattice, torch.tensor(prob.frac, device="cuda"), prob.alpha, prob.nimg, prob.kcut)
    gp = g.Problem(ctx, J, prob.site_class, prob.fixed_q, prob.z, prob.counts, allow_charged=True)
    B, lam = 4, 1.0
    L = torch.tensor(synth.random_logits(prob, B, 21), device="cuda")
    E64, g64 = gp.energy_grad(L, lam, "f64")
    z = torch.tensor(prob.z, device="cuda")
    p = torch.softmax(L.double(), dim=2)
    q = p @ z
    mass = J.abs() @ q.abs().T                       # (N, B): sum_w |J_vw q_w|
    eps = 3 * gp.Nv * 2.0 ** -24 + 2.0 ** -20
    boundE = eps * (q.abs() * mass.T).sum(dim=1) + 1e-9
    boundG = 4 * z.abs().max() * p * (eps * mass.T)[:, :, None] + 2.0 ** -23 * g64.abs()
    for form in ("tf32x2", "f16x2"):
        Etc, gtc = gp.energy_grad(L, lam, form)
        assert torch.all((Etc - E64).abs() <= boundE), form
        assert torch.all((gtc - g64).abs() <= boundG + 1e-30), form
    rng = np.random.default_rng(5)
    for _ in range(8):
        b, v, s = int(rng.integers(B)), int(rng.integers(gp.Nv)), int(rng.integers(prob.S))
        Lp, Lm = L[b:b + 1].clone(), L[b:b + 1].clone()
        Lp[0, v, s] += 1e-4
        Lm[0, v, s] -= 1e-4
        h2 = float(Lp[0, v, s].double() - Lm[0, v, s].double())
        Ep, _ = gp.energy_grad(Lp, lam, "f64")
        Em, _ = gp.energy_grad(Lm, lam, "f64")
        fd = (Ep.item() - Em.item()) / h2
        assert abs(fd - g64[b, v, s].item()) <= 1e-5 * g64[b].abs().max().item() + 1e-6


@pytest.mark.parametrize("prec", ["f64", "tf32x2", "f16x2"])
def test_relaxed_descent_equals_gradient_steps(ctx, prec):
    """goac_relaxed_descent (for TF32x2 and FP16x2 the step is fused into the
    chain-rule kernel) gives the logits of the same number of explicit steps
    L <- L - eta dE/dL taken with goac_energy_grad, up to the FP32 rounding of
    the update, and the energy decreases."""
    import paper_2409_08808_gb300 as g
    prob = synth.bcc_relaxed_problem(n_side=4)
    Jg, _ = build_pair(ctx, prob)
    gp = g.Problem(ctx, Jg, prob.site_class, prob.fixed_q, prob.z, prob.counts, allow_charged=True)
    lam, eta, n = 0.5, 0.002, 5
    L0 = torch.tensor(synth.random_logits(prob, 3, 17), device="cuda")
    E_start, _ = gp.energy_grad(L0, lam, prec)
    L1 = L0.clone()
    E1 = gp.relaxed_descent(L1, lam, eta, n, prec)
    L2 = L0.clone()
    for _ in range(n):
        _, dL = gp.energy_grad(L2, lam, prec)
        L2 = L2 - eta * dL
    E2, _ = gp.energy_grad(L2, lam, prec)
    assert torch.allclose(L1, L2, rtol=1e-5, atol=1e-5)
    assert torch.allclose(E1, E2, rtol=1e-7, atol=0)
    assert torch.all(E1 < E_start)

"""GPU parity: Ewald J, batched scoring (FP64 and tensor-core split forms),
top-k FP64 rescoring and random structures, against the CPU oracle."""
import numpy as np
import pytest
import torch

import goac_synth as synth
import oracle
from gpu_common import build_pair, form_tolerance, gpu_problem, quad_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2409_08808_gb300 as g
    return g.Context(0)


def _random_cell_problem(n, seed):
    rng = np.random.default_rng(seed)
    A = np.diag([7.0, 7.5, 8.0]) + rng.uniform(-0.7, 0.7, (3, 3))
    frac = rng.uniform(0, 1, (n, 3))
    p = synth.Problem(name="rand", lattice=A, frac=frac, site_class=np.zeros(n, np.int32), fixed_q=np.zeros(n),
                      z=np.array([1.0, -1.0]), counts=np.array([[n // 2, n - n // 2]], np.int32),
                      alpha=0.0, nimg=(0, 0, 0), kcut=0.0)
    p.alpha, p.nimg, p.kcut = synth.default_cutoffs(A)
    return p


@pytest.mark.parametrize("which", ["rocksalt", "tiny", "layered", "random50"])
def test_build_ewald_parity(ctx, which):
    prob = {"rocksalt": lambda: synth.rocksalt_problem((2, 2, 2), 4.2),
            "tiny": synth.tiny_rocksalt_problem,
            "layered": lambda: synth.layered_problem(reps=(2, 2, 1)),
            "random50": lambda: _random_cell_problem(50, 3)}[which]()
    Jg, Jo = build_pair(ctx, prob)
    Jg = Jg.cpu().numpy()
    scale = np.abs(Jo).max()
    assert np.max(np.abs(Jg - Jo)) <= 1e-10 * scale
    assert np.array_equal(Jg, Jg.T)


def test_build_ewald_sampled_full_size(ctx):
    """N = 4096 random cubic cell: 256 sampled entries computed one by one by the oracle."""
    import paper_2409_08808_gb300 as g
    prob = synth.random_cubic_problem()
    frac = torch.tensor(prob.frac, device="cuda")
    Jg = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut).cpu().numpy()
    rng = np.random.default_rng(0)
    pairs = rng.integers(0, prob.N, (256, 2))
    pairs[:16, 1] = pairs[:16, 0]      # diagonal entries
    ref = oracle.ewald_J_entries(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut, pairs)
    got = Jg[pairs[:, 0], pairs[:, 1]]
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.abs(Jg).max()


@pytest.mark.parametrize("which,B", [("rocksalt", 37), ("layered", 300), ("random200", 513)])
def test_score_f64_parity(ctx, which, B):
    prob = {"rocksalt": lambda: synth.rocksalt_problem((2, 2, 2), 4.2),
            "layered": lambda: synth.layered_problem(reps=(3, 3, 1)),
            "random200": lambda: _random_cell_problem(200, 5)}[which]()
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, B, 17)
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, pop)
    Eg = gp.score(torch.tensor(pop, device="cuda"), "f64").cpu().numpy()
    assert np.max(np.abs(Eg - Eo) / np.abs(Eo)) <= 1e-10
    phi_o, ec_o = oracle.fixed_split(Jo, prob.site_class, prob.fixed_q)
    assert gp.E_const == pytest.approx(ec_o, rel=1e-10, abs=1e-9)
    assert np.allclose(gp.phi_fix().cpu().numpy(), phi_o, rtol=1e-10, atol=1e-10 * max(1.0, np.abs(phi_o).max()))
    Eh = gp.score_host(pop, "f64")
    assert np.array_equal(Eh, Eg)


@pytest.mark.parametrize("form", ["bf16x2", "bf16x3", "tf32", "tf32x2"])
@pytest.mark.parametrize("which,B", [("layered", 300), ("random300", 700)])
def test_score_tensor_core_forms(ctx, form, which, B):
    """Split forms on tcgen05 vs the FP64 oracle, several tiles and a ragged
    tail in both the site (128) and configuration (256) dimensions."""
    prob = {"layered": lambda: synth.layered_problem(reps=(4, 4, 1)),
            "random300": lambda: _random_cell_problem(300, 9)}[which]()
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, B, 23)
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, pop)
    Eg = gp.score(torch.tensor(pop, device="cuda"), form).cpu().numpy()
    R = quad_scale(Jo, prob, pop)
    tol = form_tolerance(form, R, prob.Nv)
    err = np.abs(Eg - Eo)
    assert np.all(err <= tol), (err.max(), tol.min())


def _round_sig(x, bits):
    """Round to `bits` significant bits, ties to even (exact, via frexp)."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(np.ldexp(m, bits)), e - bits)


def _tf32_rna(x32):
    """float32 -> TF32 (10 stored mantissa bits), round to nearest, ties away."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def _split_terms(J, form):
    if form.startswith("bf16"):
        T = 3 if form == "bf16x3" else 2
        terms, r = [], J.copy()
        for _ in range(T):
            t = _round_sig(r, 8)
            terms.append(t)
            r = r - t
        return terms
    hi = _tf32_rna(J.astype(np.float32)).astype(np.float64)
    if form == "tf32":
        return [hi]
    lo = _tf32_rna((J - hi).astype(np.float32)).astype(np.float64)
    return [hi, lo]


@pytest.mark.parametrize("form", ["bf16x2", "bf16x3", "tf32", "tf32x2"])
def test_split_forms_match_their_definition(ctx, form):
    """Each form equals q^T (sum of its split terms of the oracle's J) q, the
    terms rounded exactly as the form defines them (BF16: round to nearest
    even from FP64; TF32: FP64 -> FP32 -> TF32 round half away), within the
    FP32 accumulation bound gamma_K R alone.  A dropped, duplicated or
    mis-rounded term fails this."""
    prob = synth.rocksalt_problem((2, 2, 2), 4.2)
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, 300, 41)
    vidx = np.nonzero(prob.site_class >= 0)[0]
    Jvv = Jo[np.ix_(vidx, vidx)]
    Jdef = sum(_split_terms(Jvv, form))
    Jmod = Jo.copy()
    Jmod[np.ix_(vidx, vidx)] = Jdef
    Edef = oracle.score(Jmod, prob.site_class, prob.fixed_q, prob.z, pop)
    Eg = gp.score(torch.tensor(pop, device="cuda"), form).cpu().numpy()
    R = quad_scale(Jo, prob, pop)
    K = {"bf16x2": 2, "bf16x3": 3, "tf32": 1, "tf32x2": 2}[form] * prob.Nv
    assert np.all(np.abs(Eg - Edef) <= R * K * 2.0 ** -24)


def test_topk_rescore(ctx):
    prob = synth.layered_problem(reps=(3, 3, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, 600, 29)
    sp = torch.tensor(pop, device="cuda")
    Eapprox = gp.score(sp, "bf16x2")
    idx, E = gp.topk_rescore(sp, Eapprox, 64)
    idx, E = idx.cpu().numpy(), E.cpu().numpy()
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, pop)
    # the 64 lowest approximate energies (ties by index), sorted by FP64 energy
    ea = Eapprox.cpu().numpy()
    sel = np.lexsort((np.arange(600), ea))[:64]
    assert set(idx.tolist()) == set(sel.tolist())
    assert np.allclose(E, Eo[idx], rtol=1e-10)
    assert np.all(np.diff(E) >= 0)


def test_random_configs_match_oracle(ctx):
    prob = synth.layered_problem(reps=(2, 2, 1))
    Jg, _ = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    got = gp.random_configs(50, seed=1234).cpu().numpy()
    ref = oracle.random_configs(prob.site_class, prob.counts, 50, seed=1234)
    assert np.array_equal(got, ref)


def test_score_full_size_swap_property(ctx):
    """N = 4096, B = 4096 (the scoring benchmark's workload): E(after swap) -
    E(before) from the GPU equals the oracle's dE built from two rows of the
    oracle's J, for sampled configurations and swaps."""
    import paper_2409_08808_gb300 as g
    prob = synth.random_cubic_problem()
    frac = torch.tensor(prob.frac, device="cuda")
    Jg = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, Jg)
    B = 4096
    pop = synth.random_population(prob, B, 31)
    rng = np.random.default_rng(7)
    samples = []
    pop2 = pop.copy()
    for t in range(6):
        b = int(rng.integers(0, B))
        while True:
            i, j = rng.integers(0, prob.N, 2)
            if pop[b, i] != pop[b, j]:
                break
        pop2[b, i], pop2[b, j] = pop[b, j], pop[b, i]
        samples.append((b, int(i), int(j)))
    sp1 = torch.tensor(pop, device="cuda")
    sp2 = torch.tensor(pop2, device="cuda")
    E1 = gp.score(sp1, "f64").cpu().numpy()
    E2 = gp.score(sp2, "f64").cpu().numpy()
    Et1 = gp.score(sp1, "bf16x3").cpu().numpy()
    Et2 = gp.score(sp2, "bf16x3").cpu().numpy()
    for b, i, j in samples:
        q = prob.z[pop[b]]
        rows = np.array([[i, w] for w in range(prob.N)] + [[j, w] for w in range(prob.N)])
        Jr = oracle.ewald_J_entries(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut, rows)
        Ji, Jj = Jr[:prob.N], Jr[prob.N:]
        phi_i, phi_j = Ji @ q, Jj @ q
        d = q[j] - q[i]
        dE = 2 * d * (phi_i - phi_j) + d * d * (Ji[i] + Jj[j] - 2 * Ji[j])
        assert E2[b] - E1[b] == pytest.approx(dE, rel=1e-8, abs=1e-9 * abs(E1[b]))
    untouched = np.setdiff1d(np.arange(B), [s[0] for s in samples])
    assert np.array_equal(E1[untouched], E2[untouched])
    # the BF16x3 form tracks the FP64 path at full size
    Jh = Jg.cpu().numpy()
    R = quad_scale(Jh, prob, pop[:8])
    tol = form_tolerance("bf16x3", R, prob.Nv)
    assert np.all(np.abs(Et1[:8] - E1[:8]) <= tol)


@pytest.mark.parametrize("which,B", [("rocksalt", 37), ("layered", 300), ("o3", 129), ("random300", 700)])
def test_score_exact_form(ctx, which, B):
    """Integer-digit split: |E_exact - E_oracle| <= sum_ij |q_i||q_j| 2^-47 max|J|
    (six 8-bit digits per 128-row panel I: each J' entry keeps a residual below
    2^(e_I - 48) <= 2^-46 max|J|)."""
    prob = {"rocksalt": lambda: synth.rocksalt_problem((2, 2, 2), 4.2),
            "layered": lambda: synth.layered_problem(reps=(3, 3, 1)),
            "o3": lambda: synth.o3_layered_problem((2, 2, 1)),
            "random300": lambda: _random_cell_problem(300, 9)}[which]()
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, B, 61)
    Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, pop)
    Eg = gp.score(torch.tensor(pop, device="cuda"), "exact").cpu().numpy()
    vidx = np.nonzero(prob.site_class >= 0)[0]
    qabs = np.abs(prob.z[pop]).sum(axis=1)
    bound = qabs ** 2 * 2.0 ** -47 * 2 * np.abs(Jo[np.ix_(vidx, vidx)]).max() + 1e-10 * np.abs(Eo)
    assert np.all(np.abs(Eg - Eo) <= bound), np.max(np.abs(Eg - Eo) / bound)
    assert np.max(np.abs(Eg - Eo) / np.abs(Eo)) <= 1e-10


def test_score_exact_full_size_matches_fp64_path(ctx):
    import paper_2409_08808_gb300 as g
    prob = synth.random_cubic_problem()
    J = g.build_ewald(ctx, prob.lattice, torch.tensor(prob.frac, device="cuda"), prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, J)
    pop = torch.tensor(synth.random_population(prob, 1000, 71), device="cuda")
    E64 = gp.score(pop, "f64")
    Eex = gp.score(pop, "exact")
    assert ((Eex - E64).abs() / E64.abs()).max().item() <= 1e-11


@pytest.mark.parametrize("form", ["bf16x2", "f64"])
def test_score_host_matches_device_path(ctx, form):
    """The blocking host entry point with 3,000 configurations: the same
    energies as the device entry point, bit for bit, from pinned and from
    pageable host memory."""
    prob = synth.layered_problem(reps=(3, 3, 1))
    Jg, _ = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    pop = synth.random_population(prob, 3000, 55)
    Ed = gp.score(torch.tensor(pop, device="cuda"), form).cpu().numpy()
    assert np.array_equal(gp.score_host(pop, form), Ed)
    pinned = torch.tensor(pop).pin_memory()
    assert np.array_equal(gp.score_host(pinned, form).numpy(), Ed)


def test_score_host_async_pipeline(ctx):
    """Pipelined host-buffer scoring: a stream of populations of different sizes
    (the staging slots grow mid-stream) gives, after one synchronisation, the
    energies of the device-buffer entry point bit for bit, and the F64 ones
    match the oracle."""
    prob = synth.layered_problem(reps=(3, 3, 1))
    Jg, Jo = build_pair(ctx, prob)
    gp = gpu_problem(ctx, prob, Jg)
    sizes = [64, 300, 17, 513, 300, 1]
    forms = ["f64", "bf16x2", "f64", "exact", "tf32x2", "f64"]
    pops = [torch.tensor(synth.random_population(prob, B, 200 + i)).pin_memory() for i, B in enumerate(sizes)]
    outs = [torch.full((B,), float("nan"), dtype=torch.float64).pin_memory() for B in sizes]
    for p, o, f in zip(pops, outs, forms):
        gp.score_host_async(p, f, out=o)
    ctx.synchronize()
    for p, o, f in zip(pops, outs, forms):
        ref = gp.score(p.cuda(), f).cpu()
        assert torch.equal(o, ref), f
        if f == "f64":
            Eo = oracle.score(Jo, prob.site_class, prob.fixed_q, prob.z, p.numpy())
            assert np.max(np.abs(o.numpy() - Eo) / np.abs(Eo)) <= 1e-10

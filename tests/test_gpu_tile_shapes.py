"""Tile shapes of the tensor-core scoring kernels and their autotuner.

A tile covers 128 sites x 128 or 256 configurations, over the whole column
range of its row panel or over chunks of it (each chunk adds a partial row-dot
sum); every form also has 256-site tiles on CTA pairs with 256
configurations, and the exact form one CTA with 128 configurations on the
tensor-memory lanes (its pair-panel's first two k-blocks run as 128-site MMAs,
last).  The exact integer-digit form must give the same energies bit for bit in
every shape (its chunk partials are exact integers added exactly); the split
forms must stay within their derived bound of the oracle in every shape; the
autotuner's choice must be one of the shapes and be used afterwards."""
import numpy as np
import pytest
import torch

import goac_synth as synth
import oracle
from gpu_common import build_pair, form_tolerance, gpu_problem

pytestmark = pytest.mark.gpu

SHAPES = [(256, 0), (128, 0), (256, 16), (128, 8), (256, 4), (128, 2), (256, 1)]
# (tile_m, tile_n, ksplit) of the 256-site tiles (exact form only): the CTA-pair kernel (tile_n 256) and
# the configuration-lane kernel (tile_n 128; ksplit 1 makes each pair-panel's first chunk its two
# head k-blocks alone)
PAIR_SHAPES = [(256, 256, 0), (256, 256, 8), (256, 256, 1), (256, 128, 0), (256, 128, 8), (256, 128, 1)]


@pytest.fixture(scope="module")
def ctx():
    import paper_2409_08808_gb300 as g
    return g.Context(0)


@pytest.fixture(scope="module")
def cubic(ctx):
    import paper_2409_08808_gb300 as g
    prob = synth.random_cubic_problem(n_side=16)
    frac = torch.tensor(prob.frac, device="cuda")
    Jg = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
    return prob, gpu_problem(ctx, prob, Jg), Jg.cpu().numpy()


@pytest.mark.parametrize("B", [1000, 1024])
def test_exact_form_identical_in_every_shape(cubic, B):
    prob, gp, Jc = cubic
    pop = torch.tensor(synth.random_population(prob, B, 21), device="cuda")
    gp.score_set_shape(B, "exact", 0, 0)
    ref = gp.score(pop, "exact").clone()
    for tn, kc in SHAPES:
        gp.score_set_shape(B, "exact", tn, kc)
        E = gp.score(pop, "exact")
        assert torch.equal(E, ref), (tn, kc)
    for tm, tn, kc in PAIR_SHAPES:
        gp.score_set_shape(B, "exact", tn, kc, tile_m=tm)
        E = gp.score(pop, "exact")
        assert torch.equal(E, ref), (tm, tn, kc)
    gp.score_set_shape(B, "exact", 0, 0)
    rows = np.array([0, 1, B // 2, B - 1])
    Eo = oracle.score(Jc, prob.site_class, prob.fixed_q, prob.z, pop.cpu().numpy()[rows])
    assert np.max(np.abs(ref.cpu().numpy()[rows] - Eo) / np.abs(Eo)) <= 1e-10


@pytest.mark.parametrize("form", ["bf16x2", "bf16x3", "tf32x2"])
def test_split_forms_within_bound_in_every_shape(ctx, form):
    """Layered 12x12x1 cell (Nv = 864, seven 128-row panels), a ragged population."""
    import paper_2409_08808_gb300 as g
    prob = synth.layered_problem()
    frac = torch.tensor(prob.frac, device="cuda")
    Jg = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, Jg)
    Jc = Jg.cpu().numpy()
    B = 1061
    pop_np = synth.random_population(prob, B, 5)
    pop = torch.tensor(pop_np, device="cuda")
    rows = np.array([0, 127, 128, 255, 256, 700, 1023, 1024, B - 1])
    Eo = oracle.score(Jc, prob.site_class, prob.fixed_q, prob.z, pop_np[rows])
    q = [oracle.config_charges(prob.site_class, prob.fixed_q, prob.z, pop_np[r]) for r in rows]
    R = np.array([np.sqrt(((qq[:, None] * Jc * qq[None, :]) ** 2).sum()) for qq in q])
    tol = form_tolerance(form, R, prob.Nv)
    base = None
    for tn, kc in SHAPES:
        gp.score_set_shape(B, form, tn, kc)
        E = gp.score(pop, form).cpu().numpy()
        assert np.all(np.abs(E[rows] - Eo) <= tol), (tn, kc)
        if base is None:
            base = E
        elif kc == 0:
            # the same k-order per tile: only the configuration tiling differs
            assert np.array_equal(E, base), (tn, kc)
    # CTA pairs (256 sites x 256 configurations; the last pair-panel of this cell has one panel)
    for kc in (0, 8, 1):
        gp.score_set_shape(B, form, 256, kc, tile_m=256)
        E = gp.score(pop, form).cpu().numpy()
        assert np.all(np.abs(E[rows] - Eo) <= tol), (256, kc)
    gp.score_set_shape(B, form, 0, 0)


@pytest.mark.parametrize("form,B", [("exact", 512), ("bf16x3", 1024), ("bf16x2", 4096)])
def test_autotuner_choice(cubic, form, B):
    """The tuned shape is used afterwards: the exact form's energies are those
    of the default shape bit for bit; a split form's stay within its derived
    bound of the (FP64-grade) exact energies, as a k-split only regroups the
    FP32 accumulation."""
    prob, gp, Jc = cubic
    pop_np = synth.random_population(prob, B, 3)
    pop = torch.tensor(pop_np, device="cuda")
    gp.score_set_shape(B, form, 0, 0)
    ref = gp.score(pop, form).clone()
    tm, tn, kc, ms = gp.score_autotune(pop, form)
    assert tn in (128, 256) and kc in (0, 16, 8, 4, 2) and ms > 0
    assert tm == 128 or (tm == 256 and (form == "exact" or tn == 256))
    E = gp.score(pop, form)
    if form == "exact":
        assert torch.equal(E, ref)
    else:
        rows = np.linspace(0, B - 1, 16).astype(int)
        Ex = gp.score(pop, "exact").cpu().numpy()[rows]
        q2 = prob.z[pop_np[rows]] ** 2
        R = np.sqrt(np.einsum("bi,bi->b", q2, q2 @ (Jc * Jc)))
        tol = form_tolerance(form, R, prob.Nv)
        assert np.all(np.abs(E.cpu().numpy()[rows] - Ex) <= tol)
        assert np.all(np.abs(ref.cpu().numpy()[rows] - Ex) <= tol)
    gp.score_set_shape(B, form, 0, 0)


def test_set_shape_rejects_bad_shapes(cubic):
    import paper_2409_08808_gb300 as g
    _, gp, _ = cubic
    for args in [(0, "exact", 128, 0), (16, "exact", 64, 0), (16, "exact", 128, -1), (16, "f64", 128, 0),
                 (16, "f32", 0, 4)]:
        with pytest.raises(g.GoacError):
            gp.score_set_shape(*args)
    for kw in [dict(tile_m=64), dict(tile_m=256, tile_n=128, precision="tf32x2"),
               dict(tile_m=256, tile_n=128, precision="bf16x2")]:
        args = dict(B=16, precision="exact", tile_n=256, ksplit=0)
        args.update(kw)
        with pytest.raises(g.GoacError):
            gp.score_set_shape(**args)


def test_pair_kernel_odd_panel_count(ctx):
    """Layered 12x12x1 cell: Nv = 864 sites make seven 128-row panels, so the
    last pair-panel has no second panel (the CTA pair's odd CTA idles, the
    configuration-lane kernel runs 128-site MMAs); with fixed ions (a linear
    term) and a population whose last 128-configuration block is empty.  Every
    shape gives the default shape's exact energies."""
    import paper_2409_08808_gb300 as g
    prob = synth.layered_problem()
    frac = torch.tensor(prob.frac, device="cuda")
    Jg = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, Jg)
    B = 777
    pop_np = synth.random_population(prob, B, 12)
    pop = torch.tensor(pop_np, device="cuda")
    gp.score_set_shape(B, "exact", 0, 0)
    ref = gp.score(pop, "exact").clone()
    for tm, tn, kc in PAIR_SHAPES + [(128, 256, 2)]:
        gp.score_set_shape(B, "exact", tn, kc, tile_m=tm)
        assert torch.equal(gp.score(pop, "exact"), ref), (tm, tn, kc)
    gp.score_set_shape(B, "exact", 0, 0)
    rows = np.array([0, 255, 256, B - 1])
    Eo = oracle.score(Jg.cpu().numpy(), prob.site_class, prob.fixed_q, prob.z, pop_np[rows])
    assert np.max(np.abs(ref.cpu().numpy()[rows] - Eo) / np.abs(Eo)) <= 1e-10


def test_exact_form_split_epilogue(ctx):
    """Charges +49/16, +1, -1, -49/16 in counts 64, 192, 192, 64 on 512 sites
    (neutral): scaled to integers (x16) the largest is 49, so
    32 max|q|^2 2^9 Nv_pad >= 2^31 and the epilogue splits each integer sum in
    12-bit halves; the energies must still be identical in every shape and
    match the oracle to FP64 rounding."""
    import dataclasses
    prob = dataclasses.replace(synth.random_cubic_problem(n_side=8), z=np.array([49.0 / 16, 1.0, -1.0, -49.0 / 16]),
                               counts=np.array([[64, 192, 192, 64]], dtype=np.int32))
    import paper_2409_08808_gb300 as g
    frac = torch.tensor(prob.frac, device="cuda")
    Jg = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
    gp = gpu_problem(ctx, prob, Jg)
    assert gp.exact_info() == (10, 5, 4)
    B = 777
    pop = torch.tensor(synth.random_population(prob, B, 23), device="cuda")
    gp.score_set_shape(B, "exact", 0, 0)
    ref = gp.score(pop, "exact").clone()
    for tn, kc in SHAPES:
        gp.score_set_shape(B, "exact", tn, kc)
        assert torch.equal(gp.score(pop, "exact"), ref), (tn, kc)
    for tm, tn, kc in PAIR_SHAPES:
        gp.score_set_shape(B, "exact", tn, kc, tile_m=tm)
        assert torch.equal(gp.score(pop, "exact"), ref), (tm, tn, kc)
    gp.score_set_shape(B, "exact", 0, 0)
    rows = np.array([0, 255, 256, 511, 512, B - 1])
    Eo = oracle.score(Jg.cpu().numpy(), prob.site_class, prob.fixed_q, prob.z, pop.cpu().numpy()[rows])
    assert np.max(np.abs(ref.cpu().numpy()[rows] - Eo) / np.abs(Eo)) <= 1e-10

"""Failure detection without faulting a GPU: errors made on the host (bad
arguments, non-neutral charges, no device) and a device wait made to run out
(a barrier nothing arrives on) that the host reads back as a status."""
import ctypes as C

import numpy as np
import pytest
import torch

import goac_synth as synth


def test_ctx_create_without_device_fails_cleanly():
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2409_08808_gb300 import _lib
    h = C.c_void_p()
    rc = _lib.lib.goac_ctx_create(0, None, C.byref(h))
    assert rc != 0 and not h.value
    assert len(_lib.lib.goac_last_error()) > 0


def test_null_arguments_are_rejected_on_the_host():
    from paper_2409_08808_gb300 import _lib
    L = _lib.lib
    assert L.goac_score(None, None, 1, 0, None) == -1
    assert L.goac_mc_run(None, None, 1, None, 1, 0, 0, 0, None, None, None, None) == -1
    assert L.goac_ga_generation(None, None, None, 1, 0, 0, 0, 0, None, None, None) == -1
    assert L.goac_energy_grad(None, None, 1, 0.0, 0, None, None) == -1
    assert L.goac_round_to_counts(None, None, 1, None) == -1
    assert L.goac_score_f64_noalloc(None, 64, 10, None, 1, None, None, 0.0, None, None) == -1
    assert b"NULL" in L.goac_last_error()
    assert L.goac_ga_run_populations(None, None, None, 2, 8, 1, 0, 0, 0, 0, 0) == -1
    assert L.goac_mc_autotune(None, None, 4, None, 16, 0, None, None, None) == -1
    assert L.goac_topk_rescore(None, None, 8, None, 4, None, None) == -1


def test_empty_and_oversized_batches_on_the_host():
    """B = 0 returns GOAC_OK before any buffer is touched (its per-configuration
    pointers may be NULL); B < 0 or B > GOAC_MAX_BATCH = 2^31 - 256 is rejected.
    The allocation-free entry point needs no context, so this runs without a
    GPU: the non-NULL addresses below are never dereferenced."""
    import pathlib
    import re
    from paper_2409_08808_gb300 import _lib
    L = _lib.lib
    hdr = (pathlib.Path(__file__).resolve().parents[1] / "include" / "goac.h").read_text()
    assert int(re.search(r"#define GOAC_MAX_BATCH (\d+)", hdr).group(1)) == 2 ** 31 - 256
    fake = C.c_void_p(256)
    assert L.goac_score_f64_noalloc(fake, 64, 10, None, 0, fake, fake, 0.0, None, None) == 0
    for B in (-1, 2 ** 31 - 255):
        assert L.goac_score_f64_noalloc(fake, 64, 10, fake, B, fake, fake, 0.0, None, fake) == -1
    assert L.goac_score(None, None, 0, 0, None) == -1          # the problem handle is still required


@pytest.mark.gpu
def test_device_wait_runs_out_and_context_survives():
    import paper_2409_08808_gb300 as g
    from paper_2409_08808_gb300 import _lib
    ctx = g.Context(0)
    rc = _lib.lib.goac_selftest_wait_timeout(ctx.handle, 2_000_000)     # ~1 ms of SM clock
    assert rc == -5 and b"device error -5" in _lib.lib.goac_last_error()
    ctx.synchronize()                                                    # error word was cleared
    prob = synth.tiny_rocksalt_problem()
    J = g.build_ewald(ctx, prob.lattice, torch.tensor(prob.frac, device="cuda"), prob.alpha, prob.nimg, prob.kcut)
    gp = g.Problem(ctx, J, prob.site_class, prob.fixed_q, prob.z, prob.counts)
    E = gp.score(torch.tensor(synth.random_population(prob, 4, 1), device="cuda"), "bf16x3")
    assert torch.isfinite(E).all()
    ctx.synchronize()


@pytest.mark.gpu
def test_problem_validation_errors():
    import paper_2409_08808_gb300 as g
    ctx = g.Context(0)
    prob = synth.tiny_rocksalt_problem()
    J = g.build_ewald(ctx, prob.lattice, torch.tensor(prob.frac, device="cuda"), prob.alpha, prob.nimg, prob.kcut)
    with pytest.raises(g.GoacError) as e:
        g.Problem(ctx, J, prob.site_class, prob.fixed_q, prob.z, np.array([[5, 4]]))
    assert e.value.status == -1
    with pytest.raises(g.GoacError) as e:
        g.Problem(ctx, J, prob.site_class, prob.fixed_q + 0.5 * (prob.site_class < 0), prob.z, prob.counts)
    assert e.value.status == -4
    gp = g.Problem(ctx, J, prob.site_class, prob.fixed_q, prob.z, prob.counts)
    with pytest.raises(g.GoacError):
        gp.score(torch.zeros((2, gp.Nv), dtype=torch.int8, device="cuda"), 17)
    with pytest.raises(g.GoacError):
        gp.topk_rescore(torch.zeros((2, gp.Nv), dtype=torch.int8, device="cuda"),
                        torch.zeros(2, dtype=torch.float64, device="cuda"), 3)

"""The allocation-free FP64 scoring entry point (goac_score_f64_noalloc).

Some callers cannot allocate device memory themselves: their memory belongs to
a host framework's pool, or they run under a no-allocation rule once started.
This entry point takes only their buffers and keeps its scratch (the per-tile
partial energies) in a fixed array compiled into the library.  The test calls
it through the C ABI twice in a row on raw device buffers and compares each
result with the regular FP64 scoring entry point (goac_score, which allocates
its scratch), within the FP64 tolerance the other tests use (1e-10 relative).
"""
import ctypes as C

import numpy as np
import pytest
import torch

import goac_synth as synth

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_matches_score_twice():
    import paper_2409_08808_gb300 as g
    from paper_2409_08808_gb300 import _lib

    ctx = g.Context(0)
    prob = synth.layered_problem(reps=(3, 3, 1))          # fixed ions: phi_fix and E_const matter
    frac = torch.tensor(prob.frac, device="cuda")
    J = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
    gp = g.Problem(ctx, J, prob.site_class, prob.fixed_q, prob.z, prob.counts)
    Nv = gp.Nv
    ld = ((Nv + 63) // 64) * 64
    vidx = torch.tensor(np.nonzero(prob.site_class >= 0)[0], device="cuda")
    Jvv = torch.zeros((ld, ld), dtype=torch.float64, device="cuda")
    Jvv[:Nv, :Nv] = J[vidx][:, vidx]
    z = torch.zeros(64, dtype=torch.float64, device="cuda")
    z[:prob.S] = torch.tensor(prob.z, device="cuda")
    pf = torch.zeros(ld, dtype=torch.float64, device="cuda")
    pf[:Nv] = gp.phi_fix()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    for call, (B, seed) in enumerate([(300, 5), (517, 6)]):
        sp = torch.tensor(synth.random_population(prob, B, seed), device="cuda")
        E = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
        rc = _lib.lib.goac_score_f64_noalloc(_ptr(Jvv), ld, Nv, _ptr(sp), B, _ptr(z), _ptr(pf), gp.E_const, stream,
                                             _ptr(E))
        assert rc == 0, _lib.lib.goac_last_error()
        ref = gp.score(sp, "f64")
        torch.cuda.synchronize()
        rel = ((E - ref).abs() / ref.abs()).max().item()
        assert rel <= 1e-10, (call, rel)

    # the largest accepted call: ceil(Nv/64) * B equal to the array's 524,288 entries, so the last
    # configuration tile writes the array's last entry; a sample including that tile against the oracle
    import oracle
    mt = (Nv + 63) // 64
    B_max = 524288 // mt
    assert mt * B_max == 524288
    sp = torch.tensor(synth.random_population(prob, B_max, 7), device="cuda")
    E = torch.full((B_max,), float("nan"), dtype=torch.float64, device="cuda")
    rc = _lib.lib.goac_score_f64_noalloc(_ptr(Jvv), ld, Nv, _ptr(sp), B_max, _ptr(z), _ptr(pf), gp.E_const, stream,
                                         _ptr(E))
    assert rc == 0, _lib.lib.goac_last_error()
    torch.cuda.synchronize()
    rows = np.array([0, 1, B_max // 2, B_max - 65, B_max - 2, B_max - 1])
    Eo = oracle.score(J.cpu().numpy(), prob.site_class, prob.fixed_q, prob.z, sp.cpu().numpy()[rows])
    assert np.max(np.abs(E.cpu().numpy()[rows] - Eo) / np.abs(Eo)) <= 1e-10
    assert not torch.isnan(E).any()

    # sizes beyond the fixed scratch are rejected, nothing is launched
    big = torch.zeros((1, Nv), dtype=torch.int8, device="cuda")
    too_many = (524288 // ((Nv + 63) // 64)) + 1
    rc = _lib.lib.goac_score_f64_noalloc(_ptr(Jvv), ld, Nv, _ptr(big), too_many, _ptr(z), _ptr(pf), gp.E_const,
                                         stream, _ptr(E))
    assert rc == -1 and b"exceeds" in _lib.lib.goac_last_error()
    ctx.synchronize()

"""Helpers shared by the GPU parity tests (marshalling only)."""
import numpy as np
import torch

import goac_synth as synth
import oracle


def build_pair(ctx, prob):
    """GPU J (library) and oracle J (CPU) for the same synthetic problem."""
    import paper_2409_08808_gb300 as g
    frac = torch.tensor(prob.frac, dtype=torch.float64, device="cuda")
    Jg = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
    Jo = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
    return Jg, Jo


def gpu_problem(ctx, prob, Jg):
    import paper_2409_08808_gb300 as g
    return g.Problem(ctx, Jg, prob.site_class, prob.fixed_q, prob.z, prob.counts)


def quad_scale(Jo, prob, pop):
    """R_b = sqrt(sum_ij (q_i J_ij q_j)^2) per configuration (error model of the
    split tensor-core forms)."""
    out = []
    for b in range(pop.shape[0]):
        q = oracle.config_charges(prob.site_class, prob.fixed_q, prob.z, pop[b])
        out.append(float(np.sqrt(((q[:, None] * Jo * q[None, :]) ** 2).sum())))
    return np.array(out)


#: number of BF16 / TF32 terms of each split form and the bits each term carries
FORMS = {"bf16x2": (2, 8), "bf16x3": (3, 8), "tf32": (1, 11), "tf32x2": (2, 11)}


def form_tolerance(form, R, Nv):
    """|E_form - E_64| <= R (6 * 2^-(bits * terms) + gamma_K), K = terms * Nv.

    First term: each entry's split residual is at most 2^-(bits*terms)|J_ij|
    (every term keeps `bits` significant bits of the remainder); with
    independent signs the energy error has standard deviation at most
    2^-(bits*terms) R, and 6 of those bound it.  Second term: recursive FP32
    summation of the K products of one row has backward error |theta| <=
    gamma_K = K 2^-24 per product, which again contributes at most gamma_K R
    (measured coefficients on GB300: 0.08-0.25 for N = 512..4096)."""
    terms, bits = FORMS[form]
    K = terms * Nv
    return R * (6.0 * 2.0 ** (-bits * terms) + K * 2.0 ** -24)

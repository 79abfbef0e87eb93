"""CPU FP64 oracle for the Coulomb cluster-expansion optimiser (GOAC paper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2409_08808_gb300``);
neither imports the other.

The arithmetic lives in ``goac_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``).  This module only compiles it with gcc and marshals
numpy arrays through ctypes.  Every function cites the paper passage it follows
in the C source.  Functions without a pin would be marked "parity unpinned";
every function here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "goac_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build", platform.machine())
_LIB_PATH = os.path.join(_BUILD_DIR, "libgoac_oracle.so")
_lock = threading.Lock()
_lib = None

#: Coulomb constant e^2 / (4 pi eps0) in eV * Angstrom (CODATA 2018).  The
#: paper does not state the constant it uses.
KE = 14.3996454784


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` and return the path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            _declare(lib)
            _lib = lib
    return _lib


_d = C.c_double
_i64 = C.c_int64
_i32 = C.c_int32
_u32 = C.c_uint32
_u64 = C.c_uint64
_p = C.c_void_p


def _declare(lib):
    sig = {
        "orc_philox4x32_10": (None, [_p, _p, _p]),
        "orc_cell_geometry": (None, [_p, _p, _p]),
        "orc_frac_to_cart": (None, [_p, _p, _i64, _p]),
        "orc_count_kvectors": (C.c_int, [_p, _d]),
        "orc_ewald_J_entries": (C.c_int, [_p, _p, _i64, _d, _p, _d, _d, _p, _i64, _p]),
        "orc_ewald_J": (C.c_int, [_p, _p, _i64, _d, _p, _d, _d, _p]),
        "orc_ewald_energy": (_d, [_p, _p, _p, _i64, _d, _p, _d, _d]),
        "orc_qJq": (_d, [_p, _p, _i64]),
        "orc_config_charges": (None, [_i64, _p, _p, _p, _p, _p]),
        "orc_score": (None, [_p, _i64, _p, _p, _p, _p, _i64, _p]),
        "orc_fixed_split": (None, [_p, _i64, _p, _p, _p, _p]),
        "orc_ce_from_J": (None, [_p, _i64, _p, _p, _p, _i32, _p, _p, _p]),
        "orc_ce_from_substructures": (None, [_p, _p, _i64, _d, _p, _d, _d, _p, _p, _p, _i32, _p, _p, _p]),
        "orc_ce_energy": (_d, [_i64, _i32, _d, _p, _p, _p]),
        "orc_delta_E": (_d, [_p, _i64, _p, _i64, _i64, _d, _d]),
        "orc_random_configs": (C.c_int, [_i64, _p, _i32, _p, _i64, _u64, _p]),
        "orc_mc_run": (C.c_int, [_p, _i64, _p, _p, _p, _p, _i64, _p, _i64, _u64, _u64, _p, _p, _p, _p, _p]),
        "orc_sa_run": (C.c_int, [_p, _i64, _p, _p, _p, _p, _i64, _p, _p, _i64, _i64, _u64, _u64, _p, _p, _p, _p]),
        "orc_remc_run": (C.c_int, [_p, _i64, _p, _p, _p, _p, _i64, _i64, _p, _i64, _i64, _u64, _p, _p, _p]),
        "orc_gd_run": (C.c_int, [_p, _i64, _p, _p, _p, _p, _i64, _i64, _p, _p]),
        "orc_gd_run_literal": (C.c_int, [_p, _i64, _p, _p, _p, _p, _i64, _i64, _p, _p]),
        "orc_mc_run_literal": (C.c_int, [_p, _i64, _p, _p, _p, _p, _i64, _p, _i64, _u64, _u64, _p, _p, _p, _p,
                                         _p]),
        "orc_hybrid_run": (C.c_int, [_p, _i64, _p, _p, _p, _p, _i64, _i64, _p, _i64, _i64, _i64, _i64, _i64, _u32,
                                     _u64, _p]),
        "orc_ga_generation": (C.c_int, [_i64, _p, _p, _p, _i64, _i64, _u32, _u32, _u64, _p, _p, _p]),
        "orc_ga_run": (C.c_int, [_p, _i64, _p, _p, _p, _p, _p, _i64, _i64, _i64, _u32, _u64, _u32]),
        "orc_ga_run_ex": (C.c_int, [_p, _i64, _p, _p, _p, _p, _p, _i64, _i64, _i64, _u32, _u64, _u32, _i64, _p, _p,
                                    _p]),
        "orc_mc_run_ex": (C.c_int, [_p, _i64, _p, _p, _p, _p, _i64, _p, _i64, _u64, _u64, _i64, _p, _p, _p, _p, _p,
                                    _p, _p]),
        "orc_energy_grad": (_d, [_p, _i64, _p, _p, _p, _i32, _p, _p, _d, _p]),
        "orc_round_to_counts": (C.c_int, [_i64, _p, _i32, _p, _p, _p]),
        "orc_enumerate": (_i64, [_p, _i64, _p, _p, _p, _i32, _p, _d, _p, _p, _i64, _p, _p, _i64]),
        "orc_enumerate_two_species": (_i64, [_p, _i64, _p, _p, _p, _p, _d, _p, _p, _i64, _p]),
        "orc_log10_configurations": (_d, [_i32, _p, _i32, _p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32a(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i8(a):
    return np.ascontiguousarray(a, dtype=np.int8)


# --------------------------------------------------------------------------
# Wrappers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (SC'11 counter-based generator)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def cell_geometry(A):
    A = _f64(A).reshape(9)
    B = np.zeros(9)
    V = np.zeros(1)
    _load().orc_cell_geometry(_ptr(A), _ptr(B), _ptr(V))
    return B.reshape(3, 3), float(V[0])


def frac_to_cart(A, frac):
    A = _f64(A).reshape(9)
    f = _f64(frac).reshape(-1, 3)
    out = np.zeros_like(f)
    _load().orc_frac_to_cart(_ptr(A), _ptr(f), f.shape[0], _ptr(out))
    return out


def count_kvectors(A, kcut):
    return int(_load().orc_count_kvectors(_ptr(_f64(A).reshape(9)), kcut))


def ewald_J(A, frac, alpha, nimg, kcut, ke=KE):
    """Full N x N Ewald pair matrix (every entry by the definition)."""
    A = _f64(A).reshape(9)
    f = _f64(frac).reshape(-1, 3)
    n = f.shape[0]
    img = np.ascontiguousarray(nimg, dtype=np.int32)
    J = np.zeros((n, n))
    _load().orc_ewald_J(_ptr(A), _ptr(f), n, alpha, _ptr(img), kcut, ke, _ptr(J))
    return J


def ewald_J_entries(A, frac, alpha, nimg, kcut, pairs, ke=KE):
    """Selected J entries, pairs is (m, 2) int64 of (i, j)."""
    A = _f64(A).reshape(9)
    f = _f64(frac).reshape(-1, 3)
    pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    img = np.ascontiguousarray(nimg, dtype=np.int32)
    out = np.zeros(pr.shape[0])
    rc = _load().orc_ewald_J_entries(_ptr(A), _ptr(f), f.shape[0], alpha, _ptr(img), kcut, ke,
                                     _ptr(pr), pr.shape[0], _ptr(out))
    if rc:
        raise ValueError("pair index out of range")
    return out


def ewald_energy(A, frac, q, alpha, nimg, kcut, ke=KE):
    """Direct Ewald energy (structure-factor form, no J)."""
    A = _f64(A).reshape(9)
    f = _f64(frac).reshape(-1, 3)
    qq = _f64(q)
    img = np.ascontiguousarray(nimg, dtype=np.int32)
    return float(_load().orc_ewald_energy(_ptr(A), _ptr(f), _ptr(qq), f.shape[0], alpha, _ptr(img), kcut, ke))


def qJq(J, q):
    J = _f64(J)
    q = _f64(q)
    return float(_load().orc_qJq(_ptr(J), _ptr(q), q.shape[0]))


def config_charges(site_class, fixed_q, z, species_v):
    sc = _i32a(site_class)
    out = np.zeros(sc.shape[0])
    _load().orc_config_charges(sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(_i8(species_v)),
                               _ptr(out))
    return out


def score(J, site_class, fixed_q, z, species):
    """E_b = q_b^T J q_b for a population (B x Nv int8)."""
    J = _f64(J)
    sc = _i32a(site_class)
    sp = _i8(species)
    nv = int((sc >= 0).sum())
    B = sp.size // max(nv, 1)
    E = np.zeros(B)
    _load().orc_score(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(sp), B, _ptr(E))
    return E


def fixed_split(J, site_class, fixed_q):
    J = _f64(J)
    sc = _i32a(site_class)
    nv = int((sc >= 0).sum())
    phi = np.zeros(nv)
    ec = np.zeros(1)
    _load().orc_fixed_split(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(phi), _ptr(ec))
    return phi, float(ec[0])


def ce_from_J(J, site_class, fixed_q, z):
    J = _f64(J)
    sc = _i32a(site_class)
    zz = _f64(z)
    nv = int((sc >= 0).sum())
    S = zz.shape[0]
    alpha = np.zeros(nv * S)
    beta = np.zeros((nv * S) ** 2)
    ec = np.zeros(1)
    _load().orc_ce_from_J(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(zz), S, _ptr(ec), _ptr(alpha),
                          _ptr(beta))
    return float(ec[0]), alpha, beta


def ce_from_substructures(A, frac, alpha_ew, nimg, kcut, site_class, fixed_q, z, ke=KE):
    A = _f64(A).reshape(9)
    f = _f64(frac).reshape(-1, 3)
    sc = _i32a(site_class)
    zz = _f64(z)
    img = np.ascontiguousarray(nimg, dtype=np.int32)
    nv = int((sc >= 0).sum())
    S = zz.shape[0]
    alpha = np.zeros(nv * S)
    beta = np.zeros((nv * S) ** 2)
    ec = np.zeros(1)
    _load().orc_ce_from_substructures(_ptr(A), _ptr(f), f.shape[0], alpha_ew, _ptr(img), kcut, ke, _ptr(sc),
                                      _ptr(_f64(fixed_q)), _ptr(zz), S, _ptr(ec), _ptr(alpha), _ptr(beta))
    return float(ec[0]), alpha, beta


def ce_energy(nv, S, E_const, alpha, beta, species_v):
    return float(_load().orc_ce_energy(nv, S, E_const, _ptr(_f64(alpha)), _ptr(_f64(beta)), _ptr(_i8(species_v))))


def delta_E(J, phi_site, ia, ib, qa, qb):
    J = _f64(J)
    return float(_load().orc_delta_E(_ptr(J), J.shape[0], _ptr(_f64(phi_site)), ia, ib, qa, qb))


def random_configs(site_class, counts, B, seed):
    sc = _i32a(site_class)
    cnt = _i32a(counts)
    ncls = int(sc.max()) + 1
    S = cnt.size // max(ncls, 1)
    nv = int((sc >= 0).sum())
    out = np.zeros((B, nv), dtype=np.int8)
    rc = _load().orc_random_configs(sc.shape[0], _ptr(sc), S, _ptr(cnt), B, seed, _ptr(out))
    if rc:
        raise ValueError("counts do not match class sizes")
    return out


def mc_run(J, site_class, fixed_q, z, species, kT, nsteps, seed, step0=0, trace=False):
    """Metropolis swap MC, every chain in turn.  Returns a dict of outputs."""
    J = _f64(J)
    sc = _i32a(site_class)
    sp = np.array(species, dtype=np.int8, copy=True, order="C")
    Cn = sp.shape[0]
    nv = sp.shape[1]
    kTa = _f64(np.broadcast_to(np.asarray(kT, dtype=np.float64), (Cn,)))
    E = np.zeros(Cn)
    bestE = np.zeros(Cn)
    best = np.zeros_like(sp)
    nacc = np.zeros(Cn, dtype=np.int64)
    tr = np.zeros((Cn, nsteps)) if trace else None
    rc = _load().orc_mc_run(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(sp), Cn,
                            _ptr(kTa), nsteps, seed, step0, _ptr(E), _ptr(bestE), _ptr(best), _ptr(nacc), _ptr(tr))
    if rc:
        raise ValueError("no movable class")
    assert best.shape == (Cn, nv)
    return {"species": sp, "E": E, "bestE": bestE, "best_species": best, "n_accept": nacc, "E_trace": tr}


def mc_run_ex(J, site_class, fixed_q, z, species, kT, nsteps, seed, step0=0, patience=0):
    """mc_run with a patience (0: none) and per-chain statistics (n_noop,
    best_step, steps_done)."""
    J = _f64(J)
    sc = _i32a(site_class)
    sp = np.array(species, dtype=np.int8, copy=True, order="C")
    Cn = sp.shape[0]
    kTa = _f64(np.broadcast_to(np.asarray(kT, dtype=np.float64), (Cn,)))
    E = np.zeros(Cn)
    bestE = np.zeros(Cn)
    best = np.zeros_like(sp)
    out = {k: np.zeros(Cn, dtype=np.int64) for k in ("n_accept", "n_noop", "best_step", "steps_done")}
    rc = _load().orc_mc_run_ex(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(sp), Cn,
                               _ptr(kTa), nsteps, seed, step0, patience, _ptr(E), _ptr(bestE), _ptr(best),
                               _ptr(out["n_accept"]), _ptr(out["n_noop"]), _ptr(out["best_step"]),
                               _ptr(out["steps_done"]))
    if rc:
        raise ValueError("no movable class")
    out.update({"species": sp, "E": E, "bestE": bestE, "best_species": best})
    return out


def mc_run_literal(J, site_class, fixed_q, z, species, kT, nsteps, seed, step0=0):
    """Metropolis swap MC with the paper's rule taken literally (accept iff
    dE <= 0 or u < exp(-dE/kT), plain phi update): the twin that mc_run is
    checked against.  Also returns, per chain, the proposals with
    0 < dE <= 1e-9 eV (n_band) and those within 1e-9 of the exp/log boundary
    (n_close)."""
    J = _f64(J)
    sc = _i32a(site_class)
    sp = np.array(species, dtype=np.int8, copy=True, order="C")
    Cn = sp.shape[0]
    kTa = _f64(np.broadcast_to(np.asarray(kT, dtype=np.float64), (Cn,)))
    E = np.zeros(Cn)
    bestE = np.zeros(Cn)
    nacc = np.zeros(Cn, dtype=np.int64)
    nband = np.zeros(Cn, dtype=np.int64)
    nclose = np.zeros(Cn, dtype=np.int64)
    rc = _load().orc_mc_run_literal(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(sp),
                                    Cn, _ptr(kTa), nsteps, seed, step0, _ptr(E), _ptr(bestE), _ptr(nacc),
                                    _ptr(nband), _ptr(nclose))
    if rc:
        raise ValueError("no movable class")
    return {"species": sp, "E": E, "bestE": bestE, "n_accept": nacc, "n_band": nband, "n_close": nclose}


def sa_run(J, site_class, fixed_q, z, species, kT0, kT1, total, nsteps, seed, step0=0):
    """Simulated annealing (exponential kT schedule from kT0 to kT1 over `total` steps)."""
    J = _f64(J)
    sc = _i32a(site_class)
    sp = np.array(species, dtype=np.int8, copy=True, order="C")
    Cn = sp.shape[0]
    k0 = _f64(np.broadcast_to(np.asarray(kT0, dtype=np.float64), (Cn,)))
    k1 = _f64(np.broadcast_to(np.asarray(kT1, dtype=np.float64), (Cn,)))
    E = np.zeros(Cn)
    bestE = np.zeros(Cn)
    best = np.zeros_like(sp)
    nacc = np.zeros(Cn, dtype=np.int64)
    rc = _load().orc_sa_run(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(sp), Cn, _ptr(k0),
                            _ptr(k1), total, nsteps, seed, step0, _ptr(E), _ptr(bestE), _ptr(best), _ptr(nacc))
    if rc:
        raise ValueError("no movable class")
    return {"species": sp, "E": E, "bestE": bestE, "best_species": best, "n_accept": nacc}


def remc_run(J, site_class, fixed_q, z, species, G, R, kT_ladder, n_rounds, steps_per_round, seed):
    """Replica exchange: G groups of R chains, exchanges after every round."""
    J = _f64(J)
    sc = _i32a(site_class)
    sp = np.array(species, dtype=np.int8, copy=True, order="C")
    E = np.zeros(G * R)
    perm = np.zeros(G * R, dtype=np.int32)
    nex = np.zeros(1, dtype=np.int64)
    rc = _load().orc_remc_run(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(sp), G, R,
                              _ptr(_f64(kT_ladder)), n_rounds, steps_per_round, seed, _ptr(E), _ptr(perm), _ptr(nex))
    if rc:
        raise ValueError("remc failed")
    return {"species": sp, "E": E, "perm": perm, "n_exchanges": int(nex[0])}


def gd_run(J, site_class, fixed_q, z, species, max_steps):
    """Steepest descent over single swaps; returns final species, E and steps taken."""
    J = _f64(J)
    sc = _i32a(site_class)
    sp = np.array(species, dtype=np.int8, copy=True, order="C")
    Cn = sp.shape[0]
    E = np.zeros(Cn)
    st = np.zeros(Cn, dtype=np.int64)
    _load().orc_gd_run(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(sp), Cn, max_steps,
                       _ptr(E), _ptr(st))
    return {"species": sp, "E": E, "steps": st}


def gd_run_literal(J, site_class, fixed_q, z, species, max_steps):
    """Steepest descent with the literal rule (strict dE < 0, exact argmin,
    no tie band): the twin that gd_run is checked against."""
    J = _f64(J)
    sc = _i32a(site_class)
    sp = np.array(species, dtype=np.int8, copy=True, order="C")
    Cn = sp.shape[0]
    E = np.zeros(Cn)
    st = np.zeros(Cn, dtype=np.int64)
    _load().orc_gd_run_literal(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(sp), Cn,
                               max_steps, _ptr(E), _ptr(st))
    return {"species": sp, "E": E, "steps": st}


def hybrid_run(J, site_class, fixed_q, z, species, G, R, kT_ladder, n_cycles, n_rounds, steps_per_round, n_gen,
               n_elite, p_mut, seed):
    """REMC <-> GA alternation; returns final population and energies."""
    J = _f64(J)
    sc = _i32a(site_class)
    sp = np.array(species, dtype=np.int8, copy=True, order="C")
    E = np.zeros(G * R)
    rc = _load().orc_hybrid_run(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(sp), G, R,
                                _ptr(_f64(kT_ladder)), n_cycles, n_rounds, steps_per_round, n_gen, n_elite,
                                p_mut_to_u32(p_mut), seed, _ptr(E))
    if rc:
        raise ValueError("hybrid failed")
    return {"species": sp, "E": E}


def p_mut_to_u32(p_mut: float) -> int:
    """Mutation probability as the 32-bit threshold both sides compare with."""
    return int(min(max(p_mut, 0.0), 1.0) * 4294967295.0)


def ga_generation(site_class, pop, E, n_elite, p_mut, gen, seed):
    sc = _i32a(site_class)
    pp = _i8(pop)
    P, nv = pp.shape
    children = np.zeros_like(pp)
    parents = np.zeros((P, 2), dtype=np.int32)
    nsw = np.zeros((P, 2), dtype=np.int32)
    rc = _load().orc_ga_generation(sc.shape[0], _ptr(sc), _ptr(pp), _ptr(_f64(E)), P, n_elite, p_mut_to_u32(p_mut),
                                   gen, seed, _ptr(children), _ptr(parents), _ptr(nsw))
    if rc:
        raise ValueError(f"ga_generation failed rc={rc}")
    return children, parents, nsw


def ga_run(J, site_class, fixed_q, z, pop, n_gen, n_elite, p_mut, seed, gen0=0):
    J = _f64(J)
    sc = _i32a(site_class)
    pp = np.array(pop, dtype=np.int8, copy=True, order="C")
    P = pp.shape[0]
    E = np.zeros(P)
    rc = _load().orc_ga_run(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(pp), _ptr(E), P,
                            n_gen, n_elite, p_mut_to_u32(p_mut), seed, gen0)
    if rc:
        raise ValueError(f"ga_run failed rc={rc}")
    return pp, E


def ga_run_ex(J, site_class, fixed_q, z, pop, n_gen, n_elite, p_mut, seed, gen0=0, patience=0):
    """ga_run with the no-improvement patience: returns (pop, E, generations
    run, generation of the last improvement, stopped by patience)."""
    J = _f64(J)
    sc = _i32a(site_class)
    pop = np.array(pop, dtype=np.int8, copy=True, order="C")
    E = np.zeros(pop.shape[0])
    g = np.zeros(1, np.int64)
    bg = np.zeros(1, np.int64)
    st = np.zeros(1, np.int32)
    rc = _load().orc_ga_run_ex(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)), _ptr(pop), _ptr(E),
                               pop.shape[0], n_gen, n_elite, p_mut_to_u32(p_mut), seed, gen0, patience, _ptr(g),
                               _ptr(bg), _ptr(st))
    if rc:
        raise ValueError("ga failed")
    return pop, E, int(g[0]), int(bg[0]), bool(st[0])


def energy_grad(J, site_class, fixed_q, z, counts, logits, lam):
    J = _f64(J)
    sc = _i32a(site_class)
    zz = _f64(z)
    L = _f64(logits)
    d = np.zeros_like(L)
    e = _load().orc_energy_grad(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(zz), zz.shape[0],
                                _ptr(_i32a(counts)), _ptr(L), lam, _ptr(d))
    return float(e), d


def round_to_counts(site_class, counts, p):
    sc = _i32a(site_class)
    pp = np.ascontiguousarray(p, dtype=np.float32)
    nv, S = pp.shape
    out = np.full(nv, -1, dtype=np.int8)
    rc = _load().orc_round_to_counts(sc.shape[0], _ptr(sc), S, _ptr(_i32a(counts)), _ptr(pp), _ptr(out))
    if rc:
        raise ValueError("rounding failed")
    return out


def enumerate_all(J, site_class, fixed_q, z, counts, tol=1e-9, max_argmin=4096, max_all=0):
    J = _f64(J)
    sc = _i32a(site_class)
    zz = _f64(z)
    nv = int((sc >= 0).sum())
    emin = np.zeros(1)
    amin = np.zeros((max_argmin, nv), dtype=np.int8)
    nmin = np.zeros(1, dtype=np.int64)
    allE = np.zeros(max(max_all, 1))
    total = _load().orc_enumerate(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(zz), zz.shape[0],
                                  _ptr(_i32a(counts)), tol, _ptr(emin), _ptr(amin), max_argmin, _ptr(nmin),
                                  _ptr(allE), max_all)
    k = int(min(nmin[0], max_argmin))
    return {"n_configs": int(total), "Emin": float(emin[0]), "argmin": amin[:k].copy(),
            "n_argmin": int(nmin[0]), "all_E": allE[:min(total, max_all)].copy() if max_all else None}


def enumerate_two_species(J, site_class, fixed_q, z, counts, tol=1e-9, max_argmin=4096):
    """Exhaustive minimum of a problem whose one movable class holds two
    species (orc_enumerate_two_species): every C(n, k) placement."""
    J = _f64(J)
    sc = _i32a(site_class)
    nv = int((sc >= 0).sum())
    emin = np.zeros(1)
    amin = np.zeros((max(max_argmin, 1), nv), dtype=np.int8)
    nmin = np.zeros(1, dtype=np.int64)
    total = _load().orc_enumerate_two_species(_ptr(J), sc.shape[0], _ptr(sc), _ptr(_f64(fixed_q)), _ptr(_f64(z)),
                                              _ptr(_i32a(np.asarray(counts).ravel())), tol, _ptr(emin), _ptr(amin),
                                              max_argmin, _ptr(nmin))
    if total < 0:
        raise ValueError("enumerate_two_species: needs one movable class holding two species")
    k = int(min(nmin[0], max_argmin))
    return {"n_configs": int(total), "Emin": float(emin[0]), "argmin": amin[:k].copy(), "n_argmin": int(nmin[0])}


def log10_configurations(positions, n_se):
    pos = _i32a(positions)
    nse = _i32a(n_se).reshape(pos.shape[0], -1)
    return float(_load().orc_log10_configurations(pos.shape[0], _ptr(pos), nse.shape[1], _ptr(nse)))

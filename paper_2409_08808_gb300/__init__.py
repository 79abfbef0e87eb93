"""GB300 (sm_103a) library for the pairwise Coulomb cluster-expansion optimiser
of "Optimization of Coulomb Energies in Gigantic Configurational Spaces of
Multi-Element Ionic Crystals" (GOAC).

This package is a thin binding over the C ABI of ``libgoac.so``
(``include/goac.h``): it turns torch CUDA tensors into device pointers, the
caller's current CUDA stream into the context stream, and status codes into
exceptions.  Every step of the computation runs in the library's CUDA kernels;
nothing here computes, and there is no CPU fallback.
"""
from __future__ import annotations

import atexit
import ctypes as C
import weakref

import numpy as np
import torch

from ._lib import lib, LIB_PATH, SIGNATURES, GaParams, GaStats, McStats  # noqa: F401  (raises if missing)

#: Coulomb constant e^2 / (4 pi eps0) in eV * Angstrom (CODATA 2018).
KE = 14.3996454784

PREC = {"f64": 0, "tf32": 1, "tf32x2": 2, "bf16x2": 3, "bf16x3": 4, "f32": 5, "exact": 6, "f64_incr": 7, "f16x2": 8}


class GoacError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str | None = None):
        if msg is None:
            msg = lib.goac_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


#: status of a call on a closed context or problem (GOAC_ERR_INVALID_ARG)
_ERR_INVALID_ARG = -1


def _check(rc: int, where: str):
    if rc != 0:
        raise GoacError(rc, where)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous array")
        return C.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


class Context:
    """A library context on one GPU, enqueuing on torch's current stream."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        h = C.c_void_p()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        _check(lib.goac_ctx_create(self.device, C.c_void_p(stream), C.byref(h)), "goac_ctx_create")
        self._h = h
        self._problems = weakref.WeakSet()
        self._inflight = []      # host tensors of enqueued asynchronous copies
        _live_contexts.add(self)

    @property
    def handle(self):
        self.sync_stream()
        return self._h

    @property
    def closed(self) -> bool:
        return not getattr(self, "_h", None)

    def _live(self, where: str):
        if self.closed:
            raise GoacError(_ERR_INVALID_ARG, where, "the context is closed")
        return self._h

    def sync_stream(self):
        """Point the context at torch's current stream of its device."""
        h = self._live("goac_ctx_set_stream")
        stream = torch.cuda.current_stream(self.device).cuda_stream
        _check(lib.goac_ctx_set_stream(h, C.c_void_p(stream)), "goac_ctx_set_stream")

    def synchronize(self):
        _check(lib.goac_ctx_synchronize(self.handle), "goac_ctx_synchronize")
        self._inflight.clear()

    KERNELS = {"score_tc": 0, "score_cc": 1, "mc": 2, "ga": 3, "ewald_real": 4, "ewald_syrk": 5, "ga_incr": 6}

    def set_timing(self, enable: bool):
        _check(lib.goac_ctx_set_timing(self._live("goac_ctx_set_timing"), int(bool(enable))), "goac_ctx_set_timing")

    def kernel_time(self, kernel: str):
        """(total ms, launches) of a timed kernel family since the last query."""
        ms = C.c_double()
        n = C.c_int64()
        _check(lib.goac_ctx_kernel_time(self._live("goac_ctx_kernel_time"), self.KERNELS[kernel], C.byref(ms),
                                        C.byref(n)), "goac_ctx_kernel_time")
        return float(ms.value), int(n.value)

    def close(self):
        """Destroy every problem created on this context, then the context
        (goac_problem_destroy, goac_ctx_destroy); their device memory is
        freed.  Closing twice is a no-op; any later use raises GoacError."""
        if self.closed:
            return
        for p in list(getattr(self, "_problems", ())):
            p.close()
        h, self._h = self._h, None
        _live_contexts.discard(self)
        _check(lib.goac_ctx_destroy(h), "goac_ctx_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by libgoac in this process so far."""
    return int(lib.goac_launch_count())


_live_contexts = weakref.WeakSet()


@atexit.register
def _close_all():
    for c in list(_live_contexts):
        try:
            c.close()
        except Exception:
            pass


def build_ewald(ctx: Context, lattice, frac: torch.Tensor, alpha: float, nimg, kcut: float, ke: float = KE,
                out: torch.Tensor | None = None) -> torch.Tensor:
    """Ewald pair matrix J (N x N FP64 on the device); see goac_build_ewald."""
    lat = np.ascontiguousarray(lattice, dtype=np.float64).reshape(9)
    img = np.ascontiguousarray(nimg, dtype=np.int32).reshape(3)
    frac = frac.to(device=f"cuda:{ctx.device}", dtype=torch.float64).contiguous()
    N = frac.shape[0]
    J = out if out is not None else torch.empty((N, N), dtype=torch.float64, device=frac.device)
    _check(lib.goac_build_ewald(ctx.handle, _ptr(lat), _ptr(frac), N, float(alpha), _ptr(img), float(kcut),
                                float(ke), _ptr(J)), "goac_build_ewald")
    return J


class Problem:
    """Eq. 2 problem on the device (J_vv, phi_fix, E_const, classes, counts)."""

    def __init__(self, ctx: Context, J: torch.Tensor, site_class, fixed_q, z, counts, allow_charged: bool = False):
        self.ctx = ctx
        sc = np.ascontiguousarray(site_class, dtype=np.int32)
        fq = np.ascontiguousarray(fixed_q, dtype=np.float64)
        zz = np.ascontiguousarray(z, dtype=np.float64)
        cnt = np.ascontiguousarray(counts, dtype=np.int32)
        self.S = int(zz.shape[0])
        self.n_class = int(cnt.size // self.S)
        self.N = int(sc.shape[0])
        h = C.c_void_p()
        _check(lib.goac_problem_create(ctx.handle, _ptr(J), self.N, _ptr(sc), _ptr(fq), _ptr(zz), self.S, _ptr(cnt),
                                       self.n_class, int(bool(allow_charged)), C.byref(h)), "goac_problem_create")
        self._h = h
        ctx._problems.add(self)
        nv = C.c_int32()
        ec = C.c_double()
        _check(lib.goac_problem_info(h, C.byref(nv), C.byref(ec)), "goac_problem_info")
        self.Nv = int(nv.value)
        self.E_const = float(ec.value)

    @property
    def handle(self):
        if not getattr(self, "_h", None):
            raise GoacError(_ERR_INVALID_ARG, "goac_problem", "the problem is closed")
        self.ctx.sync_stream()
        return self._h

    def exact_info(self):
        """(digit bits r, digits T, charge scaling kq) of the exact form on this
        problem, or None when its charges do not admit it."""
        r, T, kq = C.c_int32(), C.c_int32(), C.c_int32()
        rc = lib.goac_problem_exact_info(self.handle, C.byref(r), C.byref(T), C.byref(kq))
        if rc == -7:
            return None
        _check(rc, "goac_problem_exact_info")
        return int(r.value), int(T.value), int(kq.value)

    def phi_fix(self) -> torch.Tensor:
        out = torch.empty(self.Nv, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        _check(lib.goac_problem_phi_fix(self.handle, _ptr(out)), "goac_problem_phi_fix")
        return out

    def close(self):
        """Free the problem's device memory (goac_problem_destroy).  A problem
        whose context was closed first was already destroyed with it."""
        h = getattr(self, "_h", None)
        if not h:
            return
        self._h = None
        ctx = getattr(self, "ctx", None)
        if ctx is not None and not ctx.closed:
            ctx._problems.discard(self)
            _check(lib.goac_problem_destroy(h), "goac_problem_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self):
        return f"cuda:{self.ctx.device}"

    # ---- scoring --------------------------------------------------------
    def score(self, species: torch.Tensor, precision="f64", out: torch.Tensor | None = None) -> torch.Tensor:
        B = species.shape[0]
        E = out if out is not None else torch.empty(B, dtype=torch.float64, device=self._dev())
        _check(lib.goac_score(self.handle, _ptr(species), B, _prec(precision), _ptr(E)), "goac_score")
        return E

    def score_set_shape(self, B: int, precision="bf16x2", tile_n: int = 0, ksplit: int = 0, tile_m: int = 0):
        """Tile shape for scoring B configurations in a tensor-core form (all 0 = default;
        tile_m 256: CTA pairs with tile_n 256 for every form, one CTA with the
        configurations on the tensor-memory lanes with tile_n 128 for the exact
        form)."""
        _check(lib.goac_score_set_shape(self.handle, _prec(precision), int(B), int(tile_m), int(tile_n), int(ksplit)),
               "goac_score_set_shape")

    def score_autotune(self, species: torch.Tensor, precision="bf16x2"):
        """Time the scoring tile shapes on `species` and keep the fastest for this
        (precision, padded B).  Returns (tile_m, tile_n, ksplit, ms per call)."""
        tm, tn, kc, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        _check(lib.goac_score_autotune(self.handle, _ptr(species), species.shape[0], _prec(precision), C.byref(tm),
                                       C.byref(tn), C.byref(kc), C.byref(ms)), "goac_score_autotune")
        return int(tm.value), int(tn.value), int(kc.value), float(ms.value)

    def score_host(self, species: np.ndarray | torch.Tensor, precision="f64", out=None):
        """End-to-end scoring from host memory (pinned torch tensors are fastest)."""
        if isinstance(species, torch.Tensor):
            assert not species.is_cuda and species.is_contiguous()
            sp_ptr = C.c_void_p(species.data_ptr())
            B = species.shape[0]
            E = out if out is not None else torch.empty(B, dtype=torch.float64, pin_memory=True)
            e_ptr = C.c_void_p(E.data_ptr())
        else:
            species = np.ascontiguousarray(species, dtype=np.int8)
            sp_ptr = _ptr(species)
            B = species.shape[0]
            E = out if out is not None else np.empty(B, dtype=np.float64)
            e_ptr = _ptr(E)
        _check(lib.goac_score_host(self.handle, sp_ptr, B, _prec(precision), e_ptr), "goac_score_host")
        return E

    def score_host_async(self, species: torch.Tensor, precision="f64", out: torch.Tensor | None = None):
        """Pipelined end-to-end scoring: enqueue the copy of `species` (pinned
        host int8 tensor, B x Nv) to the device, the scoring and the copy of
        the energies into `out` (pinned host float64 tensor), and return at
        once.  Calls alternate two device staging slots, so the copy of the
        next population overlaps the scoring of this one.  `species` must stay
        unchanged and `out` unread until ctx.synchronize()."""
        assert isinstance(species, torch.Tensor) and not species.is_cuda and species.is_contiguous()
        assert species.dtype == torch.int8 and species.dim() == 2 and species.shape[1] == self.Nv
        B = species.shape[0]
        E = out if out is not None else torch.empty(B, dtype=torch.float64, pin_memory=True)
        assert not E.is_cuda and E.dtype == torch.float64 and E.numel() >= B and E.is_contiguous()
        _check(lib.goac_score_host_async(self.handle, C.c_void_p(species.data_ptr()), B, _prec(precision),
                                         C.c_void_p(E.data_ptr())), "goac_score_host_async")
        self.ctx._inflight.append((species, E))
        return E

    def topk_rescore(self, species: torch.Tensor, E_approx: torch.Tensor, k: int):
        idx = torch.empty(k, dtype=torch.int32, device=self._dev())
        E = torch.empty(k, dtype=torch.float64, device=self._dev())
        _check(lib.goac_topk_rescore(self.handle, _ptr(species), species.shape[0], _ptr(E_approx), int(k), _ptr(idx),
                                     _ptr(E)), "goac_topk_rescore")
        return idx, E

    def random_configs(self, B: int, seed: int) -> torch.Tensor:
        out = torch.empty((B, self.Nv), dtype=torch.int8, device=self._dev())
        _check(lib.goac_random_configs(self.handle, int(B), int(seed), _ptr(out)), "goac_random_configs")
        return out

    # ---- Monte Carlo ----------------------------------------------------
    def mc_run(self, species: torch.Tensor, kT, n_steps: int, seed: int, step0: int = 0, precision="f64",
               want_best_species: bool = True):
        """Runs in place on `species` (C x Nv int8).  Returns a dict of device tensors."""
        Cn = species.shape[0]
        dev = self._dev()
        kTt = torch.as_tensor(kT, dtype=torch.float64, device=dev).expand(Cn).contiguous()
        E = torch.empty(Cn, dtype=torch.float64, device=dev)
        bestE = torch.empty(Cn, dtype=torch.float64, device=dev)
        best = torch.empty_like(species) if want_best_species else None
        nacc = torch.empty(Cn, dtype=torch.int64, device=dev)
        _check(lib.goac_mc_run(self.handle, _ptr(species), Cn, _ptr(kTt), int(n_steps), int(seed), int(step0),
                               _prec(precision), _ptr(E), _ptr(bestE), _ptr(best), _ptr(nacc)), "goac_mc_run")
        return {"species": species, "E": E, "bestE": bestE, "best_species": best, "n_accept": nacc}

    def mc_run_ex(self, species: torch.Tensor, kT, n_steps: int, seed: int, step0: int = 0, precision="f64",
                  patience: int = 0, want_best_species: bool = True):
        """mc_run with a no-improvement patience (0: none) and per-chain statistics:
        n_accept, n_noop, best_step (step0 - 1: the start), steps (steps run)."""
        Cn = species.shape[0]
        dev = self._dev()
        kTt = torch.as_tensor(kT, dtype=torch.float64, device=dev).expand(Cn).contiguous()
        E = torch.empty(Cn, dtype=torch.float64, device=dev)
        bestE = torch.empty(Cn, dtype=torch.float64, device=dev)
        best = torch.empty_like(species) if want_best_species else None
        st = {k: torch.empty(Cn, dtype=torch.int64, device=dev) for k in ("n_accept", "n_noop", "best_step", "steps")}
        ms = McStats(st["n_accept"].data_ptr() if Cn else None, st["n_noop"].data_ptr() if Cn else None,
                     st["best_step"].data_ptr() if Cn else None, st["steps"].data_ptr() if Cn else None)
        _check(lib.goac_mc_run_ex(self.handle, _ptr(species), Cn, _ptr(kTt), int(n_steps), int(seed), int(step0),
                                  _prec(precision), int(patience), _ptr(E), _ptr(bestE), _ptr(best), C.byref(ms)),
               "goac_mc_run_ex")
        out = {"species": species, "E": E, "bestE": bestE, "best_species": best}
        out.update(st)
        return out

    def mc_autotune(self, species: torch.Tensor, kT, probe_steps: int = 256, precision="f64"):
        """Time the Monte Carlo launch shapes on a copy of `species` and keep the fastest for
        later runs of this problem.  Returns (warps per chain, chains per CTA, probe ms)."""
        Cn = species.shape[0]
        kTt = torch.as_tensor(kT, dtype=torch.float64, device=self._dev()).expand(Cn).contiguous()
        W, c, ms = C.c_int32(), C.c_int32(), C.c_double()
        _check(lib.goac_mc_autotune(self.handle, _ptr(species), Cn, _ptr(kTt), int(probe_steps), _prec(precision),
                                    C.byref(W), C.byref(c), C.byref(ms)), "goac_mc_autotune")
        return int(W.value), int(c.value), float(ms.value)

    def mc_set_shape(self, W: int = 0, chains_per_cta: int = 0, precision="f64"):
        """Fix the Monte Carlo launch shape (warps per chain, chains per CTA); 0 = by size."""
        _check(lib.goac_mc_set_shape(self.handle, _prec(precision), int(W), int(chains_per_cta)),
               "goac_mc_set_shape")

    def gd_run(self, species: torch.Tensor, max_steps: int):
        """Steepest descent over single swaps, in place on `species`.  Returns (E, steps)."""
        B = species.shape[0]
        E = torch.empty(B, dtype=torch.float64, device=self._dev())
        steps = torch.empty(B, dtype=torch.int64, device=self._dev())
        _check(lib.goac_gd_run(self.handle, _ptr(species), B, int(max_steps), _ptr(E), _ptr(steps)), "goac_gd_run")
        return E, steps

    def sa_run(self, species: torch.Tensor, kT0, kT1, total_steps: int, n_steps: int, seed: int, step0: int = 0,
               precision="f64"):
        """Simulated annealing in place on `species` (exponential schedule kT0 -> kT1 over total_steps)."""
        Cn = species.shape[0]
        dev = self._dev()
        k0 = torch.as_tensor(kT0, dtype=torch.float64, device=dev).expand(Cn).contiguous()
        k1 = torch.as_tensor(kT1, dtype=torch.float64, device=dev).expand(Cn).contiguous()
        E = torch.empty(Cn, dtype=torch.float64, device=dev)
        bestE = torch.empty(Cn, dtype=torch.float64, device=dev)
        best = torch.empty_like(species)
        nacc = torch.empty(Cn, dtype=torch.int64, device=dev)
        _check(lib.goac_sa_run(self.handle, _ptr(species), Cn, _ptr(k0), _ptr(k1), int(total_steps), int(n_steps),
                               int(seed), int(step0), _prec(precision), _ptr(E), _ptr(bestE), _ptr(best), _ptr(nacc)),
               "goac_sa_run")
        return {"species": species, "E": E, "bestE": bestE, "best_species": best, "n_accept": nacc}

    def remc_run(self, species: torch.Tensor, G: int, R: int, kT_ladder, n_rounds: int, steps_per_round: int,
                 seed: int, precision="f64"):
        """Replica exchange in place on `species` (G R x Nv).  Returns (E, perm, n_exchanges)."""
        dev = self._dev()
        lad = np.ascontiguousarray(kT_ladder, dtype=np.float64)
        E = torch.empty(G * R, dtype=torch.float64, device=dev)
        perm = torch.empty(G * R, dtype=torch.int32, device=dev)
        nex = C.c_int64()
        _check(lib.goac_remc_run(self.handle, _ptr(species), int(G), int(R), _ptr(lad), int(n_rounds),
                                 int(steps_per_round), int(seed), _prec(precision), _ptr(E), _ptr(perm),
                                 C.byref(nex)), "goac_remc_run")
        return E, perm, int(nex.value)

    def hybrid_run(self, species: torch.Tensor, G: int, R: int, kT_ladder, n_cycles: int, n_rounds: int,
                   steps_per_round: int, n_gen: int, n_elite: int, p_mut_u32: int, seed: int, precision="f64"):
        """REMC <-> GA alternation in place on `species` (G R x Nv); returns final energies."""
        lad = np.ascontiguousarray(kT_ladder, dtype=np.float64)
        E = torch.empty(G * R, dtype=torch.float64, device=self._dev())
        _check(lib.goac_hybrid_run(self.handle, _ptr(species), int(G), int(R), _ptr(lad), int(n_cycles),
                                   int(n_rounds), int(steps_per_round), int(n_gen), int(n_elite), int(p_mut_u32),
                                   int(seed), _prec(precision), _ptr(E)), "goac_hybrid_run")
        return E

    # ---- genetic algorithm ----------------------------------------------
    def ga_generation(self, pop: torch.Tensor, E: torch.Tensor, n_elite: int, p_mut_u32: int, gen: int, seed: int,
                      record: bool = False):
        P = pop.shape[0]
        dev = self._dev()
        kids = torch.empty_like(pop)
        parents = torch.empty((P, 2), dtype=torch.int32, device=dev) if record else None
        nsw = torch.empty((P, 2), dtype=torch.int32, device=dev) if record else None
        _check(lib.goac_ga_generation(self.handle, _ptr(pop), _ptr(E), P, int(n_elite), int(p_mut_u32), int(gen),
                                      int(seed), _ptr(kids), _ptr(parents), _ptr(nsw)), "goac_ga_generation")
        return kids, parents, nsw

    def ga_run(self, pop: torch.Tensor, n_gen: int, n_elite: int, p_mut_u32: int, seed: int, gen0: int = 0,
               precision="f64"):
        """Runs in place on `pop` (P x Nv).  Returns the final energies."""
        P = pop.shape[0]
        E = torch.empty(P, dtype=torch.float64, device=self._dev())
        _check(lib.goac_ga_run(self.handle, _ptr(pop), _ptr(E), P, int(n_gen), int(n_elite), int(p_mut_u32),
                               int(seed), int(gen0), _prec(precision)), "goac_ga_run")
        return E

    def ga_run_ex(self, pop: torch.Tensor, n_gen: int, n_elite: int, p_mut_u32: int, seed: int, gen0: int = 0,
                  precision="f64", patience: int = 0, R: int = 1, time_budget_s: float = 0.0, topk: int = 0):
        """GA run(s) in place on `pop` (R P x Nv) with the run-level stops (patience,
        wall-clock budget) and the topk lowest of each final population rescored in
        FP64.  Returns a dict: E (R P), stats (list of R dicts), top_idx / top_E (R x topk)."""
        RP = pop.shape[0]
        assert R > 0 and RP % R == 0
        P = RP // R
        dev = self._dev()
        E = torch.empty(RP, dtype=torch.float64, device=dev)
        prm = GaParams(P, int(n_gen), int(n_elite), int(p_mut_u32), _prec(precision), int(patience), int(gen0),
                       float(time_budget_s))
        stats = (GaStats * R)()
        ti = torch.empty((R, topk), dtype=torch.int32, device=dev) if topk else None
        tE = torch.empty((R, topk), dtype=torch.float64, device=dev) if topk else None
        _check(lib.goac_ga_run_ex(self.handle, _ptr(pop), _ptr(E), int(R), C.byref(prm), int(seed), int(topk),
                                  _ptr(ti), _ptr(tE), stats), "goac_ga_run_ex")
        st = [{"generations": x.generations, "best_generation": x.best_generation, "stop_reason": x.stop_reason,
               "best_E": x.best_E} for x in stats]
        return {"E": E, "stats": st, "top_idx": ti, "top_E": tE}

    def ga_run_populations(self, pop: torch.Tensor, R: int, n_gen: int, n_elite: int, p_mut_u32: int, seed: int,
                           gen0: int = 0, precision="f64"):
        """R independent populations in place on `pop` (R P x Nv, population r in rows r P ...);
        population r evolves as ga_run with seed + r.  Returns the final energies (R P)."""
        RP = pop.shape[0]
        assert R > 0 and RP % R == 0
        E = torch.empty(RP, dtype=torch.float64, device=self._dev())
        _check(lib.goac_ga_run_populations(self.handle, _ptr(pop), _ptr(E), int(R), RP // R, int(n_gen), int(n_elite),
                                           int(p_mut_u32), int(seed), int(gen0), _prec(precision)),
               "goac_ga_run_populations")
        return E

    # ---- relaxed occupations --------------------------------------------
    def energy_grad(self, logits: torch.Tensor, lam: float, precision="f64", want_grad: bool = True):
        B = logits.shape[0]
        E = torch.empty(B, dtype=torch.float64, device=self._dev())
        g = torch.empty_like(logits) if want_grad else None
        _check(lib.goac_energy_grad(self.handle, _ptr(logits), B, float(lam), _prec(precision), _ptr(E), _ptr(g)),
               "goac_energy_grad")
        return E, g

    def relaxed_descent(self, logits: torch.Tensor, lam: float, eta: float, n_steps: int, precision="tf32x2"):
        """In-place projected descent on `logits` (B x Nv x S float); returns the final energies."""
        B = logits.shape[0]
        E = torch.empty(B, dtype=torch.float64, device=self._dev())
        scratch = torch.empty_like(logits)
        _check(lib.goac_relaxed_descent(self.handle, _ptr(logits), B, float(lam), float(eta), int(n_steps),
                                        _prec(precision), _ptr(scratch), _ptr(E)), "goac_relaxed_descent")
        return E

    def occupations(self, logits: torch.Tensor) -> torch.Tensor:
        """p = masked softmax of the logits (B x Nv x S float)."""
        p = torch.empty_like(logits)
        _check(lib.goac_occupations(self.handle, _ptr(logits), logits.shape[0], _ptr(p)), "goac_occupations")
        return p

    def round_to_counts(self, p: torch.Tensor) -> torch.Tensor:
        B = p.shape[0]
        out = torch.empty((B, self.Nv), dtype=torch.int8, device=self._dev())
        _check(lib.goac_round_to_counts(self.handle, _ptr(p), B, _ptr(out)), "goac_round_to_counts")
        return out


def batch_mc_run(ctx: Context, problems, species, kT, n_steps: int, seed: int, step0: int = 0, precision="f64",
                 chains_per_cta: int = 4, mode: int = 2):
    """Batched MC over independent problems (goac_batch_mc_run).  Returns (E, bestE) lists."""
    n = len(problems)
    dev = f"cuda:{ctx.device}"
    E = [torch.empty(s.shape[0], dtype=torch.float64, device=dev) for s in species]
    bE = [torch.empty(s.shape[0], dtype=torch.float64, device=dev) for s in species]
    P = (C.c_void_p * n)(*[p.handle.value for p in problems])
    SP = (C.c_void_p * n)(*[s.data_ptr() for s in species])
    CH = (C.c_int32 * n)(*[s.shape[0] for s in species])
    KT = (C.c_void_p * n)(*[t.data_ptr() for t in kT])
    EE = (C.c_void_p * n)(*[t.data_ptr() for t in E])
    BE = (C.c_void_p * n)(*[t.data_ptr() for t in bE])
    _check(lib.goac_batch_mc_run(ctx.handle, P, n, SP, CH, KT, int(n_steps), int(seed), int(step0), _prec(precision),
                                 EE, BE, int(chains_per_cta), int(mode)), "goac_batch_mc_run")
    return E, bE


def batch_ga_run(ctx: Context, problems, pops, n_gen: int, n_elite: int, p_mut_u32: int, seed: int, gen0: int = 0,
                 precision="f64_incr"):
    """GA populations of several problems (pops[i]: P_i x Nv_i int8, in place) in one
    launch per step (goac_batch_ga_run); population i evolves as ga_run with seed + i.
    Returns the final energies (list of tensors)."""
    n = len(problems)
    dev = f"cuda:{ctx.device}"
    E = [torch.empty(s.shape[0], dtype=torch.float64, device=dev) for s in pops]
    PR = (C.c_void_p * n)(*[p.handle.value for p in problems])
    SP = (C.c_void_p * n)(*[s.data_ptr() for s in pops])
    EE = (C.c_void_p * n)(*[t.data_ptr() for t in E])
    PP = (C.c_int32 * n)(*[s.shape[0] for s in pops])
    _check(lib.goac_batch_ga_run(ctx.handle, PR, n, SP, EE, PP, int(n_gen), int(n_elite), int(p_mut_u32), int(seed),
                                 int(gen0), _prec(precision)), "goac_batch_ga_run")
    return E


def batch_mc_autotune(ctx: Context, problems, species, kT, probe_steps: int = 256, precision="f64"):
    """Fastest chains-per-CTA for batch_mc_run on these problems (goac_batch_mc_autotune)."""
    n = len(problems)
    P = (C.c_void_p * n)(*[p.handle.value for p in problems])
    SP = (C.c_void_p * n)(*[s.data_ptr() for s in species])
    CH = (C.c_int32 * n)(*[s.shape[0] for s in species])
    KT = (C.c_void_p * n)(*[t.data_ptr() for t in kT])
    best = C.c_int32()
    ms = C.c_double()
    _check(lib.goac_batch_mc_autotune(ctx.handle, P, n, SP, CH, KT, int(probe_steps), _prec(precision),
                                      C.byref(best), C.byref(ms)), "goac_batch_mc_autotune")
    return int(best.value), float(ms.value)


class RelaxedEnergy(torch.autograd.Function):
    """E(logits) for relaxed occupations with the library's hand-written
    adjoint (goac_energy_grad) as the backward pass."""

    @staticmethod
    def forward(ctx, logits, problem, lam, precision):
        E, g = problem.energy_grad(logits.contiguous(), lam, precision, want_grad=True)
        ctx.save_for_backward(g)
        return E

    @staticmethod
    def backward(ctx, gE):
        (g,) = ctx.saved_tensors
        return g * gE.to(g.dtype).view(-1, 1, 1), None, None, None

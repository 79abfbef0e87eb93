#!/usr/bin/env python
"""Benchmark of the GOAC hot path on GB300.

One step = batched scoring E = q^T J q of a population of B = 4096 count-
preserving configurations of a random cubic cell with N = 4096 sites (16^3
jittered grid, species +1/+2/+3/-2), in the FP64-grade exact integer-digit form
on the tcgen05 tensor cores (energies within 1e-10 relative of the FP64
oracle).  value = energy evaluations per second over all GPUs.  The same run
also reports: the BF16x2 split form (throughput, roofline, energy error), the
plain FP64 GPU path on the same population and the speed-ups, the top-64 FP64
rescoring of the BF16x2 candidates, Monte Carlo swap trials/s at N = 4096 (FP64
and FP32 chains), the live roofline of the dominant kernel, the end-to-end
rate through the host-buffer entry point, and the CPU oracle on a bounded
sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one process per GPU): replicas; every rank scores its own
population (different seed), no data-path collective; value = all ranks' work
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "config energy evals/s and MC swap trials/s at N=4096, % roofline, vs FP64 GPU path"
N_SIDE = 16          # 16^3 = 4096 sites
B_POP = 4096
FORM = "exact"          # FP64-grade headline form
SECOND_FORM = "bf16x2"  # reported beside it with its own error and roofline
E2E_CELLS = 4          # cells scored round robin in the end-to-end leg
TERMS = {"bf16x2": 2, "bf16x3": 3, "tf32": 1, "tf32x2": 2}   # exact: digits per problem (exact_info)
WORKLOAD = ("random cubic cell N=4096 (16^3 grid, spacing 2.5 A, jitter 0.3 A; +1:512 +2:1024 +3:512 -2:2048), "
            "population B=4096 uniformly random count-preserving configurations")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", default=FORM, choices=sorted(TERMS))
    ap.add_argument("--mc-steps", type=int, default=4096)
    ap.add_argument("--tile", action="append", default=[],
                    help="FORM=M,N,K: fixed scoring tile shape for a form instead of the autotuner (profiling runs)")
    ap.add_argument("--mc-shapes", default="",
                    help="'W,c:W,c' fixed Monte Carlo launch shapes (FP64:FP32) instead of the autotuner")
    ap.add_argument("--cpu-sample", type=int, default=512, help="configurations the CPU oracle scores")
    ap.add_argument("--suite", action="store_true", help="measure the other workloads, one JSON line each")
    ap.add_argument("--only", default="mc,ga,batch,forms,relaxed,gd",
                    help="suite sections to run (comma separated: mc, ga, batch, forms, relaxed)")
    ap.add_argument("--batch-cells", type=int, default=256)
    ap.add_argument("--batch-chains", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=10000)
    ap.add_argument("--grad-batch", type=int, default=2048)
    ap.add_argument("--grad-steps", type=int, default=500)
    ap.add_argument("--paper", action="store_true", help="the paper's heuristics on its O3 and NaCl workloads")
    ap.add_argument("--paper-cells", default="2x2x1,2x2x2,4x4x1,4x4x2,6x6x1,8x8x1,6x6x2,6x6x3")
    ap.add_argument("--paper-chains", type=int, default=1024)
    ap.add_argument("--paper-steps", type=int, default=20000)
    ap.add_argument("--nacl-steps", type=int, default=12_500_000, help="swaps per chain on NaCl 3x3x3")
    ap.add_argument("--nacl-methods", default="MC,SA,REMC,GA,HY")
    ap.add_argument("--no-workloads", action="store_true",
                    help="default run: leave out the light runs of the other workloads")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------
def _dist():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [r[0] for r in rows]
        mx = max(r[1] for r in rows)
        load = [s for s in sm if s > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (the bounded baseline and the reference arm)
# ---------------------------------------------------------------------------
class _OracleWork:
    """Configurations of the benchmark cell scored by the oracle's plain
    q^T J q.  The oracle's J for N = 4096 takes minutes to build, and the
    scoring cost does not depend on J's values, so the timed sample uses a
    seeded symmetric FP64 matrix of the same size in its place."""

    def __init__(self, seed: int, max_cfg: int):
        import goac_synth as synth
        import oracle
        self.oracle = oracle
        oracle.build()
        self.prob = synth.random_cubic_problem(n_side=N_SIDE)
        rng = np.random.default_rng(seed)
        J = rng.standard_normal((self.prob.N, self.prob.N))
        self.J = np.ascontiguousarray(0.5 * (J + J.T))
        self.pop = synth.random_population(self.prob, max_cfg, seed + 1)

    def time(self, n_cfg: int, offset: int = 0, threads: int = 1) -> float:
        """Wall time of scoring n_cfg configurations with the oracle, split into
        `threads` contiguous chunks scored concurrently (the C routine is
        reentrant and ctypes releases the GIL during the call)."""
        from concurrent.futures import ThreadPoolExecutor
        p = self.prob
        idx = (offset + np.arange(n_cfg)) % self.pop.shape[0]
        sub = np.ascontiguousarray(self.pop[idx])
        chunks = [np.ascontiguousarray(c) for c in np.array_split(sub, max(1, min(threads, n_cfg))) if len(c)]
        t0 = time.perf_counter()
        if len(chunks) == 1:
            self.oracle.score(self.J, p.site_class, p.fixed_q, p.z, chunks[0])
        else:
            with ThreadPoolExecutor(len(chunks)) as ex:
                list(ex.map(lambda c: self.oracle.score(self.J, p.site_class, p.fixed_q, p.z, c), chunks))
        return time.perf_counter() - t0


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, world, rank):
    """The oracle as it stands, on this host's cores, as the reference arm.
    Each step scores a bounded sample sized so that warm-up + steps take about
    a minute in total."""
    if rank != 0:
        return
    cores = _host_cores()
    work = _OracleWork(11, B_POP)
    t1 = work.time(2 * cores, threads=cores) / (2.0 * cores)
    # each step scores the GPU arm's whole population (B = 4096) when warm-up + steps fit in
    # about two and a half minutes, else a contiguous sample of it
    per_step = int(max(1, min(B_POP, 150.0 / (max(1, args.steps + args.warmup) * t1))))
    for w in range(args.warmup):
        work.time(per_step, w, threads=cores)
    times = [work.time(per_step, k * per_step, threads=cores) for k in range(args.steps)]
    ms = 1e3 * float(np.mean(times))
    value = per_step / (ms / 1e3)
    sample = (f"{per_step} of the {B_POP} configurations per step of the N=4096 cell, oracle q^T J q in plain C, "
              f"{cores} threads; J a seeded symmetric FP64 matrix of the same size")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": 4096, "B": B_POP, "configs_scored_per_step": per_step,
                       "same_population_as_gpu_arm": per_step == B_POP, "form": "f64 oracle (CPU)",
                       "parallelism": f"{cores} host threads"},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("bf16_tflops"), d.get("hbm_gbs"), "measured"
    return 1900.0, 6800.0, "fallback"


def _kernel_hash(form="bf16x2") -> str:
    """Hash of the tensor-core scoring kernel's source for `form` (its function
    body and the device helpers of common.cuh it uses); ncu counters are valid
    while it is unchanged."""
    csrc = os.path.join(ROOT, "paper_2409_08808_gb300", "csrc")
    src = open(os.path.join(csrc, "score_tc.cu")).read()
    def template_of(name):
        # the template line that opens the kernel's definition (its launch bounds may change)
        return src.rindex("template <", 0, src.index(f"\n    {name}("))

    if form == "exact_pair":
        a = template_of("k_score_exact_pair")
        b = src.index("// Split forms (BF16 or TF32 terms) on CTA pairs")
    elif form.endswith("_pair"):
        a = src.index("// Split forms (BF16 or TF32 terms) on CTA pairs")
        b = src.index("// Exact form with the configurations on the tensor-memory lanes")
    elif form == "exact_ct":
        a = src.index("// Exact form with the configurations on the tensor-memory lanes")
        b = src.index("// Per 128-row panel I of the symmetric operand")
    elif form == "exact":
        a = template_of("k_score_exact")
        b = src.index("// Exact form on CTA pairs (tcgen05 cta_group::2)")
    else:
        a = src.index("template <int T, bool TF32, int TN>\n__global__ void __launch_bounds__(192, 1)")
        b = src.index("__device__ __forceinline__ float to_tf32_rna(")
    common = open(os.path.join(csrc, "common.cuh")).read()
    h = hashlib.sha256()
    h.update(src[a:b].encode())
    h.update(common[common.index("namespace goacd {"):common.index("}  // namespace goacd")].encode())
    return h.hexdigest()[:16]


def _traffic(form):
    """DRAM bytes per launch of the scoring kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"score_tc_{form}_n4096.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("kernel_sha") != _kernel_hash(form):
        return None
    return d.get("dram_bytes_per_launch")


def _time_form(gp, pop, form, steps, flush, E):
    """Per-step CUDA-event times (ms) of `steps` scoring calls, the L2 flushed
    between steps outside the step events; also the kernels launched."""
    import torch

    import paper_2409_08808_gb300 as g
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    launches0 = g.launch_count()
    for k in range(steps):
        flush.zero_()
        starts[k].record()
        gp.score(pop, form, out=E)
        ends[k].record()
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)], g.launch_count() - launches0


def _kernel_ms(ctx, gp, pop, form, steps, flush, E):
    """Average duration of the scoring kernel: the library's CUDA events around
    each launch, on the stream it is launched on, L2 flushed between steps."""
    import torch
    ctx.set_timing(True)
    ctx.kernel_time("score_tc")
    for _ in range(steps):
        flush.zero_()
        gp.score(pop, form, out=E)
    torch.cuda.synchronize()
    kern_ms, kern_n = ctx.kernel_time("score_tc")
    ctx.set_timing(False)
    return kern_ms / max(kern_n, 1), kern_n


def _exact_split(info, z, N):
    """Whether the exact kernel's epilogue splits its integer sums in 12-bit
    halves: the library does unless 32 max|q|^2 2^(r-1) Nv_pad < 2^31 (q the
    charges scaled to integers, r the digit width)."""
    r, _, kq = info
    qmax = max(abs(float(x)) for x in z) * 2.0 ** kq
    return not (32.0 * qmax * qmax * 2.0 ** (r - 1) * (((N + 127) // 128) * 128) < 2.0 ** 31)


def _roofline(form, terms, kern_ms, kern_n, N, B, tile_m=128, split=True, tile_n=256):
    ld = ((N + 127) // 128) * 128
    bpad = ((B + 255) // 256) * 256
    nbm = ld // 128
    pair = tile_m == 256 and tile_n == 256
    ct = form == "exact" and tile_m == 256 and tile_n == 128
    # upper block triangle of the symmetric operand: m-block I runs over columns 128 I .. ld; on CTA pairs
    # both panels of pair-panel P run from column 256 P (one block of zeros for the odd panel); the
    # configuration-lane kernel skips that block and covers the configurations in blocks of 128
    blocks = (sum(min(2, nbm - 2 * P) * (nbm - 2 * P) for P in range((nbm + 1) // 2)) if pair
              else nbm * (nbm + 1) // 2)
    ncfg = ((B + 127) // 128) * 128 if ct else bpad
    flops_exec = terms * 2.0 * 128 * 128 * blocks * ncfg
    flops_useful = 2.0 * N * N * B
    bf16_peak, _, peak_kind = _peaks()
    tf32 = "tf32" in form
    peak = bf16_peak / 2.0 if tf32 else bf16_peak     # TF32 runs at half the BF16 rate; FP16 = BF16
    achieved = flops_exec / (kern_ms / 1e3) / 1e12
    kernel = (f"k_score_exact_pair<{str(split).lower()}>" if pair else
              f"k_score_exact_ct<{str(split).lower()}>" if ct else
              f"k_score_exact<256, {str(split).lower()}>") if form == "exact" else \
        f"k_score_tc_pair<{terms},{'true' if tf32 else 'false'}>" if pair else \
        f"k_score_tc<{terms},{'true' if tf32 else 'false'},256>"
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": _traffic(f"{form}_pair" if pair else "exact_ct" if ct else form), "kernel": kernel,
            "kernel_ms": kern_ms,
            "kernel_timing": f"CUDA events around each launch, a second loop of {kern_n} steps (L2 flushed "
                             f"between steps)",
            "flops_per_launch": flops_exec, "useful_flops_per_launch": flops_useful,
            "useful_frac": flops_useful / (kern_ms / 1e3) / 1e12 / peak,
            "peak_kind": f"{peak_kind} bf16_tflops (burst)" + (" x 0.5 nominal tf32/bf16 ratio" if tf32 else
                                                              (", FP16 runs at the BF16 rate" if form == "exact"
                                                               else ""))}


def _mc_profile(prec):
    """DRAM bytes and duration of the Monte Carlo kernel from the committed ncu
    summary (profiles/mc_<prec>_n4096.json) if present, else None."""
    path = os.path.join(ROOT, "profiles", f"mc_{prec}_n4096.json")
    if not os.path.exists(path):
        return None
    return json.load(open(path))


def run_ours(args, world, rank, local):
    import torch

    import goac_synth as synth
    import paper_2409_08808_gb300 as g

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = g.Context(local)
    prob = synth.random_cubic_problem(n_side=N_SIDE)
    frac = torch.tensor(prob.frac, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
    torch.cuda.synchronize()
    ewald_ms = 1e3 * (time.perf_counter() - t0)
    gp = g.Problem(ctx, J, prob.site_class, prob.fixed_q, prob.z, prob.counts)
    del J
    pop_np = synth.random_population(prob, B_POP, synth.SEED_BASE + 2 + 1000 * rank)
    pop = torch.tensor(pop_np, device=dev)
    pop_host = torch.tensor(pop_np).pin_memory()
    form = args.form
    other = SECOND_FORM if form != SECOND_FORM else "exact"
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2
    info = gp.exact_info()
    terms = {f: (info[1] if f == "exact" else TERMS[f]) for f in (form, other)}

    # tile shapes of both forms from the library's autotuner (also builds the split operand copies),
    # or fixed by --tile
    fixed = {t.split("=")[0]: tuple(int(x) for x in t.split("=")[1].split(",")) for t in args.tile}
    shapes = {}
    for f in (form, other):
        if f in fixed:
            shapes[f] = fixed[f]
            gp.score_set_shape(B_POP, f, shapes[f][1], shapes[f][2], tile_m=shapes[f][0])
        else:
            shapes[f] = gp.score_autotune(pop, f)[:3]
    for _ in range(max(3, args.warmup)):
        gp.score(pop, form)
        gp.score(pop, other)
    torch.cuda.synchronize()

    # timed steps: only the two step events per step (no per-kernel events, which would
    # sit between the chained kernels of a step)
    E = torch.empty(B_POP, dtype=torch.float64, device=dev)
    clocks = ClockSampler(local)
    _barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    step_ms, launches = _time_form(gp, pop, form, args.steps, flush, E)
    _barrier(world)
    clk = clocks.stop()
    ms = _max_over_ranks(float(np.mean(step_ms)), world)
    value = world * B_POP / (ms / 1e3)

    # the dominant kernel's own duration: the same steps again with the library's
    # per-kernel CUDA events around the scoring kernel
    kern_ms, kern_n = _kernel_ms(ctx, gp, pop, form, min(args.steps, 400), flush, E)
    split = _exact_split(info, prob.z, prob.N)
    roofline = _roofline(form, terms[form], kern_ms, kern_n, prob.N, B_POP, shapes[form][0], split, shapes[form][1])

    # the other form (BF16x2 beside the FP64-grade headline): same timing, own roofline
    o_ms, _ = _time_form(gp, pop, other, min(args.steps, 400), flush, E)
    o_ms = _max_over_ranks(float(np.mean(o_ms)), world)
    o_kms, o_kn = _kernel_ms(ctx, gp, pop, other, min(args.steps, 400), flush, E)

    # End to end through the public host-buffer API: every step copies its
    # population from pinned host memory and its energies back, through the
    # pipelined entry point (the copy of step k+1 overlaps the scoring of step
    # k).  Inputs larger than L2 instead of a flush: E2E_CELLS different
    # N = 4096 cells (jitter seeds) are scored round robin, each step a fresh
    # population, so a cell's operands were last touched E2E_CELLS - 1 steps
    # (> 129 MB of traffic) earlier.
    cells = [gp]
    for c in range(1, E2E_CELLS):
        pc = synth.random_cubic_problem(n_side=N_SIDE, seed=synth.SEED_BASE + 2 + 97 * c)
        Jc = g.build_ewald(ctx, pc.lattice, torch.tensor(pc.frac, device=dev), pc.alpha, pc.nimg, pc.kcut)
        cells.append(g.Problem(ctx, Jc, pc.site_class, pc.fixed_q, pc.z, pc.counts))
        del Jc
    pops_host = [pop_host] + [torch.tensor(synth.random_population(prob, B_POP, synth.SEED_BASE + 3 + c + 1000 * rank))
                              .pin_memory() for c in range(1, 2 * E2E_CELLS)]
    E_hosts = [torch.empty(B_POP, dtype=torch.float64).pin_memory() for _ in range(2 * E2E_CELLS)]
    n_e2e = max(2 * E2E_CELLS, min(args.steps, 400) // (2 * E2E_CELLS) * (2 * E2E_CELLS))
    for k in range(2 * E2E_CELLS):
        cells[k % E2E_CELLS].score_host_async(pops_host[k], form, out=E_hosts[k])
    ctx.synchronize()
    _barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_e2e):
        j = k % (2 * E2E_CELLS)
        cells[j % E2E_CELLS].score_host_async(pops_host[j], form, out=E_hosts[j])
    ctx.synchronize()
    e2e_s = _max_over_ranks((time.perf_counter() - t0) / n_e2e, world)
    e2e_ok = all(bool(torch.equal(E_hosts[j], cells[j % E2E_CELLS].score(pops_host[j].to(dev), form).cpu()))
                 for j in range(2 * E2E_CELLS))
    for c in cells[1:]:
        c.close()
    del cells
    # the blocking entry point (copy, score, copy back, synchronise) for comparison
    E_host = E_hosts[0]
    e2e_t = []
    for k in range(min(args.steps, 200)):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        gp.score_host(pop_host, form, out=E_host)
        e2e_t.append(time.perf_counter() - t1)
    e2e_block_s = _max_over_ranks(float(np.mean(e2e_t)), world)
    e2e = {"value": world * B_POP / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": int(pop_np.nbytes),
           "d2h_bytes_per_step": int(E_host.numel() * 8), "api": "Problem.score_host_async (goac_score_host_async)",
           "steps": n_e2e, "energies_equal_device_path": e2e_ok,
           "l2": f"no flush: {E2E_CELLS} different N=4096 cells round robin, 8 host populations "
                 f"(one cell's operands + inputs ~85 MB; a {E2E_CELLS}-step cycle > 2x the 129 MB L2)",
           "blocking_api_value": world * B_POP / e2e_block_s,
           "blocking_api_l2": "256 MB flush between steps, outside the host timer"}

    # plain FP64 GPU path on the same population, and the error of each form against it
    E_form = gp.score(pop, form).clone()
    E_other = gp.score(pop, other).clone()
    E64 = gp.score(pop, "f64")
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    reps64 = 2
    for _ in range(reps64):
        gp.score(pop, "f64", out=E64)
    b.record()
    torch.cuda.synchronize()
    f64_ms = a.elapsed_time(b) / reps64

    def err_vs_fp64(Ef):
        err = (Ef - E64).abs()
        return {"max_abs_eV": float(err.max()), "rms_abs_eV": float(err.pow(2).mean().sqrt()),
                "max_rel": float((err / E64.abs()).max()), "mean_abs_E_eV": float(E64.abs().mean())}

    # top-64 FP64 rescoring of the BF16x2 form's best candidates
    E_bf = E_form if form == SECOND_FORM else E_other
    idx, Etop = gp.topk_rescore(pop, E_bf, 64)
    torch.cuda.synchronize()
    a.record()
    for _ in range(3):
        gp.topk_rescore(pop, E_bf, 64)
    b.record()
    torch.cuda.synchronize()
    topk_ms = a.elapsed_time(b) / 3
    top_exact = bool(torch.allclose(Etop, E64[idx.long()], rtol=1e-12, atol=0))
    same_best = int(idx[0].item()) == int(torch.argmin(E64).item())

    # Monte Carlo swap trials at N = 4096 (chains continue from a warm-up segment)
    mc = {}
    for prec in ("f64", "f32"):
        Cn = 152 * (6 if prec == "f64" else 8)
        chains = gp.random_configs(Cn, 77 + rank)
        if args.mc_shapes:                                        # fixed shapes (profiling runs)
            W_t, cpc_t = (int(x) for x in args.mc_shapes.split(":")[0 if prec == "f64" else 1].split(","))
            gp.mc_set_shape(W_t, cpc_t, prec)
        else:
            W_t, cpc_t, _ = gp.mc_autotune(chains, 0.05, 128, prec)  # launch shape for this cell
        gp.mc_run(chains, 0.05, args.mc_steps, 5, step0=0, precision=prec)
        torch.cuda.synchronize()
        ctx.set_timing(True)
        ctx.kernel_time("mc")
        a.record()
        out = gp.mc_run(chains, 0.05, args.mc_steps, 5, step0=args.mc_steps, precision=prec)
        b.record()
        torch.cuda.synchronize()
        mc_kms, _ = ctx.kernel_time("mc")
        ctx.set_timing(False)
        mms = a.elapsed_time(b)
        trials = Cn * args.mc_steps
        acc = float(out["n_accept"].sum().item()) / trials
        rb = 8 if prec == "f64" else 4
        # bytes per trial: J_ab gather (one 32-byte sector) + per acceptance two J rows
        bytes_alg = trials * 32 + acc * trials * 2 * prob.N * rb
        mc[prec] = {"trials_per_s": world * trials / (_max_over_ranks(mms, world) / 1e3), "chains": Cn,
                    "steps_per_chain": args.mc_steps, "kT_eV": 0.05, "acceptance": acc, "ms": mms,
                    "kernel_ms": mc_kms, "autotuned_warps_per_chain": W_t, "autotuned_chains_per_cta": cpc_t,
                    "algorithmic_gbs": bytes_alg / (mc_kms / 1e3) / 1e9,
                    "algorithmic_bytes_served_by": (f"mostly L2: the J rows of accepted swaps "
                                                    f"({prob.N * prob.N * rb / 1e6:.0f} MB of J in "
                                                    f"{'FP64' if rb == 8 else 'FP32'}) hit in the 129 MB L2, "
                                                    f"so this rate is not an HBM rate")}
        prof = _mc_profile(prec)
        if prof:
            mc[prec]["ncu_dram"] = {"bytes_per_launch": prof["dram_bytes_per_launch"],
                                    "gbs": prof["dram_bytes_per_launch"] / (prof["gpu_time_us_ncu"] * 1e-6) / 1e9,
                                    "workload": prof["workload"], "source": prof["source"]}
        if prec == "f64":
            # the FP64 chain is bound by the FP64 pipe: per accepted swap one subtract and one FMA
            # per site (the potential update); peak = 152 SMs x 2 FP64 FMA/clk x 2.07 GHz
            # (6.29e11 instr/s, the rate the FP64 SYRK reaches at 99 % FP64-pipe activity)
            fp64_instr = acc * trials * 2.0 * prob.N
            mc[prec]["bound"] = "fp64 pipe"
            mc[prec]["fp64_instr_per_s_update"] = fp64_instr / (mc_kms / 1e3)
            mc[prec]["fp64_pipe_frac_update"] = fp64_instr / (mc_kms / 1e3) / (152 * 2 * 2.07e9)
        else:
            mc[prec]["bound"] = "L2 / load latency (J rows of accepted swaps)"

    cpu = None
    if rank == 0:
        cores = _host_cores()
        n1 = max(1, args.cpu_sample // 4)
        work = _OracleWork(11, args.cpu_sample)
        dt1 = work.time(n1)
        n = args.cpu_sample
        dt = work.time(n, threads=cores)
        cpu = {"value": n / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} configurations of the N=4096 cell, oracle q^T J q in plain C, {cores} threads "
                         f"({dt:.1f} s), J a seeded symmetric FP64 matrix of the same size",
               "single_thread": {"value": n1 / dt1, "cores": 1, "sample": f"{n1} configurations ({dt1:.1f} s)"}}

    if rank == 0:
        if form == "exact":
            dtype = "exact-int/f64"
            detail = (f"exact integer digits: J' (symmetric operand) per 128-row panel in {info[1]} FP16 digits of "
                      f"{info[0]} bits ({info[0] * info[1]} bits), charges exact in FP16, digit sums exact integers "
                      f"in the FP32 tcgen05 accumulators, combined in FP64: FP64-grade (truncation <= 2^-{info[0] * info[1]}"
                      f" of each panel's largest |J'|; within 1e-10 relative of the FP64 oracle)")
        else:
            dtype = "bf16" if "bf16" in form else "tf32"
            detail = f"J split in {terms[form]} terms, Q exact, FP32 accumulate on tcgen05, FP64 cross-tile sums"
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": {"workload": WORKLOAD, "N": prob.N, "B": B_POP, "form": form, "form_detail": detail,
                           "tile_shape": {"sites": shapes[form][0], "configurations": shapes[form][1],
                                          "k_chunk_blocks": shapes[form][2],
                                          "chosen_by": "fixed (--tile)" if form in fixed else
                                          f"goac_score_autotune (CUDA events over "
                                          f"{(4 if form == 'exact' else 3) * sum(k < (prob.N + 127) // 128 for k in (0, 16, 8, 4, 2))} shapes)"},
                           "l2": "256 MB buffer written between steps (outside the step events)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk,
                "energy_error_vs_fp64": err_vs_fp64(E_form),
                other: {"value": world * B_POP / (o_ms / 1e3), "unit": "evals/s", "ms_per_step": o_ms,
                        "roofline": _roofline(other, terms[other], o_kms, o_kn, prob.N, B_POP, shapes[other][0], split,
                                              shapes[other][1]),
                        "tile_shape": {"sites": shapes[other][0], "configurations": shapes[other][1],
                                       "k_chunk_blocks": shapes[other][2]},
                        "energy_error_vs_fp64": err_vs_fp64(E_other), "speedup_over_fp64_path": f64_ms / o_ms},
                "fp64_gpu_path": {"evals_per_s": world * B_POP / (f64_ms / 1e3), "ms_per_step": f64_ms,
                                  "speedup_of_form": f64_ms / ms},
                "topk64_fp64_rescore": {"form": SECOND_FORM, "ms": topk_ms, "exact_vs_fp64_path": top_exact,
                                        "lowest_matches_fp64_argmin": same_best},
                "mc": mc, "setup": {"ewald_build_ms": ewald_ms}}
        if not args.no_workloads:
            # light runs of the other workloads (GA, gradient descent, the uneven batch of cells, the relaxed-
            # occupation gradient, the paper's O3 cells and NaCl), one dict each, timed with CUDA events
            t_w = time.perf_counter()
            light = argparse.Namespace(**vars(args))
            light.only, light.batch_steps, light.grad_steps = "mc,ga,gd,batch,relaxed", 2000, 100
            light.paper_cells, light.paper_steps, light.nacl_methods = "2x2x1,4x4x1,6x6x1", 20000, "SA"
            workloads = []
            run_suite(light, ctx, workloads)
            run_paper(light, ctx, workloads)
            line["workloads"] = workloads
            line["workloads_s"] = time.perf_counter() - t_w
        print(json.dumps(line), flush=True)


def run_suite(args, ctx=None, out=None):
    """One JSON line per workload of the build's configuration list (the
    scoring benchmark of the default run is not repeated): rocksalt MC parity
    run, layered-oxide GA, the uneven batch of cells (persistent / graph /
    per-problem launches, autotuned chains per CTA), the relaxed-occupation
    gradient at N = 8192, and Ewald build times."""
    import torch

    import goac_synth as synth
    import oracle
    import paper_2409_08808_gb300 as g

    ctx = ctx or g.Context(0)
    dev = torch.device("cuda", 0)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def timed(fn):
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def problem(prob, allow=False):
        frac = torch.tensor(prob.frac, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        return g.Problem(ctx, J, prob.site_class, prob.fixed_q, prob.z, prob.counts, allow_charged=allow), J, ms

    def emit(d):
        if out is None:
            print(json.dumps(d), flush=True)
        else:
            out.append(d)

    oracle.build()
    only = set(x.strip() for x in args.only.split(","))

    def want(section):
        return section in only

    if want("mc"):
        # ---- rocksalt 2x2x2, N = 64: 8 chains x 20,000 swaps at kT = 0.05 eV, FP64, parity with the oracle
        prob = synth.rocksalt_problem((2, 2, 2), 4.2)
        gp, J, jms = problem(prob)
        start = synth.random_population(prob, 8, synth.SEED_BASE)
        gp.mc_run(torch.tensor(start, device=dev), 0.05, 2000, 1)
        chains = torch.tensor(start, device=dev)
        ms = timed(lambda: gp.mc_run(chains, 0.05, 20000, synth.SEED_BASE))
        Jo = oracle.ewald_J(prob.lattice, prob.frac, prob.alpha, prob.nimg, prob.kcut)
        t0 = time.perf_counter()
        ref = oracle.mc_run(Jo, prob.site_class, prob.fixed_q, prob.z, start, 0.05, 20000, synth.SEED_BASE)
        cpu_s = time.perf_counter() - t0
        emit({"workload": "rocksalt 2x2x2 (N=64, 32 cations +1/+3), MC 8 chains x 20,000 swaps, kT=0.05 eV, FP64",
              "gpu_ms": ms, "trials_per_s": 160000 / (ms / 1e3), "cpu_oracle_s": cpu_s,
              "cpu_oracle_trials_per_s": 160000 / cpu_s, "cpu_cores": 1,
              "trajectory_parity": bool(np.array_equal(chains.cpu().numpy(), ref["species"])),
              "ewald_build_ms": jms})

    if want("ga"):
        # ---- layered R-3m 12x12x1, N = 1296: GA population 1024, 200 generations
        prob = synth.layered_problem()
        gp, J, jms = problem(prob)
        pop0 = gp.random_configs(1024, 3)
        res = {}
        for prec in ("f64", "f64_incr", "exact", "f32", "bf16x3"):
            pop = pop0.clone()
            gp.ga_run(pop.clone(), 2, 20, oracle.p_mut_to_u32(0.1), 9, 0, prec)
            box = {}
            ctx.set_timing(True)
            ctx.kernel_time("ga")
            ctx.kernel_time("ga_incr")
            ms = timed(lambda: box.setdefault("E", gp.ga_run(pop, 200, 20, oracle.p_mut_to_u32(0.1), 9, 0, prec)))
            gk_ms, gk_n = ctx.kernel_time("ga")
            ik_ms, ik_n = ctx.kernel_time("ga_incr")
            ctx.set_timing(False)
            E = box["E"]
            # children kernel: reads both parents, writes the child (int8 species)
            ga_bytes = 3.0 * 1024 * prob.Nv
            gk_avg = gk_ms / max(gk_n, 1)
            E64 = gp.score(pop, "f64")
            gen_bytes = 3.0 * 1024 * prob.Nv + (8.0 * 1024 * prob.Nv * 3 if prec == "f64_incr" else 0.0)
            res[prec] = {"ms": ms, "generations_per_s": 200 / (ms / 1e3), "child_evals_per_s": 1024 * 200 / (ms / 1e3),
                         "generation_algorithmic_gbs_min": gen_bytes / (ms / 200 / 1e3) / 1e9,
                         "best_E_eV": float(E.min()), "best_E_fp64_rescored_eV": float(E64.min()),
                         "max_rel_dev_from_fp64_rescoring": float(((E - E64).abs() / E64.abs()).max()),
                         "children_kernel_ms": gk_avg,
                         "children_kernel_hbm_gbs_algorithmic": ga_bytes / (gk_avg / 1e3) / 1e9}
            if ik_n:
                res[prec]["incremental_kernel_ms"] = ik_ms / ik_n
        # R independent populations in one run: the children of all come from one launch and
        # are rescored by one call over R P configurations
        for prec in ("f64_incr", "exact", "bf16x3"):
            R_pop = 8
            popR = gp.random_configs(R_pop * 1024, 17)
            gp.ga_run_populations(popR.clone(), R_pop, 2, 20, oracle.p_mut_to_u32(0.1), 9, 0, prec)
            ms = timed(lambda: gp.ga_run_populations(popR, R_pop, 50, 20, oracle.p_mut_to_u32(0.1), 9, 0, prec))
            res[f"{prec}_{R_pop}_populations"] = {
                "ms": ms, "generations_per_s": 50 / (ms / 1e3),
                "population_generations_per_s": R_pop * 50 / (ms / 1e3),
                "child_evals_per_s": R_pop * 1024 * 50 / (ms / 1e3)}
            del popR
        # the incremental rescoring kernel on one generation bred from the random population:
        # M_c changed sites per child -> M_c Nv FP64 FMAs and M_c J rows (Nv doubles each)
        kids, par, _ = gp.ga_generation(pop0, gp.score(pop0, "f64"), 20, oracle.p_mut_to_u32(0.1), 0, 9, record=True)
        pa, pb = par[:, 0].long(), par[:, 1].long()
        M = torch.minimum((kids != pop0[pa]).sum(1), (kids != pop0[pb]).sum(1)).double().sum().item()
        ctx.set_timing(True)
        ctx.kernel_time("ga_incr")
        for _ in range(20):
            gp.ga_run(pop0.clone(), 1, 20, oracle.p_mut_to_u32(0.1), 9, 0, "f64_incr")
        ik_ms, ik_n = ctx.kernel_time("ga_incr")
        ctx.set_timing(False)
        ik = ik_ms / max(ik_n, 1) / 1e3
        incr_bytes = 8.0 * M * prob.Nv + 2 * 8.0 * 1024 * prob.Nv + 3.0 * 1024 * prob.Nv
        _, hbm_peak_ga, _ = _peaks()
        res["f64_incr_one_generation"] = {
            "changed_sites_per_child": M / 1024, "kernel_ms": ik * 1e3,
            "fp64_tflops": 2.0 * M * prob.Nv / ik / 1e12,
            # FP64 pipe peak: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz = 1.26 TFLOP/s
            "fp64_pipe_frac": 2.0 * M * prob.Nv / ik / 1.2585e12,
            "algorithmic_gbs": incr_bytes / ik / 1e9,
            "algorithmic_frac_of_hbm_copy_peak": incr_bytes / ik / 1e9 / hbm_peak_ga,
            "note": "J rows of the changed sites + parent and child potentials + species; the rows mostly come "
                    "from L2 (J_vv is 6 MB)"}
        work = None
        Jr = np.random.default_rng(1).standard_normal((prob.N, prob.N))
        Jr = 0.5 * (Jr + Jr.T)
        popn = pop0[:256].cpu().numpy()
        En = oracle.score(Jr, prob.site_class, prob.fixed_q, prob.z, popn)
        t0 = time.perf_counter()
        kids, _, _ = oracle.ga_generation(prob.site_class, popn, En, 5, 0.1, gen=0, seed=9)
        oracle.score(Jr, prob.site_class, prob.fixed_q, prob.z, kids)
        cpu_gen = (time.perf_counter() - t0) * 4.0   # population 256 -> 1024 (generation and scoring are linear in P)
        emit({"workload": "layered R-3m 12x12x1 (N=1296: 432 O fixed, Li/vac 346/86, Ni2/Ni3/Mn4/Co3 108 each), "
                          "GA population 1024 x 200 generations, elite 20, p_mut 0.1",
              "forms": res, "cpu_oracle_s_per_generation": cpu_gen, "cpu_oracle_note":
              "one generation of 256 children timed and scaled x4 (scoring is linear in the population), 1 thread",
              "ewald_build_ms": jms})

    if want("gd"):
        # ---- all-pairs steepest descent: layered R-3m 12x12x1 (N = 1296), 256 random configurations
        prob = synth.layered_problem()
        gp, J, jms = problem(prob)
        B_gd = 256
        start = gp.random_configs(B_gd, 41)
        gp.gd_run(start.clone(), 2)
        sp = start.clone()
        box = {}
        ms = timed(lambda: box.setdefault("r", gp.gd_run(sp, 1000)))
        E_gd, steps = box["r"]
        st = steps.double()
        vclass = prob.site_class[prob.site_class >= 0]
        pairs = float(sum(int((vclass == k).sum()) * (int((vclass == k).sum()) - 1) // 2 for k in range(prob.n_class)))
        # per step of a live configuration: pass 0 (minimum) and pass 1 (lowest pair within the tie);
        # the step that finds the local minimum runs pass 0 only
        checks = pairs * float((2 * st + 1).sum())
        E0 = gp.score(start, "f64")
        emit({"workload": f"layered R-3m 12x12x1 (N=1296, Nv=864), {B_gd} random configurations, all-pairs steepest "
                          "descent over single swaps to a local minimum, FP64",
              "ms": ms, "steps_max": int(st.max()), "steps_mean": float(st.mean()),
              "same_class_pairs_per_configuration": pairs,
              "pair_checks_per_s": checks / (ms / 1e3),
              "mean_E_start_eV": float(E0.mean()), "mean_E_end_eV": float(E_gd.mean()),
              "end_is_fp64_consistent": bool(((E_gd - gp.score(sp, "f64")).abs() / E_gd.abs()).max() < 1e-10),
              "ewald_build_ms": jms})
        del gp, J

    if want("batch"):
        # ---- uneven batch: 256 rocksalt / spinel-like cells, N in [64, 2048], 512 chains each
        cells = synth.batch_problems(args.batch_cells)
        gps, sps, kts = [], [], []
        tb = 0.0
        for i, pr in enumerate(cells):
            gpi, _, bms = problem(pr)
            tb += bms
            gps.append(gpi)
            sps.append(gpi.random_configs(args.batch_chains, 100 + i))
            kts.append(torch.full((args.batch_chains,), pr.kT, dtype=torch.float64, device=dev))
        best_cpc, tune_ms = g.batch_mc_autotune(ctx, gps, sps, kts, 256, "f64")
        steps = args.batch_steps
        trials = steps * args.batch_chains * len(cells)
        modes = {}
        for mode, name in ((0, "per_problem_launches"), (1, "persistent"), (2, "persistent_graph")):
            cpc = best_cpc if mode else min(best_cpc, 4)
            g.batch_mc_run(ctx, gps, sps, kts, 64, 7, step0=0, chains_per_cta=cpc, mode=mode)
            ms = timed(lambda: g.batch_mc_run(ctx, gps, sps, kts, steps, 7, step0=64, chains_per_cta=cpc, mode=mode))
            modes[name] = {"ms": ms, "trials_per_s": trials / (ms / 1e3), "chains_per_cta": cpc}
        emit({"workload": f"{len(cells)} rocksalt/spinel-like cells, N log-uniform 64..2048, {args.batch_chains} chains "
                          f"each, {steps} swaps per chain (kT per cell 0.01..0.2 eV), FP64",
              "trials": trials, "modes": modes, "autotuned_chains_per_cta": best_cpc, "autotune_probe_ms": tune_ms,
              "ewald_build_total_ms": tb,
              "trials_per_chain_in_config": 100000,
              "extrapolated_s_for_1e5_swaps": modes["persistent_graph"]["ms"] / 1e3 * 100000 / steps})
        del gps, sps, kts

    if want("forms"):
        # ---- every scoring form at N = 4096, B = 4096 (throughput, error vs the FP64 path, roofline)
        prob = synth.random_cubic_problem(n_side=N_SIDE)
        gp, J, jms = problem(prob)
        pop = torch.tensor(synth.random_population(prob, B_POP, synth.SEED_BASE + 2), device=dev)
        E64 = gp.score(pop, "f64")
        bf16_peak, hbm_peak, _ = _peaks()
        ld = ((prob.N + 127) // 128) * 128
        nbm = ld // 128
        forms = {}
        for form in ("f64", "f32", "tf32", "tf32x2", "bf16x2", "bf16x3", "exact"):
            for _ in range(3):
                gp.score(pop, form)
            reps = 2 if form in ("f64", "f32") else 50
            ctx.set_timing(True)
            ctx.kernel_time("score_tc")
            ctx.kernel_time("score_cc")
            box = {}
            ms = timed(lambda: [box.setdefault("E", gp.score(pop, form)) for _ in range(reps)]) / reps
            tc_form = form in TERMS or form == "exact"
            kms, kn = ctx.kernel_time("score_tc" if tc_form else "score_cc")
            ctx.set_timing(False)
            E = gp.score(pop, form)
            err = (E - E64).abs()
            d = {"ms_per_population": ms, "evals_per_s": B_POP / (ms / 1e3), "speedup_vs_f64": None,
                 "max_abs_err_eV": float(err.max()), "rms_abs_err_eV": float(err.pow(2).mean().sqrt()),
                 "kernel_ms": kms / max(kn, 1)}
            if tc_form:
                terms = gp.exact_info()[1] if form == "exact" else TERMS[form]
                flops = terms * 2.0 * 128 * 128 * (nbm * (nbm + 1) // 2) * ((B_POP + 255) // 256 * 256)
                peak = bf16_peak / 2.0 if "tf32" in form else bf16_peak
                d["tensor_tflops"] = flops / (d["kernel_ms"] / 1e3) / 1e12
                d["tensor_frac_of_measured_peak"] = d["tensor_tflops"] / peak
            forms[form] = d
        for f in forms:
            forms[f]["speedup_vs_f64"] = forms["f64"]["ms_per_population"] / forms[f]["ms_per_population"]
        idx, Etop = gp.topk_rescore(pop, gp.score(pop, "bf16x3"), 64)
        # top-k selection alone against the batch size: the 16-site rocksalt cell makes the FP64
        # rescoring of the k = 64 candidates negligible; up to 512 configurations the pairwise
        # rank kernel, above it the radix select
        tiny = synth.tiny_rocksalt_problem()
        gpt, _, _ = problem(tiny)
        sel_ms = {}
        for Bs in (512, 513, 4096, 262144, 1048576):
            spt = gpt.random_configs(Bs, 5)
            Et = torch.randn(Bs, dtype=torch.float64, device=dev)
            gpt.topk_rescore(spt, Et, 64)
            sel_ms[str(Bs)] = timed(lambda: [gpt.topk_rescore(spt, Et, 64) for _ in range(10)]) / 10
            del spt, Et
        emit({"workload": WORKLOAD + ", every scoring form", "forms": forms,
              "top64_after_bf16x3_equals_fp64_top64": bool(set(idx.tolist()) == set(torch.argsort(E64)[:64].tolist())),
              "topk64_select_ms_vs_batch": sel_ms, "ewald_build_ms": jms})
        del gp, J, pop, E64

    if want("relaxed"):
        # ---- relaxed occupations: bcc 16^3, N = 8192, B = 2048 logits sets, 5 species
        prob = synth.bcc_relaxed_problem()
        gp, J, jms = problem(prob, allow=True)
        B = args.grad_batch
        L = torch.tensor(synth.random_logits(prob, B, 5), device=dev)
        lam, eta = 1.0, 0.01
        res = {}
        for prec in ("f64", "tf32x2", "f16x2"):
            gp.energy_grad(L[:2].contiguous(), lam, prec)
            box = {}
            ms = timed(lambda: box.setdefault("r", gp.energy_grad(L, lam, prec)))
            res[prec] = {"energy_grad_ms": ms, "grad_steps_per_s": 1e3 / ms}
        E64, g64 = gp.energy_grad(L, lam, "f64")
        for prec in ("tf32x2", "f16x2"):
            Etc, gtc = gp.energy_grad(L, lam, prec)
            res[prec]["max_rel_E_err"] = float(((Etc - E64).abs() / E64.abs()).max())
            res[prec]["max_abs_grad_err_rel_to_max"] = float((gtc - g64).abs().max() / g64.abs().max())
        steps = args.grad_steps
        box = {}
        Lf = L.clone()
        dms16 = timed(lambda: box.setdefault("E16", gp.relaxed_descent(Lf, lam, eta, steps, "f16x2")))
        Ld = L.clone()
        E0 = gp.energy_grad(Ld, lam, "tf32x2")[0]
        dms = timed(lambda: box.setdefault("E", gp.relaxed_descent(Ld, lam, eta, steps, "tf32x2")))
        p_occ = gp.occupations(Ld)
        rms = timed(lambda: box.setdefault("sp", gp.round_to_counts(p_occ)))
        seeded = box["sp"]
        E_seed = gp.score(seeded, "bf16x3")
        rand = gp.random_configs(B, 9)
        E_rand = gp.score(rand, "bf16x3")
        gms = timed(lambda: box.setdefault("Eg", gp.ga_run(seeded, 5, 40, oracle.p_mut_to_u32(0.1), 3, 0, "bf16x3")))
        emit({"workload": f"bcc 16^3 (N=8192, 5 species +1/+2/+3/+4/0), relaxed occupations, B={B} logits sets, "
                          f"counts penalty lambda={lam}", "forms": res,
              "descent": {"form": "tf32x2", "steps": steps, "eta": eta, "ms": dms, "steps_per_s": steps / (dms / 1e3),
                          "mean_E_before_eV": float(E0.mean()), "mean_E_after_eV": float(box["E"].mean())},
              "descent_f16x2": {"steps": steps, "ms": dms16, "steps_per_s": steps / (dms16 / 1e3),
                                "mean_E_after_eV": float(box["E16"].mean())},
              "round_to_counts_ms": rms,
              "seeded_population": {"mean_E_eV": float(E_seed.mean()), "min_E_eV": float(E_seed.min()),
                                    "random_population_mean_E_eV": float(E_rand.mean()),
                                    "random_population_min_E_eV": float(E_rand.min()),
                                    "ga_5_generations_ms": gms, "ga_best_E_eV": float(box["Eg"].min())},
              "ewald_build_ms": jms})

def run_paper(args, ctx=None, out=None):
    """The paper's heuristics on its own workloads, one JSON line per cell: the
    O3 layered-oxide sqrt(3) supercells of Table 1 and NaCl 3x3x3 (known
    optimum, Eq. 3).  Per method: best energy per ion (FP64 rescored), GPU time.
    Budgets are fixed numbers of steps, not the paper's wall-clock budgets."""
    import torch

    import goac_synth as synth
    import oracle
    import paper_2409_08808_gb300 as g

    ctx = ctx or g.Context(0)

    def emit(d):
        if out is None:
            print(json.dumps(d), flush=True)
        else:
            out.append(d)
    dev = torch.device("cuda", 0)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        out = fn()
        b.record()
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    def methods(prob, C, steps, ga_pop, ga_gen, which=("MC", "SA", "REMC", "GA", "HY")):
        frac = torch.tensor(prob.frac, device=dev)
        (J, gp), build_ms = timed(lambda: (lambda J_: (J_, g.Problem(ctx, J_, prob.site_class, prob.fixed_q, prob.z,
                                                                     prob.counts)))(
            g.build_ewald(ctx, prob.lattice, frac, prob.alpha, prob.nimg, prob.kcut)))
        res = {"ewald_J_and_problem_ms": build_ms}
        best_any = None

        def record(name, sp, ms, extra=None):
            nonlocal best_any
            E = gp.score(sp, "f64")
            i = int(torch.argmin(E))
            e = float(E[i])
            res[name] = {"best_E_eV": e, "best_E_per_ion_eV": e / prob.N, "gpu_ms": ms}
            if extra:
                res[name].update(extra)
            if best_any is None or e < best_any[0]:
                best_any = (e, sp[i].clone())

        if "MC" in which:
            sp = gp.random_configs(C, 1)
            o, ms = timed(lambda: gp.mc_run(sp, 0.75, steps, 11, precision="f64"))
            record("MC", o["best_species"], ms, {"kT_eV": 0.75, "chains": C, "steps": steps})
        if "SA" in which:
            sp = gp.random_configs(C, 2)
            o, ms = timed(lambda: gp.sa_run(sp, 1.0, 0.002, steps, steps, 12))
            record("SA", o["best_species"], ms, {"kT_eV": "1.0 -> 0.002 (exponential)", "chains": C, "steps": steps})
        R = 8
        lad = list(np.geomspace(0.02, 1.0, R))
        G = max(1, C // R)
        rounds = 20
        if "REMC" in which:
            sp = gp.random_configs(G * R, 3)
            (Er, perm, nex), ms = timed(lambda: gp.remc_run(sp, G, R, lad, rounds, steps // rounds, 13))
            record("REMC", sp, ms, {"groups": G, "ladder_eV": [round(x, 4) for x in lad], "rounds": rounds,
                                    "steps_per_round": steps // rounds, "exchanges": nex})
        if "GA" in which:
            pop = gp.random_configs(ga_pop, 4)
            E, ms = timed(lambda: gp.ga_run(pop, ga_gen, max(1, ga_pop // 50), oracle.p_mut_to_u32(0.1), 14, 0,
                                            "bf16x2"))
            record("GA", pop, ms, {"population": ga_pop, "generations": ga_gen, "scoring": "bf16x2, FP64 rescored"})
        if "HY" in which:
            sp = gp.random_configs(G * R, 5)
            E, ms = timed(lambda: gp.hybrid_run(sp, G, R, lad, 4, rounds // 4, steps // rounds, ga_gen // 4,
                                                max(1, (G * R) // 50), oracle.p_mut_to_u32(0.1), 15))
            record("HY", sp, ms, {"cycles": 4})
        return res, best_any

    for reps in [tuple(int(x) for x in c.split("x")) for c in args.paper_cells.split(",") if c]:
        prob = synth.o3_layered_problem(reps)
        res, best = methods(prob, args.paper_chains, args.paper_steps, 1024, 200)
        pos = [int((prob.site_class == k).sum()) for k in range(2)]
        line = {"workload": f"O3-Na2/3[Li1/6Fe1/6Co1/6Ni1/6Mn1/3]O2 sqrt3 {reps[0]}x{reps[1]}x{reps[2]} "
                            f"(N={prob.N}, 10^{oracle.log10_configurations(pos, prob.counts):.0f} configurations)",
                "methods": res, "best_E_per_ion_eV": best[0] / prob.N,
                "budget": f"{args.paper_chains} chains x {args.paper_steps} swaps; GA 1024 x 200 generations"}
        emit(line)
    # NaCl 3x3x3: 216 positions, 108 Na+ / 108 Cl- on one class; optimum = rocksalt order
    prob, _ = synth.nacl_problem((3, 3, 3), 5.62)
    res, best = methods(prob, args.paper_chains, args.nacl_steps, 1024, 1000, tuple(args.nacl_methods.split(",")))
    M_ref = 1.747564594633182
    E_opt = -108 * M_ref * 14.3996454784 / 2.81
    for k, v in res.items():
        if not isinstance(v, dict):
            continue
        v["madelung"] = abs(v["best_E_eV"]) * 2.81 / (108 * 14.3996454784)
        v["found_optimum"] = bool(abs(v["best_E_eV"] - E_opt) < 1e-6 * abs(E_opt))
    emit({"workload": "NaCl 3x3x3, 216 positions 50/50 Na/Cl (10^64 configurations), r = 2.81 A",
          "optimum_E_eV": E_opt, "madelung_ref": M_ref, "methods": res,
          "budget": f"{args.paper_chains} chains x {args.nacl_steps} swaps"})


def main():
    args = _args()
    if args.suite:
        run_suite(args)
        return
    if args.paper:
        run_paper(args)
        return
    world, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Throughput benchmark: particle-steps/s of the full time step at N = 1e5.

Workload: 100,000 two-species active disks (a = 1, area fraction 0.30,
L = 1023.3, reflecting walls), non-reciprocal long-range law
A = [[0.05, 0.2], [-0.1, 0.05]] with F = A r_hat / r^2 summed over all pairs,
self-propulsion v0 = 1, D = 1, D_r = 0.5, dt = 1e-4, Philox seed 100, start by
random sequential addition.  One step = forces (all pairs) + Euler-Maruyama
+ triangulation check/repair/flips + overlap correction until no overlap.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Under torchrun (N > 1) every rank advances its own
independent replica (a different Philox replica stream); `value` sums them.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "particle-steps/s at N=1e5 (all-pairs + Delaunay repair)"
UNIT = "particle-steps/s"
WORKLOAD = "n1e5: N=100000 two-species ABP disks, rho=0.30, all-pairs 1/r^2 non-reciprocal, Delaunay overlap correction"
# algorithmic work of the all-pairs force per ordered pair (the count the
# roofline's `achieved` uses for every sweep): 2 FADD + 2 FFMA (r^2) + 2 FMUL
# (s^3) + 2 FFMA (accumulate) = 12 flops (FMA = 2) + 1 MUFU rsqrt
FLOPS_PER_PAIR = 12
FP32_INST_PER_PAIR = 8   # the same work counted as FP32-pipe instructions
# work each sweep executes (frac_executed, fp32_pipe_frac).  Symmetric sweep:
# per unordered pair 2 FADD + 2 FFMA + 2 FMUL + 4 FFMA (both sides) = 16 flops
# in 10 FP32 lane operations (+1 MUFU), i.e. per ordered pair:
FLOPS_PER_PAIR_SYM = 8
LANES_PER_PAIR_SYM = 5
# one-sided periodic sweep: per ordered pair 2 hi + 2 lo differences and 2 adds
# (exact near-pair vectors), 2 FFMA (r^2), 2 FMUL, 2 FFMA (accumulate) = 12 lane
# operations (16 flops), plus the minimum-image tests (not counted).  The
# symmetric sweep's periodic form counts as the symmetric sweep (its per-pair
# minimum images, in the tiles near the antipode, are not counted)
FLOPS_PER_PAIR_PER = 16
LANES_PER_PAIR_PER = 12


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest x over the ranks (the job's time is its slowest rank's);
    the only collective of the replicas path, outside the timed region."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_params(bd, cfg, rank, modes=()):
    """Rank r advances its own replica of the workload: the same start and
    parameters, its own Philox stream (key word 1 = seed_hi xor r)."""
    p = bd.params_from_config(cfg)
    if "verlet" in modes:
        p.overlap_mode = bd.OVERLAP_VERLET   # Algorithm 2 over the Verlet lists, no triangulation
    if "periodic" in modes:
        p.boundary = bd.BOUNDARY_PERIODIC    # the paper's periodic box (minimum image, torus triangulation)
    p.replica = rank
    return p


def shard_replicas(ns, laws, world, short_cost=3000.0):
    """Cost-balanced assignment of independent replicas to ranks (greedy:
    largest cost first, each to the least-loaded rank).  A long-range replica
    costs N^2 (all pairs), a short-range one short_cost * N (its per-disk work
    measured against the all-pairs sweep's per-pair work on one GPU: about
    0.5 ns per disk-step at 2^20 disks against 1.65e-4 ns per pair at
    N = 1e5).  Returns one ascending list of replica indices per rank."""
    cost = [float(n) * n if law == 1 else short_cost * float(n) for n, law in zip(ns, laws)]
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for r in sorted(range(len(cost)), key=lambda k: (-cost[k], k)):
        w = min(range(world), key=lambda k: (load[k], k))
        out[w].append(r)
        load[w] += cost[r]
    return [sorted(v) for v in out]


def sharded_step(system, F, ws):
    """One step of a system whose all-pairs sweep is shared among the ranks:
    this rank's partial forces into F, one sum over the ranks, then the move
    and the correction with the summed forces on every rank."""
    system.step_begin(F.data_ptr())
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(F)
    return system.step_end(F.data_ptr())


def run_reference(args):
    """The oracle (plain FP64 CPU restatement) on the same workload, host cores.

    Every timed step is one whole oracle step of the N = 1e5 system (exact
    all-pairs FP64 forces with OpenMP over all host cores, Euler-Maruyama,
    Delaunay triangulations and overlap correction), the state carried from
    step to step.  At about 3.5 s a step the run is bounded: at most 20 timed
    steps and 2 warm-up steps, and the line's `steps` / `warmup` say how many
    ran."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import step as ostep
    from paper_1703_02484_gb300 import workloads
    cfg = workloads.CONFIGS["n1e5"]
    xy, sp, th = workloads.initial_state(cfg)
    cores = os.cpu_count() or 1
    op = ostep.Params(L=cfg.L, a=cfg.a, law=cfg.law, alpha=cfg.alpha, D=cfg.D, Dr=cfg.Dr,
                      v0=cfg.v0, dt=cfg.dt, seed=cfg.seed)
    steps = max(1, min(args.steps, 20))
    warm = min(args.warmup, 2)
    th = th.astype(np.float64)
    k = 0
    for _ in range(warm):
        r = ostep.step(xy, th, sp, k, op, threads=cores)
        xy, th, k = r["xy"], r["theta"], k + 1
    t0 = time.perf_counter()
    for _ in range(steps):
        r = ostep.step(xy, th, sp, k, op, threads=cores)
        if r["rejected"]:
            raise RuntimeError("oracle step %d rejected" % k)
        xy, th, k = r["xy"], r["theta"], k + 1
    total = time.perf_counter() - t0
    ms = 1e3 * total / steps
    value = cfg.n / (ms / 1e3)
    sample = ("%d whole FP64 oracle steps of the N=%d workload, state carried (all-pairs forces "
              "with OpenMP over %d threads, Delaunay rebuilds and overlap correction), after %d "
              "warm-up steps" % (steps, cfg.n, cores, warm))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": cfg.n, "seed": cfg.seed, "same_config": True,
                       "steps_requested": args.steps, "warmup_requested": args.warmup},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def force_kernel_name(variant, periodic):
    """The all-pairs sweep (and its reduction) the autotuner's variant runs."""
    kernel = {0: "k_force_long_f32", 1: "k_force_long_f32x2<4>",
              2: "k_force_long_sym<4,2> + k_force_sym_reduce",
              3: "k_force_long_sym<2,4> + k_force_sym_reduce"}[variant]
    if periodic:
        kernel = "k_force_long_per" if variant < 2 else kernel.replace("> +", ", periodic> +")
    return kernel


def force_roofline(N, avg_force_s, variant, periodic, sms, f_hz, pk_kind, traffic=None):
    """FP32 roofline of the all-pairs force evaluation: achieved = the
    algorithmic 12 flops per ordered pair over N(N-1) pairs per launch time;
    frac_executed and fp32_pipe_frac from the flops and lane operations the
    chosen sweep executes per ordered pair."""
    peak_tflops = sms * 128 * 2 * f_hz / 1e12
    pairs = N * (N - 1)
    flops_pp, lanes_pp = (FLOPS_PER_PAIR_SYM, LANES_PER_PAIR_SYM) if variant >= 2 else \
        (FLOPS_PER_PAIR, FP32_INST_PER_PAIR)
    if periodic and variant < 2:
        flops_pp, lanes_pp = FLOPS_PER_PAIR_PER, LANES_PER_PAIR_PER
    achieved = FLOPS_PER_PAIR * pairs / avg_force_s / 1e12
    executed = flops_pp * pairs / avg_force_s / 1e12
    return {"bound": "alu", "kernel": force_kernel_name(variant, periodic), "achieved": achieved,
            "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "traffic": traffic, "fp32_pipe_frac": lanes_pp * pairs / avg_force_s / (sms * 128 * f_hz),
            "frac_executed": executed / peak_tflops,
            "pair_interactions_per_s": pairs / avg_force_s,
            "avg_launch_ms": avg_force_s * 1e3,
            "peak_note": "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s max clock); achieved "
                         "counts the algorithmic %d flops per ordered pair over N(N-1) pairs; "
                         "the sweep executes %d flops in %d FP32 lane ops per ordered pair "
                         "(frac_executed, capped at %.2f), so frac is capped at %.2f"
                         % (sms, f_hz / 1e6, pk_kind, FLOPS_PER_PAIR, flops_pp, lanes_pp,
                            flops_pp / (2.0 * lanes_pp), FLOPS_PER_PAIR / (2.0 * lanes_pp))}


def correction_roofline(system, stage_raw, steps, N, verlet_mode, pk, pk_kind, visits=None, flips=0.0):
    """HBM roofline of the per-step correction kernel of the short-range path.

    Duration: the kernel's own device-clock stage timers (bd_stage_times),
    summed over its stages, per launch (one launch per step).  Algorithmic
    bytes per launch, from the pass counts of the same timers and the
    triangles the check passes visited (bd_step_stats.tri_visits, V):
      k_triangulation: a check pass reads the corner table of each triangle
        it visits (32 B) and, in the first pass of the step, each disk's moved
        flag, FP32 position and FP32 move (25 B); a flip (bd_step_stats.flips)
        reads its candidate entry, six claims and the pair's corner tables and
        writes the pair, four back-pointers and the pair's undo journal (about
        200 B); an apply pass reads and writes positions, displacements and
        flags (100 B per disk).
      k_overlap_verlet: a scan pass reads each disk's count, flag, both
        position copies and its list with the neighbours' flags (38 + 5 m B
        per disk, m the mean list length) and writes its displacement and hit
        flag (17 B); an apply pass 100 B per disk."""
    ms = sum(v[0] for k, v in stage_raw.items() if k != "check_lists") / steps   # check_lists is part of check
    if not ms > 0:
        return None
    if verlet_mode:
        cnt = system.neighbors()
        m = float(np.mean([len(c) for c in cnt]))
        scans, applies = stage_raw["check"][1] / steps, stage_raw["apply"][1] / steps
        per = scans * N * (38 + 5 * m + 17) + applies * N * 100
        kernel = "k_overlap_verlet"
        note = "%.2f scan passes (mean list %.1f) and %.2f apply passes per launch" % (scans, m, applies)
    else:
        T = system.n_tri
        P, F, A = (stage_raw[k][1] / steps for k in ("check", "flip", "apply"))
        V = visits if visits else P * T
        per = 32 * V + 25 * N + 200 * flips + A * 100 * N
        kernel = "k_triangulation"
        note = ("%.2f check passes visiting %.0f triangles, %.2f flip rounds, %.2f apply passes per "
                "launch; %d triangles" % (P, V, F, A, T))
    gbs = per / (ms / 1e3) / 1e9
    peak = float(pk.get("hbm_gbs", 6800.0))
    return {"bound": "hbm", "kernel": kernel, "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak, "traffic": None, "algorithmic_bytes_per_launch": per,
            "avg_launch_ms": ms,
            "peak_note": "%s copy bandwidth (MEASURED_PEAKS.json hbm_gbs); duration from the kernel's "
                         "device-clock stage timers; %s" % (pk_kind, note)}


def cpu_baseline(cfg, xy, sp, th, periodic=False, one_core=True):
    """The oracle as it stands, timed on the host cores: one whole step of the
    workload with its all-pairs force sum in OpenMP over every core, and (for
    `value_1core`) the same step on one thread."""
    from oracle import step as ostep
    cores = os.cpu_count() or 1
    L = float(np.float32(cfg.L)) if periodic else cfg.L
    op = ostep.Params(L=L, a=cfg.a, law=cfg.law, alpha=cfg.alpha, D=cfg.D, Dr=cfg.Dr,
                      v0=cfg.v0, dt=cfg.dt, seed=cfg.seed, periodic=periodic)
    t0 = time.perf_counter()
    ostep.step(xy, th, sp, 0, op, threads=cores)
    t = time.perf_counter() - t0
    out = {"value": cfg.n / t, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "one whole FP64 oracle step of the N=%d workload (all-pairs forces with "
                     "OpenMP over %d threads, Delaunay rebuilds and overlap correction): %.2f s"
                     % (cfg.n, cores, t)}
    if one_core and cores > 1:
        t0 = time.perf_counter()
        ostep.step(xy, th, sp, 0, op, threads=1)
        t1 = time.perf_counter() - t0
        out["value_1core"] = cfg.n / t1
        out["sample"] += "; the same step on one thread: %.2f s" % t1
    return out


def run_batched(args):
    """Batched workload: 256 replicas advanced together, against the same
    replicas advanced one handle at a time (the plain single-system step)."""
    import torch
    import paper_1703_02484_gb300 as bd
    from paper_1703_02484_gb300 import workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfgs = workloads.batch_configs(256)
    params_all = []
    for r, cfg in enumerate(cfgs):
        p = bd.params_from_config(cfg)
        p.replica = r
        p.seed = 3 + 1000 * r
        params_all.append(p)
    # N > 1: the replicas are shared out by cost (strong scaling: the same 256)
    mine = shard_replicas([p.n for p in params_all], [p.law for p in params_all], ws)[rank]
    params = [params_all[r] for r in mine]
    N_all = sum(p.n for p in params_all)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    b = bd.System(params, stream=stream.cuda_stream)
    t_init = time.perf_counter() - t0
    N = b.n
    for _ in range(args.warmup):
        b.step(1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        st = b.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, "cuda") / args.steps
    tune = b.tuning()
    b.close()
    if ws > 1:
        if rank == 0:
            line = {"metric": "particle-steps/s (c4: 256 batched replicas)", "value": N_all / (ms / 1e3),
                    "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                    "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                    "data": "synthetic",
                    "config": {"workload": "c4: 256 replicas shared out by cost over %d ranks" % ws, "N": N_all,
                               "replicas_rank0": len(mine), "disks_rank0": N, "tuning_rank0": tune},
                    "clocks": clk.summary(), "gpu_launches": None}
            print(json.dumps(line), flush=True)
        dist.destroy_process_group()
        return
    # the same replicas one handle at a time (sampled: every 8th replica)
    sample = list(range(0, 256, 8))
    alone_ms = 0.0
    n_sample = 0
    for r in sample:
        s1 = bd.System(params[r], stream=stream.cuda_stream)
        for _ in range(2):
            s1.step(1)
        torch.cuda.synchronize()
        a0 = time.perf_counter()
        s1.step(args.steps)
        torch.cuda.synchronize()
        alone_ms += (time.perf_counter() - a0) * 1e3 / args.steps
        n_sample += params[r].n
        s1.close()
    seq_ms = alone_ms * (256 / len(sample))
    line = {"metric": "particle-steps/s (c4: 256 batched replicas)", "value": N / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "c4: 256 replicas, N log-uniform [512, 65536] (sum %d), rho U[0.3,0.5], "
                                   "half c1 long-range law, half c3 short-range law" % N,
                       "N": N, "init_s": t_init, "tuning": tune,
                       "sequential_ms_per_step_estimate": seq_ms,
                       "sequential_sample": "every 8th replica alone, scaled by 8",
                       "batched_speedup": seq_ms / ms,
                       "steps_done": st["steps_done"], "rejected": st["rejected"]},
            "clocks": clk.summary(), "gpu_launches": None}
    print(json.dumps(line), flush=True)


def run_sharded(args):
    """The N = 1e5 system on N ranks at once: each rank computes its share of
    the all-pairs sweep, the partial forces are summed by one all-reduce per
    step, and every rank advances the whole system (strong scaling: one
    system, N = 1e5 whatever the rank count)."""
    import torch
    import paper_1703_02484_gb300 as bd
    from paper_1703_02484_gb300 import workloads
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg = workloads.CONFIGS["n1e5"]
    xy, sp, th = workloads.initial_state(cfg)
    stream = torch.cuda.current_stream()
    system = bd.System(bd.params_from_config(cfg), xy, sp, th, stream=stream.cuda_stream)
    system.set_force_shard(rank, ws)
    F = torch.empty(2 * system.force_slots(), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        sharded_step(system, F, ws)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            sharded_step(system, F, ws)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, "cuda") / args.steps
    if rank == 0:
        line = {"metric": "particle-steps/s (n1e5, all-pairs sweep shared over the ranks)",
                "value": cfg.n / (ms / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD + "; force sweep sharded over %d ranks, one FP64 all-reduce of "
                                                  "%d bytes per step" % (ws, F.numel() * 8),
                           "N": cfg.n, "seed": cfg.seed, "parallelism": "force-shard%d" % ws},
                "clocks": clk.summary(), "gpu_launches": None}
        print(json.dumps(line), flush=True)
    system.close()
    if ws > 1:
        dist.destroy_process_group()


def run_adjoint(args):
    """Differentiated rollout (4096 disks, rho 0.35, two species, v0 = 1, 200
    steps, checkpoints every 20): each timed unit is one recorded rollout
    (bd_rollout) plus its reverse pass (bd_rollout_vjp), against the plain
    steps (bd_step) over the same number of steps."""
    import torch
    import paper_1703_02484_gb300 as bd
    from paper_1703_02484_gb300 import workloads
    torch.cuda.set_device(0)
    cfg = workloads.CONFIGS["c5"]
    hist = args.workload.endswith("-hist")
    kind = bd.LOSS_HIST if hist else bd.LOSS_MSD
    xy, sp, th = workloads.initial_state(cfg)
    stream = torch.cuda.current_stream()
    s = bd.System(bd.params_from_config(cfg), xy, sp, th, stream=stream.cuda_stream)
    T = cfg.steps
    for _ in range(args.warmup):
        s.rollout(T, 20, 0.1, kind)
        s.rollout_vjp()
        s.step(T)
    K = max(1, min(args.steps, 20))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    launches = 0
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        for k in range(K):
            ev[k][0].record(stream)
            s.rollout(T, 20, 0.1, kind)
            launches += s.last_launch_count()
            ev[k][1].record(stream)
            g = s.rollout_vjp()
            launches += s.last_launch_count()
            ev[k][2].record(stream)
            s.step(T)
            ev[k][3].record(stream)
        torch.cuda.synchronize()
    fwd = sum(e[0].elapsed_time(e[1]) for e in ev) / K
    bwd = sum(e[1].elapsed_time(e[2]) for e in ev) / K
    plain = sum(e[2].elapsed_time(e[3]) for e in ev) / K
    npass, npairs = s.rollout_log_size()
    s.close()
    line = {"metric": "particle-steps/s (c5: recorded rollout + reverse pass)",
            "value": cfg.n * T / ((fwd + bwd) / 1e3), "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": (fwd + bwd) / T, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (adjoint sums f64)", "data": "synthetic",
            "config": {"workload": "c5: N=4096, rho=0.35, two species, v0=1, 200 steps, checkpoints every 20, "
                                   "%s loss; gradient w.r.t. (A00, A01, A10, A11, v0)"
                                   % ("pair-distance histogram" if hist else "MSD"),
                       "N": cfg.n, "rollout_steps": T,
                       "forward_ms": fwd, "reverse_ms": bwd, "plain_steps_ms": plain,
                       "gradient_evals_per_s": 1e3 / (fwd + bwd),
                       "overhead_vs_plain": (fwd + bwd) / plain,
                       "log_passes": npass, "log_pairs": npairs, "last_grad": list(map(float, g)),
                       "l2": "working set (< 2 MB) stays in L2; not flushed"},
            "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--workload", default="n1e5",
                    help="configuration name (n1e5 is the headline; n1e5-shard (its all-pairs sweep shared "
                         "over the ranks); c1, c2, c3, c5, c4 (batched), "
                         "c5-grad (differentiated rollout, MSD loss; c5-grad-hist: histogram loss); suffixes -verlet (overlap correction over "
                         "the Verlet lists) and -periodic (periodic box), e.g. c3-verlet, n1e5-periodic)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    args.warmup = max(3, args.warmup)
    if args.workload == "c4":
        run_batched(args)
        return
    if args.workload in ("c5-grad", "c5-grad-hist"):
        run_adjoint(args)
        return
    if args.workload == "n1e5-shard":
        run_sharded(args)
        return

    import torch
    import paper_1703_02484_gb300 as bd
    from paper_1703_02484_gb300 import workloads

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    base, *modes = args.workload.split("-")
    verlet_mode = "verlet" in modes
    periodic_mode = "periodic" in modes
    cfg = workloads.CONFIGS[base]
    xy, sp, th = workloads.initial_state(cfg)
    p = rank_params(bd, cfg, rank, modes)
    stream = torch.cuda.current_stream()
    system = bd.System(p, xy, sp, th, stream=stream.cuda_stream)
    N = cfg.n

    # warm-up
    for _ in range(args.warmup):
        system.step(1)
    # L2 flush buffer (> 129 MB of L2): written between timed steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    system.force_timing(True, reset=True)
    system.stage_times(reset=True)
    launches = 0
    stats_tot = {}
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            st = system.step(1)
            ev[k][1].record(stream)
            launches += system.last_launch_count()
            for key in ("corr_iters", "flips", "repair_flips", "overlap_pairs", "inverted", "tri_visits"):
                stats_tot[key] = stats_tot.get(key, 0) + st[key]
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    t_ms = float(sum(ms_steps))
    force_ms, force_n = system.force_timing(False)
    stage_raw = system.stage_times(reset=True)
    stage_ms = {k: v[0] / args.steps for k, v in stage_raw.items()}
    t_ms = max_over_ranks(t_ms, ws, "cuda")
    ms_per_step = t_ms / args.steps
    value = ws * N * args.steps / (t_ms / 1e3)

    # roofline of the dominant kernel (the all-pairs sweep): ALU-bound
    pk, pk_kind = peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    f_hz = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    peak_tflops = sms * 128 * 2 * f_hz / 1e12
    avg_force_s = (force_ms / max(1, force_n)) / 1e3
    pairs = N * (N - 1)
    if force_n == 0:
        avg_force_s = float("nan")
    tune = system.tuning()
    variant = tune["variant"]
    kernel = force_kernel_name(variant, periodic_mode)
    traffic = None
    # ncu DRAM bytes of one launch, used only while the kernel source is the
    # one the counters were taken on
    prof = os.path.join(ROOT, "profiles", "force_long_traffic_n1e5.json")
    if os.path.exists(prof) and args.workload == "n1e5":
        try:
            import hashlib
            with open(prof) as f:
                rec = json.load(f)
            src = "kernels_sym.cu" if variant >= 2 else "kernels_force.cu"
            with open(os.path.join(ROOT, "paper_1703_02484_gb300", "csrc", src), "rb") as f:
                h = hashlib.sha256(f.read()).hexdigest()[:16]
            if rec.get("kernel") == kernel and rec.get("kernel_source_sha256_16") == h:
                traffic = rec.get("traffic_bytes_per_launch")
        except Exception:
            traffic = None

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        hxy = torch.empty((N, 2), dtype=torch.float64).pin_memory().numpy()
        hth = torch.empty((N,), dtype=torch.float32).pin_memory().numpy()
        cur = system.state(want_tri=False)
        hxy[:] = cur["xy"]
        hth[:] = cur["theta"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            system.set_state(hxy, hth)          # host -> device (positions, directions)
            system.step(1)
            system.read_state(hxy, hth)         # device -> host
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te = max_over_ranks(te, ws, "cuda")
        e2e = {"value": ws * N * args.e2e_steps / te, "unit": UNIT,
               "h2d_bytes_per_step": N * (16 + 4), "d2h_bytes_per_step": N * (16 + 4)}

    if rank == 0:
        if args.workload != "n1e5":
            line_cfg = {"workload": "%s: N=%d, rho=%.2f, law=%d" % (args.workload, N, cfg.rho, cfg.law), "N": N}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "seed": cfg.seed,
                       "parallelism": "replicas%d" % ws,
                       "l2": "flushed between timed steps (256 MB write)",
                       "force_tuning": tune,
                       "per_step_stats": {k: v / args.steps for k, v in stats_tot.items()}},
            "roofline": force_roofline(N, avg_force_s, variant, periodic_mode, sms, f_hz, pk_kind, traffic),
            "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
        }
        if args.workload != "n1e5":
            line["metric"] = "particle-steps/s (%s)" % args.workload
            line["config"].update(line_cfg)
            if verlet_mode:
                line["config"]["overlap_pairs_from"] = "Verlet lists (no triangulation)"
            if periodic_mode:
                line["config"]["boundary"] = "periodic (minimum image, torus triangulation)"
        line["config"]["triangulation_stage_ms_per_step"] = stage_ms
        if not (avg_force_s > 0):
            # no all-pairs launch (short-range law): the dominant kernel is the
            # persistent correction kernel, bound by memory (gathers), so its
            # line is HBM bytes against the measured copy bandwidth
            line["roofline"] = correction_roofline(system, stage_raw, args.steps, N, verlet_mode, pk, pk_kind,
                                                   stats_tot.get("tri_visits", 0) / args.steps,
                                                   stats_tot.get("flips", 0) / args.steps)
        elif cfg.precision == 1:
            # FP64 sweep (one disk per thread, 12 FP64 flops per ordered pair);
            # FP64 issues at 1/64 of the FP32 rate on this part
            p64 = peak_tflops / 64.0
            a64 = FLOPS_PER_PAIR * pairs / avg_force_s / 1e12
            line["roofline"] = {"bound": "fp64", "kernel": "k_force_long_f64", "achieved": a64, "peak": p64,
                                "unit": "TFLOP/s", "frac": a64 / p64, "traffic": None,
                                "avg_launch_ms": avg_force_s * 1e3,
                                "peak_note": "FP32 peak / 64 (the part's FP64 issue rate)"}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(cfg, xy, sp, th, periodic_mode)
        print(json.dumps(line), flush=True)
    system.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

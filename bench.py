"""Benchmark: spin-flip attempts/s of replica-parallel Metropolis annealing.

Default workload (N = 1): an 80 x 100 +-1 torus (the shape of the Gset
spin-glass instance G65: 8,000 spins, 16,000 edges), 1,024 replicas packed 32
per word, geometric beta 0.1 -> 5.0 over 10,000 sweeps, one instance per
launch.  One step = one full anneal of that instance (all sweeps, energy and
best-state tracking, result unpacking) = 8.19e10 attempts.

  value      attempts/s, CUDA events around each step on the launching stream,
             instance already resident on the device; L2 flushed between steps.
  e2e        the same metric through the public C ABI with HOST buffers: each
             step creates the instance from host couplings, anneals, and reads
             final spins, energies and the best state back to the host.
  roofline   the sweep kernel's algorithmic integer-ALU instruction rate
             against the integer ALU pipe's peak (bound "alu").
  cpu_baseline  the CPU oracle on the host cores on a bounded replica sample.

Other workloads: --config random (n = 10,000, m = 9,999 random graph, 256
replicas), --config batch (512 uneven tori in one persistent kernel vs the
one-launch-per-sweep plain form), --config served (Poisson request stream).

--impl reference times the CPU oracle (the only reference this project has)
on the same workload, metric and unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2311_09275_gb300 import inputs as I  # noqa: E402

METRIC = "spin-flip attempts/s"
UNIT = "attempts/s"
# Integer instructions one attempt needs by the algorithm, per pipe: a quarter
# of a Philox4x32-10 block (10 rounds x 2 three-input XORs on the logic pipe,
# 10 rounds x 2 widening multiplies on the multiply pipe) plus one threshold
# compare (logic pipe).  The roofline takes the pipe whose share of the work
# needs the longer time at its measured rate (isg_integer_peaks).
ALGO_LOP3_PER_ATTEMPT = 20 / 4 + 1
ALGO_MUL_PER_ATTEMPT = 20 / 4
# Widening multiplies the torus kernel issues per attempt: per site and replica
# word (32 attempts) the two of the site's round-1/2 prefix and 8 blocks x 8
# remaining rounds x 2; the per-(block, sweep) prefix is shared by a whole band.
EXEC_MUL_PER_ATTEMPT = (2 + 8 * 8 * 2) / 32
SMSP_PER_SM = 4
ALU_LANES_PER_SMSP = 16  # nominal: the logic pipe takes half a warp instruction per cycle
MUL_LANES_PER_SMSP = 8   # nominal: a widening multiply holds the multiply pipe 4 cycles per warp
KERNEL_NAMES = {1: "torus_kernel", 2: "csr_kernel", 3: "plain per-sweep launches",
                4: "gm_kernel"}


def profiled_traffic(workload_name: str, kernel_name: str):
    """DRAM bytes per launch of a sweep kernel from the committed ncu summaries
    (profiles/*.md carrying `workload`, `kernel`, `kernel_sources`,
    `kernel_source_sha256_16` and `traffic_bytes_per_launch` lines), or None when
    no summary covers this workload and kernel or a source changed since."""
    import glob
    import hashlib
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith(("|", "#", " ", "`")):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("workload") != workload_name or fields.get("kernel") != kernel_name:
            continue
        h = hashlib.sha256()
        for rel in fields.get("kernel_sources", "").split(","):
            src = os.path.join(ROOT, "paper_2311_09275_gb300", "csrc", rel.strip())
            if not rel.strip() or not os.path.exists(src):
                return None
            with open(src, "rb") as f:
                h.update(f.read())
        if fields.get("kernel_source_sha256_16") != h.hexdigest()[:16]:
            return None
        try:
            return int(fields["traffic_bytes_per_launch"])
        except (KeyError, ValueError):
            return None
    return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if (torch.cuda.is_available() and args.impl != "reference") else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend, init_method="env://")
    return world, rank, local, dist


def max_over_ranks(x: float, dist, device) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def global_best(e_best: int, local_replica: int, first_replica: int, dist, device):
    """Final argmin of a replica-sharded solve: every rank's lowest best energy and
    its global replica index (first_replica + local index) gathered to all ranks;
    the overall best is the lowest energy, ties to the lowest global replica (the
    rule of isg_best within one call)."""
    mine = (int(e_best), int(first_replica) + int(local_replica))
    if dist is None:
        return mine
    import torch
    t = torch.tensor(mine, dtype=torch.int64, device=device)
    allv = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(allv, t)
    return min((int(x[0]), int(x[1])) for x in allv)


COLOURINGS = {"greedy": 0, "smallest-last": 1}


def workload(config: str, rank: int, sweeps: int | None = None, colouring: str = "greedy"):
    """The Solve of this rank and its first global replica.  Ranks anneal the
    same instance with the same seed, rank k its own replicas [kR, (k+1)R)
    (a replica-sharded solve of N x R replicas: weak scaling, no exchange but
    the final argmin).  `sweeps` shortens the schedule (profiling runs only;
    the benchmark line uses the full 10,000).  A graph workload coloured other
    than greedy by id names its colouring."""
    if config == "torus":
        sv = I.torus_80x100(sweeps=sweeps or 10000)
        name = f"torus_80x100_R1024_S{sv.sweeps}_geometric_0.1_5.0"
    elif config == "random":
        sv = I.random_10000(sweeps=sweeps or 10000)
        name = f"random_n10000_m9999_R256_S{sv.sweeps}_geometric_0.1_5.0"
    elif config == "mis":
        sv = I.independent_set_10000(sweeps=sweeps or 10000)
        name = f"independent_set_geometric_n10000_deg6_R256_S{sv.sweeps}_geometric_0.1_5.0"
    else:
        raise ValueError(config)
    if colouring != "greedy" and config != "torus":
        name += "_" + colouring.replace("-", "_")
    return sv, name, rank * sv.replicas


def oracle_colour(c, colouring: str):
    """The oracle's colour classes for the library's colouring of the same instance."""
    return (c.smallest_last_colouring() if colouring == "smallest-last" and c.torus_shape is None
            else c.colouring())[0]


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(sv, budget_s: float = 12.0, max_replicas: int | None = None,
                    colouring: str = "greedy"):
    """Oracle attempts/s on the host cores over a bounded sample of the workload:
    whole replicas (a multiple of the core count, one thread per replica block)
    over a sweep prefix, sized to about budget_s seconds; plus the rate of one
    thread on one replica."""
    import oracle
    cores = os.cpu_count() or 1
    c = oracle.csr_of(sv.problem)
    colour = oracle_colour(c, colouring)
    # calibrate on a short prefix, then size the sample to the budget
    reps = min(sv.replicas, max_replicas or cores)
    probe = max(1, min(sv.sweeps, 20))
    t0 = time.perf_counter()
    oracle.anneal(c, reps, sv.betas[:probe], sv.seed, colour=colour, nthreads=cores)
    rate = reps * sv.n * probe / max(time.perf_counter() - t0, 1e-6)
    sweeps = int(max(1, min(sv.sweeps, budget_s * rate / (reps * sv.n))))
    if sweeps == sv.sweeps and max_replicas is None:
        fit = int(budget_s * rate / (sv.n * sv.sweeps) // cores) * cores
        reps = max(reps, min(sv.replicas, fit))
    t0 = time.perf_counter()
    oracle.anneal(c, reps, sv.betas[:sweeps], sv.seed, colour=colour, nthreads=cores)
    dt = time.perf_counter() - t0
    one_sweeps = int(max(1, min(sv.sweeps, 2.0 * rate / cores / sv.n)))
    t1 = time.perf_counter()
    oracle.anneal(c, 1, sv.betas[:one_sweeps], sv.seed, colour=colour, nthreads=1)
    one = sv.n * one_sweeps / (time.perf_counter() - t1)
    return {"value": reps * sv.n * sweeps / dt, "unit": UNIT, "cores": min(cores, reps),
            "kind": "oracle", "single_thread_value": one,
            "sample": f"replicas 0..{reps - 1} of {sv.replicas}, first {sweeps} of {sv.sweeps} "
                      f"sweeps ({reps * sv.n * sweeps:.3g} attempts, {dt:.1f} s); single thread: "
                      f"replica 0, {one_sweeps} sweeps"}


def run_reference(args):
    world, rank, local, dist = dist_setup(args)
    if rank != 0:
        return
    if args.config not in ("torus", "random", "mis"):
        print(json.dumps({"impl": "reference", "unavailable":
                          f"the oracle arm times the single-instance workloads (torus, random, "
                          f"mis); --config {args.config} has no oracle timing line"}))
        return
    sv, name, _ = workload(args.config, 0, args.sweeps, args.colouring)
    import oracle
    cores = os.cpu_count() or 1
    reps = min(sv.replicas, cores)
    c = oracle.csr_of(sv.problem)
    colour = oracle_colour(c, args.colouring)
    # each step: `reps` replicas over a sweep prefix sized to ~per_step_s
    probe = 10
    t0 = time.perf_counter()
    oracle.anneal(c, reps, sv.betas[:probe], sv.seed, colour=colour, nthreads=cores)
    rate = reps * sv.n * probe / max(time.perf_counter() - t0, 1e-6)
    per_step_s = 4.0
    sweeps = int(max(1, min(sv.sweeps, per_step_s * rate / (reps * sv.n))))
    for _ in range(args.warmup):
        oracle.anneal(c, reps, sv.betas[:sweeps], sv.seed, colour=colour, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.anneal(c, reps, sv.betas[:sweeps], sv.seed, colour=colour, nthreads=cores)
    dt = time.perf_counter() - t0
    attempts = reps * sv.n * sweeps * args.steps
    value = attempts / dt
    sample = (f"each step: replicas 0..{reps - 1} of {sv.replicas}, first {sweeps} of "
              f"{sv.sweeps} sweeps ({reps * sv.n * sweeps:.3g} attempts)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": name, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(cores, reps),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    world, rank, local, dist = dist_setup(args)
    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2311_09275_gb300 import isg

    sv, name, first = workload(args.config, rank, args.sweeps, args.colouring)
    stream = torch.cuda.current_stream()
    p = isg.problem_of(sv.problem, colouring=COLOURINGS[args.colouring])
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=device)  # 512 MB > L2

    shape = {"kernel": args.kernel} if args.kernel else {}
    if args.launch:
        parts = [int(x) for x in args.launch.split(",")]
        shape.update({"cluster_ctas": parts[0], "threads": parts[1]})
        if len(parts) > 2:
            shape["quads_per_cta"] = parts[2]

    def step(time_kernels=True):
        return isg.isg_anneal(p, sv.replicas, sv.betas, sv.seed, stream=stream,
                              time_kernels=time_kernels, first_replica=first, **shape)

    # launch-shape autotuning (untimed, part of warm-up); results never depend on it
    tuned = None
    if not args.no_tune and not args.launch and not args.kernel:
        tuned = isg.isg_autotune(p, sv.replicas, 64, stream=stream)
    for _ in range(args.warmup):
        r = step()
        r.final(spins=False)
        r.close()

    # ---- device-timed steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    results = []
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k)
            ev[k][0].record(stream)
            results.append(step())
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier(dist)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kernel_ms, launches, sweep_launches = [], 0, 0
    stats = None
    for r in results:
        stats = r.stats()
        kernel_ms.append(stats["sweep_kernel_ms"])
        launches += stats["launches"]
        sweep_launches += stats["sweep_launches"]
    be, br, _, _, _ = results[-1].best(spins=False)       # outside the timed region
    best_e, best_r = global_best(be, br, first, dist, device)
    for r in results:
        r.close()
    dev_s = max_over_ranks(sum(step_ms) / 1e3, dist, device)
    attempts_rank = float(sv.attempts) * args.steps
    attempts_all = sum_over_ranks(attempts_rank, dist, device)
    value = attempts_all / dev_s

    # ---- end to end through the C ABI with host buffers
    e2e_steps = max(1, min(args.steps, 5))
    h2d = d2h = 0
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        q = isg.problem_of(sv.problem, colouring=COLOURINGS[args.colouring])  # host -> library
        r = isg.isg_anneal(q, sv.replicas, sv.betas, sv.seed, stream=stream)
        spins, energies, done = r.final(spins=True)           # D2H final state
        be, br, bspins, per, hit = r.best(spins=True)         # D2H best state
        h2d = r.stats()["h2d_bytes"]                          # instance arrays + thresholds
        r.close()
        q.close()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, device)
    # spins and energies read back: final [R][n] + energies [R] + sweeps, best [n] +
    # per-replica best [R] + energy, replica, hit
    d2h = spins.nbytes + energies.nbytes + 4 + bspins.nbytes + per.nbytes + 12
    e2e_value = sum_over_ranks(float(sv.attempts) * e2e_steps, dist, device) / e2e_s

    # ---- roofline of the sweep kernel (integer issue)
    pipes = isg.isg_integer_peaks(stream)
    philox = isg.isg_philox_rates(stream)
    props = torch.cuda.get_device_properties(device)
    peaks, _ = load_peaks()
    nominal_lop3 = (props.multi_processor_count * SMSP_PER_SM * ALU_LANES_PER_SMSP *
                    float(peaks.get("sm_max_mhz", 2070.0)) * 1e6)
    k_ms = statistics.mean(kernel_ms)
    rate = float(sv.attempts) / (k_ms / 1e3)                  # attempts/s of the sweep kernel
    t_lop3 = ALGO_LOP3_PER_ATTEMPT / pipes["lop3_per_s"]      # s per attempt at each pipe's peak
    t_mul = ALGO_MUL_PER_ATTEMPT / pipes["mul_wide_per_s"]
    if t_lop3 >= t_mul:
        pipe, ops, peak = "lop3 (logic pipe)", ALGO_LOP3_PER_ATTEMPT, pipes["lop3_per_s"]
    else:
        pipe, ops, peak = "mul.wide.u32 (multiply pipe)", ALGO_MUL_PER_ATTEMPT, pipes["mul_wide_per_s"]
    nominal_mul = (props.multi_processor_count * SMSP_PER_SM * MUL_LANES_PER_SMSP *
                   float(peaks.get("sm_max_mhz", 2070.0)) * 1e6)
    achieved = ops * rate
    kname = KERNEL_NAMES.get(stats["kernel"], "sweep kernel")
    traffic = profiled_traffic(name, kname)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": name, "replicas": sv.replicas, "spins": sv.n,
                   "sweeps": sv.sweeps, "attempts_per_step": sv.attempts,
                   "parallelism": (f"replica-sharded: rank k anneals replicas [k*{sv.replicas}, "
                                   f"(k+1)*{sv.replicas}) of one solve" if world > 1
                                   else "single GPU"),
                   "l2": "flushed (512 MB write) before every timed step",
                   "launch": {k: stats[k] for k in ("kernel", "ctas", "cluster_ctas", "threads")},
                   "autotuned": tuned is not None},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": e2e_steps},
        "gpu_launches": launches,
        # the solve's overall best over all ranks' replicas (final argmin gather)
        "global_best": {"energy": best_e, "replica": best_r, "replicas": sv.replicas * world},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": "T instr/s", "frac": achieved / peak, "traffic": traffic,
                     "kernel": kname, "kernel_ms": k_ms, "pipe": pipe,
                     "algorithmic_per_attempt": {"lop3": ALGO_LOP3_PER_ATTEMPT,
                                                 "mul.wide": ALGO_MUL_PER_ATTEMPT},
                     "frac_per_pipe": {"lop3": ALGO_LOP3_PER_ATTEMPT * rate / pipes["lop3_per_s"],
                                       "mul.wide": ALGO_MUL_PER_ATTEMPT * rate /
                                       pipes["mul_wide_per_s"]},
                     # the multiplies the torus kernel actually issues (rounds 1-2
                     # factored) against the same peak
                     "executed_mul_per_attempt": EXEC_MUL_PER_ATTEMPT,
                     "frac_executed": (EXEC_MUL_PER_ATTEMPT * rate / pipes["mul_wide_per_s"]
                                       if stats["kernel"] == 1 else None),
                     "peak_source": f"measured on this GPU by isg_integer_peaks: lop3 "
                                    f"{pipes['lop3_per_s'] / 1e12:.2f}T/s, mul.wide "
                                    f"{pipes['mul_wide_per_s'] / 1e12:.2f}T/s "
                                    f"({props.multi_processor_count} SMs)",
                     "nominal_lop3_peak": nominal_lop3 / 1e12,
                     "nominal_mul_peak": nominal_mul / 1e12,
                     # the sweeps' own Philox code alone (and with the threshold masks):
                     # one uniform per attempt, so an upper bound on the attempt rate
                     "random_number_ceiling": {
                         "uniforms_per_s": philox["uniforms_per_s"],
                         "with_masks_per_s": philox["masked_per_s"],
                         "frac": rate / philox["masked_per_s"]}},
        "clocks": clocks.summary(),
        "wall_s": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(sv, colouring=args.colouring)
    if rank == 0 and world == 1 and args.config == "torus" and not args.no_forms:
        # the batched and served forms on the same GPU, after the headline
        # measurement and outside its timed region, each with its own clock sample
        line["batched"] = batched_form(steps=3, warmup=1)
        line["served"] = served_form()
    if rank == 0:
        print(json.dumps(line))


# ---------------------------------------------------------------- batched form
def batched_form(steps: int, warmup: int, sweeps: int = 2000):
    """512 uneven tori (even L, W in [16, 140]), 32 replicas, 2,000 sweeps, in
    one persistent kernel launched through a CUDA graph; against the plain form
    (one instance per launch sequence, one launch per sweep) on a size-stratified
    sample of the same instances, and against one persistent launch per instance.
    Returns the measurements (with their own clock samples) as a dict."""
    import torch
    from paper_2311_09275_gb300 import isg
    stream = torch.cuda.current_stream()
    batch = I.torus_batch(sweeps=sweeps)
    probs = [isg.problem_of(sv.problem) for sv in batch]
    betas, seeds = batch[0].betas, [sv.seed for sv in batch]
    attempts = float(sum(sv.attempts for sv in batch))
    # launch shape measured for this size histogram (untimed; results never depend on it)
    tuned = isg.isg_autotune_batch(probs, 32, betas, probe_sweeps=128, stream=stream)
    for _ in range(warmup):
        for r in isg.isg_anneal_batch(probs, 32, betas, seeds, stream=stream):
            r.close()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for k in range(steps):
            ev[k][0].record(stream)
            outs = isg.isg_anneal_batch(probs, 32, betas, seeds, stream=stream)
            ev[k][1].record(stream)
            torch.cuda.synchronize()
            stats = outs[0].stats()
            for r in outs:
                r.close()
        ms = [a.elapsed_time(b) for a, b in ev]
        value = attempts * steps / (sum(ms) / 1e3)
        # plain forms on a sample: every 32nd instance in size order
        order = sorted(range(len(batch)), key=lambda k: batch[k].n)
        sample = order[::32]
        sample_attempts = float(sum(batch[k].attempts for k in sample))
        rates = {}
        for label, kernel in (("plain_one_launch_per_sweep", isg.KERNEL_PLAIN),
                              ("one_persistent_launch_per_instance", isg.KERNEL_AUTO)):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs = [isg.isg_anneal(probs[k], 32, betas, seeds[k], stream=stream, kernel=kernel)
                  for k in sample]
            e1.record(stream)
            torch.cuda.synchronize()
            for r in rs:
                r.close()
            rates[label] = sample_attempts / (e0.elapsed_time(e1) / 1e3)
    for p in probs:
        p.close()
    return {"workload": f"batch512_tori_L_W_even_16_140_R32_S{sweeps}_geometric_0.1_5.0",
            "attempts_per_s": value, "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": sum(ms) / steps, "attempts_per_step": attempts,
            "launch": f"CUDA graph: 1 persistent kernel ({stats['ctas']} CTAs x "
                      f"{stats['threads']} threads) + 1 unpack",
            "autotuned_shape": tuned,
            "gpu_launches_per_step": stats["launches"],
            "plain": {"sample": f"{len(sample)} instances (every 32nd by size)",
                      "attempts_per_s": rates},
            "batched_over_plain": {k: value / v for k, v in rates.items()},
            "clocks": clocks.summary()}


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    b = batched_form(args.steps, args.warmup, args.sweeps or 2000)
    line = {"metric": METRIC, "value": b["attempts_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": b["workload"], "attempts_per_step": b["attempts_per_step"],
                       "launch": b["launch"],
                       "l2": "working set of each CTA in shared memory; inputs ~12 MB"},
            "plain": dict(b["plain"], batched_over_plain=b["batched_over_plain"]),
            "gpu_launches": b["gpu_launches_per_step"], "clocks": b["clocks"]}
    print(json.dumps(line))


# ---------------------------------------------------------------- served form
def served_form(count: int = 2000, sweeps: int = 10000, slots: int = 512, chunk: int = 250,
                mem_gb: int = 32):
    """Poisson request stream (200/s): half +-1 tori 40..100 x 40..200, half
    random graphs of 2,000..20,000 vertices and mean degree 2..4; 32 replicas,
    10,000-sweep budget, target = the plain run's best over the full budget.
    Measures p50/p99 time-to-target (arrival -> result) and throughput; after
    the timed stream, 16 evenly spaced requests are compared with the same
    request run alone (tests/test_gpu_served_oracle.py checks a seeded sample of
    64 served requests against the oracle).  Returns the measurements as a dict."""
    import torch
    from paper_2311_09275_gb300 import isg, metrics
    reqs = I.served_stream(count=count, sweeps=sweeps)
    probs = [isg.problem_of(r.solve.problem) for r in reqs]
    # targets from plain runs of the full budget (batched through a server, untimed)
    srv = isg.Server(64 << 30, 512, 500)
    ids = {srv.submit(p, r.solve.replicas, r.solve.betas, r.solve.seed): k
           for k, (p, r) in enumerate(zip(probs, reqs))}
    targets = [None] * count
    while any(t is None for t in targets):
        got = srv.poll(60.0)
        assert got is not None, "target precomputation timed out"
        k = ids[got[0]]
        targets[k] = got[1].best(spins=False)[0]
        got[1].close()
    srv.close()
    # timed served run
    srv = isg.Server(mem_gb << 30, slots, chunk)
    t_submit, t_done, hit, attempts = {}, {}, {}, 0.0
    check = {j: None for j in range(0, count, max(1, count // 16))}
    kept = {}
    t0 = time.perf_counter()
    k = 0
    ids = {}
    with ClockSampler(torch.cuda.current_device()) as clocks:
        while len(t_done) < count:
            now = time.perf_counter() - t0
            while k < count and reqs[k].arrival_s <= now:
                rid = srv.submit(probs[k], reqs[k].solve.replicas, reqs[k].solve.betas,
                                 reqs[k].solve.seed, targets[k])
                ids[rid] = k
                t_submit[k] = t0 + reqs[k].arrival_s
                k += 1
            wait = (reqs[k].arrival_s - (time.perf_counter() - t0)) if k < count else 1.0
            got = srv.poll(max(0.0, min(wait, 0.05)))
            if got is None:
                continue
            j = ids[got[0]]
            t_done[j] = time.perf_counter()
            _, _, done = got[1].final(spins=False)
            hit[j] = got[1].best(spins=False)[4]
            attempts += reqs[j].solve.replicas * reqs[j].solve.n * done
            if j in check:
                kept[j] = got[1]  # checked after the timed region
            else:
                got[1].close()
    wall = time.perf_counter() - t0
    sstats = srv.stats()
    srv.close()
    # bit-exactness in the mix: sampled requests against the same request alone
    exact = 0
    for j in check:
        res, r = kept[j], reqs[j].solve
        solo = isg.isg_anneal(probs[j], r.replicas, r.betas, r.seed, target=targets[j])
        same = all(np.array_equal(a, b) for a, b in zip(res.final(), solo.final()))
        same = same and np.array_equal(res.best_all(), solo.best_all())
        same = same and res.best(spins=False)[4] == solo.best(spins=False)[4]
        exact += int(same)
        solo.close()
    for res in kept.values():
        res.close()
    for p in probs:
        p.close()
    ttt = [t_done[j] - t_submit[j] for j in range(count)]
    return {"workload": f"served_poisson200_{count}req_R32_B{sweeps}",
            "slots": slots, "sweeps_per_chunk": chunk, "device_mem_budget_gb": mem_gb,
            "ttt_p50_s": metrics.percentile(ttt, 50), "ttt_p99_s": metrics.percentile(ttt, 99),
            "attempts_per_s": attempts / wall, "requests_per_s": count / wall,
            "wall_s": wall, "requests": count,
            "targets_hit": sum(1 for j in range(count) if hit[j] >= 0),
            "peak_resident_slots": sstats["peak_active"], "chunk_passes": sstats["passes"],
            "bit_exact_vs_alone": f"{exact}/{len(check)} sampled requests",
            "clocks": clocks.summary()}


def run_served(args):
    import torch
    torch.cuda.set_device(0)
    f = served_form(args.requests, args.sweeps or 10000, args.slots, args.chunk, args.mem_gb)
    line = {"metric": "time-to-target (served)", "value": f["ttt_p99_s"], "unit": "s",
            "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": f["wall_s"] * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f["workload"], "slots": f["slots"],
                       "sweeps_per_chunk": f["sweeps_per_chunk"],
                       "device_mem_budget_gb": f["device_mem_budget_gb"]}}
    line.update({k: v for k, v in f.items() if k not in ("workload", "slots", "sweeps_per_chunk",
                                                          "device_mem_budget_gb")})
    line["throughput_attempts_per_s"] = f["attempts_per_s"]
    print(json.dumps(line))


# ---------------------------------------------------------------- parallel tempering
def run_pt(args):
    """Parallel tempering on the 80x100 torus: 32 temperature slots (geometric
    beta 0.2 -> 3.0) x 32 chains = 1,024 replicas, 1,000 rounds of 10 sweeps
    with an exchange step after each round (10,000 sweeps, the annealing
    workload's attempt count).  Device time covers sweeps and exchanges."""
    import torch
    from paper_2311_09275_gb300 import isg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    K, per_round = 32, 10
    rounds = (args.sweeps or 10000) // per_round
    betas = I.geometric_betas(0.2, 3.0, K)
    t = I.torus(80, 100, 1)
    p = isg.problem_of(t)
    attempts = 32.0 * K * t.L * t.W * rounds * per_round
    icm = args.icm
    for _ in range(args.warmup):
        isg.isg_parallel_tempering(p, betas, rounds, per_round, 1, stream=stream,
                                   icm_slots=icm).close()
    torch.cuda.synchronize()
    ms, res = [], None
    with ClockSampler(0) as clocks:
        for k in range(args.steps):
            r = isg.isg_parallel_tempering(p, betas, rounds, per_round, 1 + k, stream=stream,
                                           time_kernels=True, icm_slots=icm)
            ms.append(r.stats()["sweep_kernel_ms"])
            if res is not None:
                res.close()
            res = r
    acc, att = isg.isg_result_exchanges(res, K - 1)
    flips = isg.isg_result_cluster_flips(res, K)
    st = res.stats()
    best = res.best(spins=False)
    res.close()
    dev_s = sum(ms) / 1e3
    line = {"metric": METRIC, "value": attempts * args.steps / dev_s, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"tempering_torus_80x100_K{K}x32_rounds{rounds}x{per_round}"
                                   f"_geometric_0.2_3.0" + (f"_houdayer{icm}" if icm else ""),
                       "attempts_per_step": attempts, "cluster_move_slots": icm,
                       "launch": {k: st[k] for k in ("kernel", "ctas", "cluster_ctas", "threads")},
                       "l2": "state of each word in shared memory during a round"},
            "exchange_acceptance": [round(float(a) / float(b), 4) for a, b in zip(acc, att)],
            "best_energy": int(best[0]), "gpu_launches": st["launches"],
            "cluster_sites_flipped_per_round": [round(float(f) / rounds, 2) for f in flips],
            "clocks": clocks.summary()}
    print(json.dumps(line))


# ---------------------------------------------------------------- paper-style TTT
QUALITY_LEVELS = (0.99, 0.995, 0.997, 0.999, 1.0)
HEADLINE_QUALITY = 0.995


def run_ttt(args):
    """Sweeps-to-target and time-to-target (Sec. II.B, eq. (1)-(2)) on synthetic
    stand-ins with the shapes of Table I.  Each replica is one trial (one run of
    the schedule).  The target stands in for the best-known value: the best
    energy of a reference solve with four times the sweep budget and its own
    seed.  P_s = fraction of the budget run's replicas whose best energy is at
    or below the target; r from eq. (1); sweeps-to-target = budget x r;
    TTT = t_trial x r with t_trial the device time of one replica's run when
    all replicas share the GPU (kernel time / replicas), and the time until
    at least one of a batch of all replicas succeeds with 99 %.  Targets: cut
    values at several fractions of the reference cut (solution quality)."""
    import torch
    from paper_2311_09275_gb300 import isg, metrics
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sweeps = args.sweeps or 10000
    R = 1024
    betas = I.geometric_betas(0.1, 5.0, sweeps)
    ref_betas = I.geometric_betas(0.1, 5.0, 4 * sweeps)
    rows = []
    with ClockSampler(0) as clocks:
        for label, prob in I.table1_stand_ins():
            p = isg.problem_of(prob)
            total_w = p.total_weight
            ref = isg.isg_anneal(p, R, ref_betas, 7777, stream=stream)
            target = int(ref.best(spins=False)[0])
            ref.close()
            res = isg.isg_anneal(p, R, betas, 1, stream=stream, time_kernels=True)
            per = res.best(spins=False)[3]
            k_s = res.stats()["sweep_kernel_ms"] / 1e3
            res.close()
            row = {"instance": label, "n": p.n, "run_s": k_s,
                   "mean_best_energy": float(np.mean(per)), "targets": []}
            # targets at fractions of the reference cut (solution quality, Sec. II.B):
            # cut >= ceil(q * reference cut), i.e. E <= W - 2 ceil(q * cut_ref)
            cut_ref = metrics.cut_value(total_w, target)
            for q in QUALITY_LEVELS:
                cut_t = int(np.ceil(q * cut_ref - 1e-9))
                tgt = total_w - 2 * cut_t
                ps = float(np.mean(per <= tgt))
                p_batch = 1.0 - (1.0 - ps) ** R
                fin = (lambda x: x if np.isfinite(x) else None)
                row["targets"].append({
                    "quality": q, "target_cut": cut_t, "target_energy": tgt, "p_success": ps,
                    "repetitions": fin(metrics.repetitions(ps)),
                    "sweeps_to_target": fin(metrics.sweeps_to_target(sweeps, ps)),
                    "ttt_s_per_trial": fin(metrics.time_to_target(k_s / R, ps)),
                    "ttt_s_batch": fin(metrics.time_to_target(k_s, p_batch))})
            # MaxCut form (Sec. II.A): cut = (W - E) / 2; quality = cut / reference cut
            row["mean_quality"] = ((total_w - float(np.mean(per))) / 2.0 /
                                   metrics.cut_value(total_w, target))
            rows.append(row)
            p.close()
    head = next(t for t in rows[0]["targets"] if t["quality"] == HEADLINE_QUALITY)
    line = {"metric": "sweeps-to-target (99%)", "value": head["sweeps_to_target"],
            "unit": "sweeps", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * sum(x["run_s"] for x in rows), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"table1_stand_ins_R{R}_S{sweeps}_geometric_0.1_5.0",
                       "target": "best of a 4x-budget reference solve (1,024 replicas, seed 7777)",
                       "value_is": f"{rows[0]['instance']}, target cut = {HEADLINE_QUALITY} x "
                                   f"reference cut"},
            "instances": rows, "clocks": clocks.summary()}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--colouring", default="greedy", choices=list(COLOURINGS),
                    help="colour classes of a graph workload (default: greedy by id)")
    ap.add_argument("--config", default="torus",
                    choices=["torus", "random", "mis", "batch", "served", "ttt", "pt"])
    ap.add_argument("--requests", type=int, default=2000, help="served: number of requests")
    ap.add_argument("--slots", type=int, default=512, help="served: maximum resident requests")
    ap.add_argument("--chunk", type=int, default=250, help="served: sweeps per chunk")
    ap.add_argument("--mem-gb", type=int, default=32, help="served: device memory budget (GB)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload: skip the batched and served measurements")
    ap.add_argument("--kernel", type=int, default=0,
                    help="kernel family (1 torus, 2 colour-class int8, 3 plain, 4 graph "
                         "multi-spin; 0 = tuned)")
    ap.add_argument("--launch", default=None,
                    help="explicit launch shape CLUSTER,THREADS (skips the autotuner)")
    ap.add_argument("--icm", type=int, default=0,
                    help="pt: Houdayer cluster moves on the last ICM temperature slots")
    ap.add_argument("--sweeps", type=int, default=None,
                    help="shorter schedule for profiling captures (default: the full workload)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batch":
        run_batch(args)
    elif args.config == "served":
        run_served(args)
    elif args.config == "ttt":
        run_ttt(args)
    elif args.config == "pt":
        run_pt(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

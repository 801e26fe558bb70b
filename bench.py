"""Throughput of the MTP planner hot path on one node.

A step is one full planner iteration (Alg. 2: tensor sampling, interpolation,
local samples, batched rollout + cost, top-E, FP64 update) over one batch of
candidates, launched through the C ABI (mtp_plan_step).  The default workload
is the 7-link torque-controlled arm: 4096 candidates x 128 steps, Akima,
graph 8 x 32, beta 0.5, 64 elites.  Each rank plans its own independent
instance (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  The reference arm times the FP64 CPU oracle
on the host on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rollout-steps/s"
HEADLINE_METRIC = "rollout-steps/s & plan-steps/s at p99 re-plan latency, served/batched vs plain"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
SMS = 152
FP32_LANES_PER_SM = 128


ROLLOUT_KERNEL = {"pointmass": "k_rollout_pm", "chain": "k_rollout_chain",
                  "legged": "k_rollout_legged"}


def workload(name: str) -> dict:
    from paper_2505_01059_gb300 import workloads as W
    if name == "arm7":
        return W.chain()
    if name == "pointmass2":
        return W.pointmass()
    if name == "legged16":
        return W.legged()
    raise SystemExit(f"unknown workload {name}")


def workload_label(spec: dict, name: str) -> str:
    return (f"{name}: {spec['dyn']} n={spec['n']} d={spec['d']} B={spec['B']} H={spec['H']} "
            f"M={spec['M']} N={spec['N']} beta={spec['beta']} {spec['interp']} E={spec['E']}")


def flops_per_step(spec: dict) -> int:
    """FP32 flops (an FMA counts 2) of one rollout step of one candidate as the
    rollout kernel computes it; transcendental MUFU ops (sincos, sqrt, rsqrt)
    are not counted."""
    if spec["dyn"] == "chain":
        L = spec["n_links"]
        pairs = L * (L - 1) // 2
        cost = 6 * L + 12            # tip position, reach error, torque penalty, compensated add
        rhs = 3 * L                  # tau_j - tau_{j+1} - g l_j beta_j cos(phi_j)
        mass_matrix = 5 * pairs      # D_jk cos(phi_j - phi_k) below the diagonal
        velocity = 21 * L - 4        # O(L) prefix / suffix form of the velocity terms
        chol = L * (L - 1) + sum((L - 1 - j) * (2 * j + 1) for j in range(L))
        solves = 2 * L * L
        integrate = 4 * L
        return cost + rhs + mass_matrix + velocity + chol + solves + integrate
    if spec["dyn"] == "legged":
        L = spec["n_links"]
        cost = 2 * (L - 1) + 14                 # base height / pitch / velocity, torque penalty
        forces = 3 * L + 4 * L                  # torque and gravity terms; tip position / velocity
        contact_walk = 10 * L                   # back-walk of the contact points and their moments
        velocity = 21 * L                       # prefix / suffix velocity terms
        schur_rhs = 6 * L                       # Schur right-hand side
        factor = 24 * L                         # semiseparable Cholesky: 2 x 2 recursion per link
        solves = 18 * L                         # forward and backward solves with running 2-vectors
        integrate = 4 * L + 4 * L + 8
        return cost + forces + contact_walk + velocity + schur_rhs + factor + solves + integrate
    if spec["dyn"] == "pointmass":
        k = spec["n"]
        return 9 * k + 8 + len(spec.get("obs_c", [])) * (3 * k + 3)
    raise ValueError(spec["dyn"])


def peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def fp32_peak_tflops(sm_mhz: float) -> float:
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


KERNEL_HEADERS = ("paper_2505_01059_gb300/csrc/rollout_common.cuh",
                  "paper_2505_01059_gb300/csrc/mtp_device.cuh", "include/mtp.h")


def _code_text(path: str) -> str:
    """A C / CUDA source with its comments removed and its whitespace
    collapsed: what the compiler sees, less the prose."""
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_digest(kernel_file: str) -> str:
    """sha256 over the code of a rollout kernel's source file and of the
    headers it is compiled with (comments and whitespace left out), so that
    a change to the code of either retires its profile."""
    h = hashlib.sha256()
    for rel in ("paper_2505_01059_gb300/csrc/" + kernel_file,) + KERNEL_HEADERS:
        h.update(_code_text(os.path.join(ROOT, rel)).encode())
        h.update(b"\0")
    return h.hexdigest()


def profiled_traffic(kernel_file: str, summary: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current sources of the kernel (else None)."""
    prof = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(prof):
        return None
    text = open(prof).read()
    m_hash = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_bytes = re.search(r"dram_bytes_per_launch_full_workload:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != source_digest(kernel_file):
        return None
    return float(m_bytes.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"mtp_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for _, _, flags in rows:
            for nm, v in zip(names, flags):
                if v.lower() == "active":
                    seen.add(nm)
        busy = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(seen)}


def rank_spec(spec: dict, rank: int) -> dict:
    """Each rank plans its own independent instance: same workload, own seed."""
    return dict(spec, seed=spec["seed"] + 7919 * rank)


def max_over_ranks(value: float, pg, device) -> float:
    """The slowest rank's time (the contract's max over ranks)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds_max: float) -> float:
    """Whole-job throughput: units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_rate(spec: dict, seconds: float, sample_rows: int):
    """Single-thread FP64 oracle: full planner iterations on `sample_rows`
    candidates of the workload, repeated for about `seconds`."""
    import numpy as np

    import oracle
    from paper_2505_01059_gb300 import workloads as W
    s = dict(spec, B=sample_rows, E=min(spec["E"], sample_rows))
    mu, sigma = W.initial_distribution(s)
    x0 = np.array(s["x0"], np.float64)
    steps = 0
    its = 0
    t0 = time.perf_counter()
    while True:
        out = oracle.plan_iteration(s, its, x0, mu, sigma)
        mu, sigma = out["mu"], out["sigma"]
        its += 1
        steps += s["B"] * s["H"]
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return steps / dt, its / dt, its, dt


def run_reference(args, spec, name):
    world, rank, _ = dist_init()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2505_01059_gb300 import workloads as W
    # size each step's sample so that warm-up + timed steps take about
    # args.reference_seconds on one core
    probe = dict(spec, B=32, E=min(spec["E"], 32))
    mu, sigma = W.initial_distribution(probe)
    x0 = np.array(probe["x0"], np.float64)
    t0 = time.perf_counter()
    oracle.plan_iteration(probe, 0, x0, mu, sigma)
    rate = 32 * spec["H"] / max(time.perf_counter() - t0, 1e-6)
    rows = int(args.reference_seconds * rate / ((args.steps + args.warmup) * spec["H"]))
    rows = max(8, min(rows, spec["B"]))
    s = dict(spec, B=rows, E=min(spec["E"], rows))
    mu, sigma = W.initial_distribution(s)
    for it in range(args.warmup):
        out = oracle.plan_iteration(s, it, x0, mu, sigma)
        mu, sigma = out["mu"], out["sigma"]
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        out = oracle.plan_iteration(s, args.warmup + k, x0, mu, sigma)
        times.append(time.perf_counter() - t0)
        mu, sigma = out["mu"], out["sigma"]
    total = sum(times)
    value = rows * s["H"] * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_label(spec, name), "sample_rows_per_step": rows},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                         "sample": f"each step one planner iteration on {rows} of the "
                                   f"{spec['B']} candidates (FP64 C oracle, one thread)"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "headline_metric": HEADLINE_METRIC,
    }
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Batched vs plain on many uneven instances (one GPU): the plain form
    plans each instance with its own launches, one after the other on one
    stream; the batched form runs one CUDA graph per iteration for all."""
    import numpy as np
    import torch

    from paper_2505_01059_gb300 import _build, mtp
    from paper_2505_01059_gb300 import workloads as W
    _build.build_library()
    mtp.load_library()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    specs = W.batch(count=args.instances)
    handles = [mtp.mtp_create(s) for s in specs]
    b = mtp.mtp_batch_create(handles)
    tiles = mtp.mtp_batch_autotune(b)
    x0 = torch.tensor(np.concatenate([np.array(s["x0"], np.float32) for s in specs]), device=dev)
    us = torch.empty(b.ustar_offset[-1], device=dev)
    x0_each = [torch.tensor(s["x0"], dtype=torch.float32, device=dev) for s in specs]
    u_each = [torch.empty(s["n"], device=dev) for s in specs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    steps_per_iter = sum(s["B"] * s["H"] for s in specs)
    flops_per_iter = sum(flops_per_step(s) * s["B"] * s["H"] for s in specs)

    def timed(fn, k):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        for i in range(k):
            flush.zero_()
            st[i].record(stream)
            fn()
            en[i].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(c) for a, c in zip(st, en)) / k

    def batched():
        mtp.mtp_batch_plan_step(b, x0, 1, us)

    def plain():
        for h, xx, uu in zip(handles, x0_each, u_each):
            mtp.mtp_plan_step(h, xx, 1, uu)

    for _ in range(args.warmup):
        batched()
        plain()
    torch.cuda.synchronize()
    with ClockSampler(0) as clocks:
        ms_b = timed(batched, args.steps)
    ms_p = timed(plain, max(3, min(args.steps, 20)))
    value = steps_per_iter / (ms_b / 1e3)
    achieved = flops_per_iter / (ms_b / 1e3) / 1e12
    peak = fp32_peak_tflops(peaks().get("sm_max_mhz", 2070.0))
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch of {len(specs)} uneven instances (point masses k 2..12, "
                               f"chains 3..9 links, H 32..256, B 512..8192)",
                   "l2": "flushed between steps (256 MB write)",
                   "rollout_steps_per_iteration": steps_per_iter},
        "plan_steps_per_s": len(specs) / (ms_b / 1e3),
        "plain": {"ms_per_step": ms_p, "value": steps_per_iter / (ms_p / 1e3),
                  "plan_steps_per_s": len(specs) / (ms_p / 1e3)},
        "batched_over_plain": ms_p / ms_b,
        "whole_step_fp32": {"achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                            "frac": achieved / peak,
                            "note": "rollout flops of all instances over the whole iteration time"},
        "tiles": tiles, "clocks": clocks.summary(), "headline_metric": HEADLINE_METRIC,
    }
    print(json.dumps(line), flush=True)
    mtp.mtp_batch_destroy(b)
    for h in handles:
        mtp.mtp_destroy(h)


def run_ours(args, spec, name):
    import numpy as np
    import torch

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    from paper_2505_01059_gb300 import _build, mtp
    if rank == 0 or not os.path.exists(mtp.LIB_PATH):
        _build.build_library()
    if pg:
        pg.barrier()
    mtp.load_library()

    spec = rank_spec(spec, rank)  # independent instance per rank
    h = mtp.mtp_create(spec)
    s = h.sizes
    x0 = torch.tensor(spec["x0"], dtype=torch.float32, device=dev)
    ustar = torch.empty(s["n"], dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        mtp.mtp_plan_step(h, x0, 1, ustar)
    torch.cuda.synchronize()

    # timed region: mtp_plan_step as a user calls it (CUDA graph replay), one
    # iteration per step, L2 flushed between steps outside the step events
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            mtp.mtp_plan_step(h, x0, 1, ustar)
            ends[k].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if pg:
        pg.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), pg, dev)
    steps_per_iter = s["B"] * s["H"]
    value = job_rate(world, steps_per_iter * args.steps, total_ms / 1e3)
    plan_steps = job_rate(world, args.steps, total_ms / 1e3)

    # stage pass over the same number of steps (at most 500): the same
    # kernels launched directly with CUDA events between them on the launch
    # stream, for the per-stage times and the rollout kernel's duration; a
    # pipelined handle's preparation of the next iteration is timed on its
    # own stream (it overlaps the rollout)
    hp = mtp.mtp_create(dict(spec, flags=spec.get("flags", 0) | mtp.FLAG_NO_GRAPH))
    for _ in range(3):
        mtp.mtp_plan_step(hp, x0, 1, ustar)
    mtp.mtp_set_profiling(hp, True)
    n_stage = min(args.steps, 500)
    for k in range(n_stage):
        flush.zero_()
        mtp.mtp_plan_step(hp, x0, 1, ustar)
    torch.cuda.synchronize()
    stage5, n_it = mtp.mtp_stage_times5(hp)
    stage_ms, prep_ms = stage5[:4], stage5[4]
    mtp.mtp_destroy(hp)

    # end to end through the host-pointer entry point: pinned x0 in, u* out
    x0_h = torch.tensor(spec["x0"], dtype=torch.float32).pin_memory()
    u_h = torch.empty(s["n"], dtype=torch.float32).pin_memory()
    lat = []
    n_e2e = min(args.steps, 2000)
    for _ in range(min(args.warmup, 10)):
        mtp.mtp_plan_step_host(h, x0_h, 1, u_h)
    for _ in range(n_e2e):
        flush.zero_()  # L2 flushed between calls as between the timed steps, outside the timing
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mtp.mtp_plan_step_host(h, x0_h, 1, u_h)
        lat.append(time.perf_counter() - t0)
    e2e_total = max_over_ranks(sum(lat), pg, dev)
    e2e_value = job_rate(world, steps_per_iter * n_e2e, e2e_total)
    lat_sorted = sorted(lat)
    p50 = 1e3 * lat_sorted[len(lat) // 2]
    p99 = 1e3 * lat_sorted[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]

    # roofline of the dominant kernel (the fused rollout): FP32 ALU bound
    rollout_ms = stage_ms[1] / max(n_it, 1)
    fl = flops_per_step(spec) * steps_per_iter
    achieved = fl / (rollout_ms / 1e3) / 1e12
    pk = peaks()
    clk = clocks.summary()
    peak_mhz = pk.get("sm_max_mhz", 2070.0)
    peak = fp32_peak_tflops(peak_mhz)
    kernel_file = "rollout.cu"
    summary = {"chain": "rollout_chain7_arm_B4096.txt", "pointmass": "rollout_pointmass2_B512.txt",
               "legged": "rollout_legged16_B16384.txt"}[spec["dyn"]]
    if spec["dyn"] == "legged":
        kernel_file = "legged.cu"
    traffic = profiled_traffic(kernel_file, summary)
    share = {st: ms / max(sum(stage_ms), 1e-12) for st, ms in
             zip(("generate", "rollout", "select", "update"), stage_ms)}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            r_steps, r_plans, its, dt = cpu_oracle_rate(spec, args.cpu_seconds, args.reference_rows)
            cpu = {"value": r_steps, "unit": METRIC, "cores": 1, "kind": "oracle",
                   "sample": f"{its} planner iterations on {args.reference_rows} of the "
                             f"{spec['B']} candidates in {dt:.1f} s (FP64 C oracle, one thread)"}
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_label(spec, name), "parallelism": f"replicas{world}",
                       "iters_per_step": 1, "l2": "flushed between steps (256 MB write)",
                       "timed_mode": "CUDA graph replay of mtp_plan_step (the default path)"},
            "plan_steps_per_s": plan_steps,
            "replan_latency_ms": {"p50": p50, "p99": p99, "path": "mtp_plan_step_host"},
            "stage_pass_ms_per_step": sum(stage_ms) / max(n_it, 1),
            "stage_ms_per_step": dict(zip(("generate", "rollout", "select", "update"),
                                          [v / max(n_it, 1) for v in stage_ms])),
            "stage_share": share,
            "pipelined": {0: "no", 1: "graph rows", 2: "graph rows and draws"}[s["pipelined"]],
            "prepare_overlapped_ms_per_step": prep_ms / max(n_it, 1),
            "roofline": {"bound": "alu", "kernel": ROLLOUT_KERNEL[spec["dyn"]],
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "flops_per_launch": fl,
                         "duration_us": rollout_ms * 1e3,
                         "timing": f"CUDA events around the rollout launch on its stream, "
                                   f"{n_it} iterations of the stage pass (kernels launched "
                                   f"directly, L2 flushed between steps)",
                         "peak_note": f"FP32 FMA: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                                      f"{peak_mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": 4 * s["d"],
                    "d2h_bytes_per_step": 4 * s["n"],
                    "timing": "host clock around each mtp_plan_step_host call (pinned x0 in, "
                              "u* out, synchronised); L2 flushed before each call, outside it"},
            "gpu_launches": s["kernels_per_iteration"] * args.steps,
            "clocks": clk,
            "headline_metric": HEADLINE_METRIC,
            "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
    mtp.mtp_destroy(h)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def _advance(x, u, dt):
    """Host stand-in for the robots' true motion between re-plans: one control
    step of a double integrator per controlled coordinate (point masses: the
    position; arms: the joint angles, unit inertia), FP64."""
    import numpy as np
    half = x.shape[0] // 2
    v = x[half:] + dt * u[:half]
    return np.concatenate([x[:half] + dt * v, v])


def run_serve(args):
    """The re-plan server under the fleet workload: every robot is an
    independent Poisson process of re-plan requests at --rate-hz (open loop),
    its next start state the previous one advanced on the host with the
    returned control.  Reports completed re-plans/s, rollout-steps/s and the
    submit -> poll-success latency; then the saturation capacity (closed
    loop, every robot resubmits at once) and the plain path's capacity (one
    request at a time through mtp_plan_step_host on its own handle)."""
    import time

    import numpy as np
    import torch

    from paper_2505_01059_gb300 import _build, mtp
    from paper_2505_01059_gb300 import workloads as W
    _build.build_library()
    mtp.load_library()
    torch.cuda.set_device(0)
    specs = W.robots(count=args.instances)
    R = len(specs)
    srv = mtp.mtp_server_create(max_batch=args.max_batch, iters_per_request=1, shift_after=1,
                                max_queue=8, max_robots=R)
    ids = np.array([mtp.mtp_server_register(srv, s) for s in specs], dtype=np.int32)
    d = np.array([s["d"] for s in specs])
    n = np.array([s["n"] for s in specs])
    steps_of = np.array([s["B"] * s["H"] for s in specs], dtype=np.float64)
    rng = np.random.default_rng(4)
    state = [np.asarray(s["x0"], np.float64) + rng.uniform(-0.1, 0.1, size=s["d"]) for s in specs]
    dts = [s["dt"] for s in specs]

    refused = [0]

    def open_loop(seconds, record):
        """Poisson arrivals; returns (completed, rollout steps, latencies)."""
        t0 = time.perf_counter()
        next_t = t0 + rng.exponential(1.0 / args.rate_hz, size=R)
        out_t, out_r, out_sub = [], [], []  # outstanding tickets, robots, submit times
        done = 0
        steps = 0.0
        lat = []
        while True:
            now = time.perf_counter()
            if now - t0 >= seconds and not out_t:
                break
            if now - t0 < seconds:
                due = np.nonzero(next_t <= now)[0]
                if len(due):
                    next_t[due] += rng.exponential(1.0 / args.rate_hz, size=len(due))
                while len(due):
                    x0 = np.concatenate([state[r] for r in due]).astype(np.float32)
                    try:
                        ts = mtp.mtp_submit_many(srv, ids[due], x0)
                        skip = 0
                    except mtp.MtpError as e:  # a full queue drops that arrival
                        if e.status != 4:
                            raise
                        ts, skip = e.tickets, 1
                        refused[0] += record
                    k = len(ts)
                    out_t.extend(ts.tolist())
                    out_r.extend(due[:k].tolist())
                    out_sub.extend([now] * k)
                    due = due[k + skip:]
            if out_t:
                status, u, ready = mtp.mtp_poll_many(srv, np.array(out_t, np.uint64), 32, 0.0)
                if ready:
                    t_obs = time.perf_counter()
                    keep_t, keep_r, keep_s = [], [], []
                    for k, st in enumerate(status):
                        r = out_r[k]
                        if st == 0:
                            state[r] = _advance(state[r], u[k, :n[r]].astype(np.float64), dts[r])
                            done += 1
                            steps += steps_of[r]
                            if record:
                                lat.append(t_obs - out_sub[k])
                        elif st in (5, 6):
                            keep_t.append(out_t[k])
                            keep_r.append(r)
                            keep_s.append(out_sub[k])
                        else:
                            raise RuntimeError(f"serving poll failed: status {st}")
                    out_t, out_r, out_sub = keep_t, keep_r, keep_s
                    continue
            time.sleep(100e-6)
        return done, steps, lat

    open_loop(args.serve_warmup, False)
    s0 = mtp.mtp_server_get_stats(srv)
    with ClockSampler(0) as clocks:
        t0 = time.perf_counter()
        done, steps, lat = open_loop(args.serve_seconds, True)
        wall = time.perf_counter() - t0
    s1 = mtp.mtp_server_get_stats(srv)
    lat_ms = np.sort(np.array(lat)) * 1e3
    value = steps / wall
    cycles = s1["cycles"] - s0["cycles"]

    # saturation: all robots resubmit at once, several rounds
    def closed_loop(k):
        t0 = time.perf_counter()
        for _ in range(k):
            ts = mtp.mtp_submit_many(srv, ids, np.concatenate([state[r] for r in range(R)]).astype(np.float32))
            status, _, ready = mtp.mtp_poll_many(srv, ts, 32, 60.0)
            if ready != R:
                raise RuntimeError("serving request timed out")
        return time.perf_counter() - t0

    closed_loop(2)
    k_sat = 10
    t_sat = closed_loop(k_sat)
    srv.close()
    # the plain path: one request at a time on its own handle
    sample = list(range(0, R, max(1, R // 64)))
    hs = {r: mtp.mtp_create(specs[r]) for r in sample}
    u = np.empty(32, np.float32)
    for r in sample:
        mtp.mtp_plan_step_host(hs[r], state[r].astype(np.float32), 1, u)
    t0 = time.perf_counter()
    for _ in range(3):
        for r in sample:
            mtp.mtp_plan_step_host(hs[r], state[r].astype(np.float32), 1, u)
            mtp.mtp_shift(hs[r], 1)
    t_plain = (time.perf_counter() - t0) / (3 * len(sample))
    torch.cuda.synchronize()
    for h in hs.values():
        mtp.mtp_destroy(h)
    sat_rps = R * k_sat / t_sat
    plain_rps = 1.0 / t_plain
    mean_steps = float(steps_of.mean())
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": done,
        "warmup": args.warmup, "ms_per_step": wall / max(done, 1) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"re-plan server, {R} robots (2-D point masses and 3..9-link arms, "
                               f"H 64..128, B 1024..4096), each a Poisson process at "
                               f"{args.rate_hz:g} Hz; 1 iteration + shift per request; "
                               f"max_batch {args.max_batch}; {args.serve_seconds:g} s after "
                               f"{args.serve_warmup:g} s warm-up",
                   "l2": "not flushed: the robots' candidate tensors together exceed L2",
                   "step": "one completed re-plan"},
        "offered_requests_per_s": R * args.rate_hz,
        "refused": refused[0],
        "requests_per_s": done / wall,
        "latency_p50_ms": float(lat_ms[len(lat_ms) // 2]) if len(lat_ms) else None,
        "latency_p99_ms": float(lat_ms[min(len(lat_ms) - 1, int(0.99 * len(lat_ms)))]) if len(lat_ms) else None,
        "latency": "mtp_submit -> mtp_poll success, host wall time, polled every ~0.1 ms",
        "mean_robots_per_cycle": (s1["planned"] - s0["planned"]) / max(cycles, 1),
        "saturation": {"requests_per_s": sat_rps, "rollout_steps_per_s": sat_rps * mean_steps,
                       "note": "closed loop: all robots resubmit together"},
        "plain": {"requests_per_s": plain_rps, "rollout_steps_per_s": plain_rps * mean_steps,
                  "latency_ms": t_plain * 1e3,
                  "note": f"mtp_plan_step_host + mtp_shift one request at a time, {len(sample)} robots"},
        "served_over_plain_capacity": sat_rps / plain_rps,
        "e2e": {"value": value, "unit": METRIC,
                "h2d_bytes_per_step": float(4 * d.mean()), "d2h_bytes_per_step": float(4 * n.mean())},
        "clocks": clocks.summary(), "headline_metric": HEADLINE_METRIC,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="arm7", choices=["arm7", "pointmass2", "legged16", "batch", "serve"])
    ap.add_argument("--instances", type=int, default=None,
                    help="batch: instances (256); serve: robots (1024)")
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--rate-hz", type=float, default=50.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-warmup", type=float, default=2.0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--reference-rows", type=int, default=512)
    ap.add_argument("--reference-seconds", type=float, default=90.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.instances is None:
        args.instances = 1024 if args.workload == "serve" else 256
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    spec = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, spec, args.workload)
    else:
        run_ours(args, spec, args.workload)


if __name__ == "__main__":
    main()

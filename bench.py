"""Throughput of the MTP planner hot path on one node: batched and served
planning against the plain one-instance-per-launch planner.

A step is one full planner iteration (Alg. 2: tensor sampling,
interpolation, local samples, batched rollout + cost, top-E, FP64 update)
of every instance of the batched workload: 256 independent instances of
uneven size (point masses with 2..12 axes and 3..9-link arms, H 32..256,
512..8192 candidates, graph 4..16 x 8..64, B-spline or Akima), the B-spline
instances contracting their basis with BF16 operands, all planned by one
mtp_batch_plan_step (one CUDA graph per iteration).  Beside it the same
instances in FP32 through the plain path (one mtp_plan_step per instance, in
turn on one stream), the re-plan server under the 1024-robot Poisson fleet
against the plain path serving the same request stream one request at a
time (plan-steps/s compared at a matched p99 latency), and the single-
instance 7-link arm and 16-link legged workloads.  Each rank plans its own
independent batch (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batch|serve|arm7|legged16|pointmass2|sweep]

Prints one JSON line (rank 0).  The reference arm times the FP64 CPU oracle
on the host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import collections
import gc
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

METRIC = "rollout-steps/s & plan-steps/s at p99 re-plan latency, served/batched vs plain"
UNIT = "rollout-steps/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
FP32_LANES_PER_SM = 128


ROLLOUT_KERNEL = {"pointmass": "k_rollout_pm", "chain": "k_rollout_chain",
                  "legged": "k_rollout_legged"}
DYN_NAMES = {0: "pointmass", 1: "chain", 2: "legged"}
ROLLOUT_MODES = {"groups": 0, "persistent-staged": 1, "persistent-direct": 2, "persistent-split": 3}


def workload(name: str, B: int | None = None) -> dict:
    """A single-instance workload; B overrides its candidate count (a
    smaller case of the same kernel, for profiler captures)."""
    from paper_2505_01059_gb300 import workloads as W
    over = {"B": B} if B else {}
    if name == "arm7":
        return W.chain(**over)
    if name == "pointmass2":
        return W.pointmass(**over)
    if name == "legged16":
        return W.legged(**over)
    raise SystemExit(f"unknown workload {name}")


def workload_label(spec: dict, name: str) -> str:
    bf16 = " bf16-basis" if spec.get("flags", 0) & 0x4 else ""
    return (f"{name}: {spec['dyn']} n={spec['n']} d={spec['d']} B={spec['B']} H={spec['H']} "
            f"M={spec['M']} N={spec['N']} beta={spec['beta']} {spec['interp']}{bf16} E={spec['E']}")


BATCH_LABEL = ("batched: 256 uneven instances (point masses k 2..12 and 3..9-link arms, H 32..256, "
               "B 512..8192, M 4..16, N 8..64, B-spline with BF16 basis operands or Akima), "
               "one mtp_batch_plan_step per iteration (CUDA graph), vs the same instances in FP32 "
               "through the plain path")


# chains of at least this many links use the semiseparable mass-matrix solve
# (kSemisepLinks of the rollout kernels)
SEMISEP_LINKS = 8


def flops_per_step(spec: dict) -> int:
    """FP32 flops (an FMA counts 2) of one rollout step of one candidate as the
    rollout kernel computes it; transcendental MUFU ops (sincos, sqrt, rsqrt)
    are not counted."""
    if spec["dyn"] == "chain":
        L = spec["n_links"]
        pairs = L * (L - 1) // 2
        cost = 6 * L + 12            # tip position, reach error, torque penalty, compensated add
        rhs = 3 * L                  # tau_j - tau_{j+1} - g l_j beta_j cos(phi_j)
        velocity = 21 * L - 4        # O(L) prefix / suffix form of the velocity terms
        integrate = 4 * L
        if L >= SEMISEP_LINKS:
            # rank-2 semiseparable Cholesky (2 x 2 recursion per link) and the
            # forward / backward solves with running 2-vectors
            mass_matrix, chol, solves = 0, 24 * L, 18 * L
        else:
            mass_matrix = 5 * pairs  # D_jk cos(phi_j - phi_k) below the diagonal
            chol = L * (L - 1) + sum((L - 1 - j) * (2 * j + 1) for j in range(L))
            solves = 2 * L * L
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


def device_sms(dev: int = 0) -> int:
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def fp32_peak(sm_mhz: float, sms: int) -> tuple[float, str]:
    """FP32 FMA peak (TFLOP/s) of this device and how it was derived."""
    tf = sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    return tf, (f"FP32 FMA: {sms} SMs (queried) x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz "
                f"(sm_max_mhz of MEASURED_PEAKS.json)")


KERNEL_HEADERS = ("paper_2505_01059_gb300/csrc/rollout_common.cuh",
                  "paper_2505_01059_gb300/csrc/rollout_kernels.cuh",
                  "paper_2505_01059_gb300/csrc/mtp_device.cuh", "include/mtp.h")
KERNEL_FILE = {"pointmass": "rollout_pm.cu", "chain": "rollout_chain.cu", "legged": "legged.cu"}
BATCH_KERNEL_FILE = {"pointmass": "rollout_pm_batch.cu", "chain": "rollout_chain_batch.cu",
                     "legged": "legged.cu"}


def _code_text(path: str) -> str:
    """A C / CUDA source with its comments removed and its whitespace
    collapsed: what the compiler sees, less the prose.  Of the public header
    only the types, constants and macros count: its function prototypes are
    the host interface, which no kernel is compiled from."""
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    if path.endswith(os.path.join("include", "mtp.h")):
        text = re.sub(r"\b(?:mtp_status|const\s+char\s*\*)\s*\w+\s*\([^;{]*\)\s*;", " ", text)
    return " ".join(text.split())


def source_digest(kernel_file: str) -> str:
    """sha256 over the code of a kernel's source file and of the headers it
    is compiled with (comments and whitespace left out), so that a change to
    the code of either retires its profile."""
    h = hashlib.sha256()
    for rel in ("paper_2505_01059_gb300/csrc/" + kernel_file,) + KERNEL_HEADERS:
        h.update(_code_text(os.path.join(ROOT, rel)).encode())
        h.update(b"\0")
    return h.hexdigest()


def profiled_traffic(kernel_file: str, summary: str, key: str = "dram_bytes_per_launch_full_workload"):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current sources of the kernel (else None)."""
    prof = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(prof) or not os.path.exists(
            os.path.join(ROOT, "paper_2505_01059_gb300/csrc", kernel_file)):
        return None
    text = open(prof).read()
    # a summary covering several kernel files names each one's digest
    m_hash = (re.search(r"source_sha256 " + re.escape(kernel_file) + r":\s*([0-9a-f]{64})", text) or
              re.search(r"source_sha256:\s*([0-9a-f]{64})", text))
    m_bytes = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", text)
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
        self.path = os.path.join("/tmp", f"mtp_clocks_{os.getpid()}_{gpu_index}.csv")

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


def percentile(sorted_vals, q: float):
    if not sorted_vals:
        return None
    k = min(len(sorted_vals) - 1, max(0, int(math.ceil(q * len(sorted_vals))) - 1))
    return float(sorted_vals[k])


# ----------------------------------------------------------------------------
# processes and ranks
# ----------------------------------------------------------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


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


def rank_specs(specs: list[dict], rank: int) -> list[dict]:
    """Each rank plans its own independent instances: same shapes, own seeds."""
    return [dict(s, seed=s["seed"] + 7919 * rank) for s in specs]


def host_cpu() -> dict:
    """Host cores and CPU model (nproc / lscpu)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cores": int(cores or 1), "model": model}


def setup_gpu(local: int, world: int):
    """Device, process group (NCCL for N > 1: only the contract's barrier and
    max-over-ranks use it) and the loaded library."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    from paper_2505_01059_gb300 import _build, mtp
    rank = int(os.environ.get("RANK", "0"))
    if rank == 0 or not os.path.exists(mtp.LIB_PATH):
        _build.build_library()
    if pg:
        pg.barrier()
    mtp.load_library()
    return dev, pg, mtp


# ----------------------------------------------------------------------------
# CPU oracle timings (the oracle is only ever called here, in the CPU legs)
# ----------------------------------------------------------------------------

def cpu_oracle_batch(specs: list[dict], seconds: float, threads: int) -> dict:
    """The FP64 oracle (as it stands) planning a sample of every instance:
    one Alg. 2 iteration per instance on its first `rows` candidates, the
    rollouts spread over `threads` host threads, `rows` sized so that the
    pass takes about `seconds`."""
    import numpy as np

    import oracle
    from paper_2505_01059_gb300 import workloads as W

    def one_pass(rows: int):
        steps = 0
        t0 = time.perf_counter()
        for spec in specs:
            r = min(rows, spec["B"])
            s = dict(spec, B=r, E=min(spec["E"], r))
            mu, sigma = W.initial_distribution(s)
            oracle.plan_iteration(s, 0, np.array(s["x0"], np.float64), mu, sigma, threads=threads)
            steps += r * s["H"]
        return steps, time.perf_counter() - t0

    probe_rows = max(2, 2 * threads)
    steps, dt = one_pass(probe_rows)
    rows = int(probe_rows * seconds / max(dt, 1e-3))
    rows = max(probe_rows, min(rows, max(s["B"] for s in specs)))
    steps, dt = one_pass(rows)
    return {"value": steps / dt, "rows_per_instance": rows, "seconds": dt, "steps": steps,
            "instances": len(specs)}


def cpu_oracle_single(spec: dict, seconds: float, threads: int) -> dict:
    """The FP64 oracle planning full iterations of one instance on a row
    sample sized to take about `seconds`."""
    import numpy as np

    import oracle
    from paper_2505_01059_gb300 import workloads as W
    probe = max(4, 2 * threads)
    s = dict(spec, B=probe, E=min(spec["E"], probe))
    mu, sigma = W.initial_distribution(s)
    x0 = np.array(s["x0"], np.float64)
    t0 = time.perf_counter()
    oracle.plan_iteration(s, 0, x0, mu, sigma, threads=threads)
    rows = int(probe * seconds / max(time.perf_counter() - t0, 1e-4))
    rows = max(probe, min(rows, spec["B"]))
    s = dict(spec, B=rows, E=min(spec["E"], rows))
    mu, sigma = W.initial_distribution(s)
    t0 = time.perf_counter()
    oracle.plan_iteration(s, 0, x0, mu, sigma, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": rows * s["H"] / dt, "rows": rows, "seconds": dt}


def run_reference(args):
    """The FP64 CPU oracle on the host cores (the reference arm): each step
    one Alg. 2 iteration of every instance of the batched workload on a row
    sample, sized so that warm-up and timed steps take about
    --reference-seconds."""
    world, rank, _ = dist_init()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2505_01059_gb300 import workloads as W
    specs = W.batch(count=args.instances, bf16=True)
    cpu = host_cpu()
    threads = cpu["cores"]
    per_step = args.reference_seconds / (args.steps + args.warmup)
    probe = cpu_oracle_batch(specs, min(per_step, 5.0), threads)
    rows = probe["rows_per_instance"]
    rows = max(2, int(rows * per_step / max(probe["seconds"], 1e-3)))
    rows = min(rows, max(s["B"] for s in specs))
    samples = [dict(s, B=min(rows, s["B"]), E=min(s["E"], min(rows, s["B"]))) for s in specs]
    state = [W.initial_distribution(s) for s in samples]
    x0s = [np.array(s["x0"], np.float64) for s in samples]

    def step(it):
        for i, s in enumerate(samples):
            out = oracle.plan_iteration(s, it, x0s[i], *state[i], threads=threads)
            state[i] = (out["mu"], out["sigma"])

    for it in range(args.warmup):
        step(it)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        step(args.warmup + k)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    steps_per_iter = sum(s["B"] * s["H"] for s in samples)
    value = steps_per_iter * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BATCH_LABEL, "sample_rows_per_instance": rows},
        "plan_steps_per_s": len(samples) * args.steps / total,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "cpu_model": cpu["model"],
                         "sample": f"each step one Alg. 2 iteration of all {len(samples)} instances "
                                   f"on their first {rows} candidates (FP64 C oracle, rollouts on "
                                   f"{threads} threads)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the batched workload: batched vs plain
# ----------------------------------------------------------------------------

def time_steps(fn, k: int, flush, stream) -> list[float]:
    """Device milliseconds of k calls of fn, CUDA events on `stream`, L2
    flushed before each call outside its events."""
    import torch
    st = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    for i in range(k):
        flush.zero_()
        st[i].record(stream)
        fn()
        en[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(st, en)]


def batch_rollout_roofline(mtp, b, specs, sms: int) -> tuple[dict, list]:
    """Each (dynamics, dimension) group's rollout launch timed alone with
    CUDA events on its stream; achieved FP32 flops over that time against
    the FP32 peak.  The dominant kernel is the group rollout with the
    largest device time."""
    groups = mtp.mtp_batch_rollout_times(b, reps=5)
    peak_mhz = peaks().get("sm_max_mhz", 2070.0)
    peak, note = fp32_peak(peak_mhz, sms)
    out = []
    for g in groups:
        dyn = DYN_NAMES[g["dyn"]]
        members = [s for s in specs if s["dyn"] == dyn and
                   (s["n"] if dyn == "pointmass" else s["n_links"]) == g["dim"]]
        fl = sum(flops_per_step(s) * s["B"] * s["H"] for s in members)
        achieved = fl / (g["ms"] / 1e3) / 1e12
        out.append({"kernel": f"{ROLLOUT_KERNEL[dyn]}_batch<{g['dim']}>", "dyn": dyn,
                    "dim": g["dim"], "block": g["block"], "chunk": g["chunk"],
                    "samples_per_thread": g["samples"],
                    "instances": g["instances"],
                    "rollout_steps": g["steps"], "flops_per_launch": fl,
                    "duration_us": g["ms"] * 1e3, "achieved_tflops": achieved,
                    "frac": achieved / peak})
    dom = max(out, key=lambda r: r["duration_us"])
    roof = {"bound": "alu", "kernel": dom["kernel"], "achieved": dom["achieved_tflops"],
            "peak": peak, "unit": "TFLOP/s", "frac": dom["frac"],
            "traffic": profiled_traffic(BATCH_KERNEL_FILE[dom["dyn"]], "rollout_batch_groups.txt",
                                        key=f"dram_bytes_per_launch_{dom['dyn']}{dom['dim']}"),
            "flops_per_launch": dom["flops_per_launch"], "duration_us": dom["duration_us"],
            "timing": "CUDA events around the group's rollout launch, run alone on its stream "
                      "with its tuned tile (5 launches averaged), after the timed region",
            "peak_note": note + " (of measured clock)"}
    return roof, out


def run_batch_arms(args, mtp, dev, pg, world, rank) -> dict:
    """The batched workload (timed region) and, on rank 0, its plain arm,
    group rooflines and end-to-end rate."""
    import numpy as np
    import torch
    from paper_2505_01059_gb300 import workloads as W

    specs = rank_specs(W.batch(count=args.instances, bf16=True), rank)
    handles = [mtp.mtp_create(s) for s in specs]
    b = mtp.mtp_batch_create(handles)
    tiles = mtp.mtp_batch_autotune(b)
    tuned_mode, mode_ms = mtp.mtp_batch_rollout_mode(b)
    if args.rollout_mode != "auto":
        mtp.mtp_batch_set_rollout_mode(b, ROLLOUT_MODES[args.rollout_mode])
    mode = mtp.mtp_batch_rollout_mode(b)[0]
    x0 = torch.tensor(np.concatenate([np.array(s["x0"], np.float32) for s in specs]), device=dev)
    us = torch.empty(b.ustar_offset[-1], device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    steps_per_iter = sum(s["B"] * s["H"] for s in specs)

    def batched():
        mtp.mtp_batch_plan_step(b, x0, 1, us)

    for _ in range(args.warmup):
        batched()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clocks:
        t_wall = time.perf_counter()
        ms = time_steps(batched, args.steps, flush, stream)
        t_wall = time.perf_counter() - t_wall
    if pg:
        pg.barrier()
    total_ms = max_over_ranks(sum(ms), pg, dev)
    res = {
        "specs": specs, "steps_per_iter": steps_per_iter, "tiles": tiles,
        "value": job_rate(world, steps_per_iter * args.steps, total_ms / 1e3),
        "plan_steps_per_s": job_rate(world, len(specs) * args.steps, total_ms / 1e3),
        "ms_per_step": total_ms / args.steps, "clocks": clocks.summary(), "wall_s_timed": t_wall,
        "latency_ms": {"p50": percentile(sorted(ms), 0.5), "p99": percentile(sorted(ms), 0.99),
                       "what": "device time of one batched iteration: every instance's re-plan "
                               "completes at its end"},
        "gpu_launches": mtp.mtp_batch_launches(b, 1) * args.steps,
        "rollout_mode": {"timed": mtp.BATCH_ROLLOUT_NAMES[mode],
                         "autotuner_pick": mtp.BATCH_ROLLOUT_NAMES[tuned_mode],
                         "autotuner_iteration_ms": {mtp.BATCH_ROLLOUT_NAMES[k]: v
                                                    for k, v in enumerate(mode_ms)}},
    }
    if rank != 0 or args.quick:
        mtp.mtp_batch_destroy(b)
        for h in handles:
            mtp.mtp_destroy(h)
        return res

    # group rollouts, each alone, for the roofline
    res["roofline"], res["rollout_groups"] = batch_rollout_roofline(mtp, b, specs, device_sms(dev.index))
    peak, note = fp32_peak(peaks().get("sm_max_mhz", 2070.0), device_sms(dev.index))
    if mode != 0:
        # the iteration's rollouts are the persistent launch: it is the dominant kernel
        p_ms, p_steps = mtp.mtp_batch_persistent_time(b, reps=5)
        covered = [s for s in specs if (s["dyn"] == "pointmass" and s["n"] <= 16) or
                   (s["dyn"] == "chain" and s["n_links"] <= 9)]
        assert sum(s["B"] * s["H"] for s in covered) == p_steps
        fl = sum(flops_per_step(s) * s["B"] * s["H"] for s in covered)
        achieved = fl / (p_ms / 1e3) / 1e12
        res["roofline"] = {
            "bound": "alu", "kernel": "k_rollout_persistent", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": profiled_traffic("rollout_persist.cu", "rollout_persist_batch64.txt",
                                        key="dram_bytes_per_launch_batch256"),
            "flops_per_launch": fl, "duration_us": p_ms * 1e3, "rollout_steps": p_steps,
            "timing": "CUDA events around the persistent rollout launch run alone on its stream "
                      "(5 launches averaged), after the timed region",
            "peak_note": note + " (of measured clock)"}
    flops_iter = sum(flops_per_step(s) * s["B"] * s["H"] for s in specs)
    res["whole_step_fp32"] = {"achieved": flops_iter / (res["ms_per_step"] / 1e3) / 1e12,
                              "peak": peak, "unit": "TFLOP/s",
                              "frac": flops_iter / (res["ms_per_step"] / 1e3) / 1e12 / peak,
                              "note": "rollout flops of all instances over the whole iteration"}

    # end to end through the public batch call from host memory: pinned
    # packed start states in, packed u* out, synchronised, every step
    x0_h = x0.cpu().pin_memory()
    us_h = torch.empty(us.numel(), dtype=torch.float32).pin_memory()
    lat = []
    for k in range(args.steps + 3):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x0.copy_(x0_h, non_blocking=True)
        mtp.mtp_batch_plan_step(b, x0, 1, us)
        us_h.copy_(us, non_blocking=True)
        stream.synchronize()
        if k >= 3:
            lat.append(time.perf_counter() - t0)
    res["e2e"] = {"value": steps_per_iter * len(lat) / sum(lat), "unit": UNIT,
                  "h2d_bytes_per_step": 4 * x0.numel(), "d2h_bytes_per_step": 4 * us.numel(),
                  "plan_steps_per_s": len(specs) * len(lat) / sum(lat),
                  "timing": "host clock around pinned x0 -> device, mtp_batch_plan_step, "
                            "u* -> pinned host, stream synchronise; L2 flushed before each step, "
                            "outside it"}
    mtp.mtp_batch_destroy(b)
    for h in handles:
        mtp.mtp_destroy(h)

    # the plain arm: the same instances in FP32, one mtp_plan_step each in
    # turn on one stream (their own captured graphs)
    plain_specs = rank_specs(W.batch(count=args.instances, bf16=False), rank)
    ph = [mtp.mtp_create(s) for s in plain_specs]
    x0_each = [torch.tensor(s["x0"], dtype=torch.float32, device=dev) for s in plain_specs]
    u_each = [torch.empty(s["n"], device=dev) for s in plain_specs]

    def plain():
        for h, xx, uu in zip(ph, x0_each, u_each):
            mtp.mtp_plan_step(h, xx, 1, uu)

    for _ in range(3):
        plain()
    torch.cuda.synchronize()
    ms_p = time_steps(plain, max(3, min(args.steps, 10)), flush, stream)
    mp = sum(ms_p) / len(ms_p)
    res["plain"] = {"ms_per_step": mp, "value": steps_per_iter / (mp / 1e3),
                    "plan_steps_per_s": len(plain_specs) / (mp / 1e3),
                    "latency_ms": {"p50": percentile(sorted(ms_p), 0.5),
                                   "p99": percentile(sorted(ms_p), 0.99)},
                    "dtype": "f32",
                    "what": "every instance through its own mtp_plan_step (graph replay), one "
                            "after the other on one stream",
                    "gpu_launches_per_step": sum(h.sizes["kernels_per_iteration"] for h in ph)}
    for h in ph:
        mtp.mtp_destroy(h)
    res["batched_over_plain"] = mp / res["ms_per_step"]
    return res


# ----------------------------------------------------------------------------
# serving: the re-plan server against the plain path at a matched p99
# ----------------------------------------------------------------------------

class HostSim:
    """The robots' true motion on the host, FP64: each re-plan's u* drives
    one planner step of the robot's own nominal model (sim-to-sim, as the
    planner models it).  Point masses: v += dt u, p += dt v.  Arms: uniform
    thin rods in a vertical plane, joint torques, semi-implicit Euler, with
    the Lagrangian written in absolute link angles (mass matrix D_jk
    cos(phi_j - phi_k), velocity terms D_jk sin(phi_j - phi_k) w_k^2,
    gravity and torque differences), solved for all robots of one link
    count at once.  Completions are buffered and advanced in batches; a
    robot's state is brought up to date before it submits again.  A robot
    whose motion leaves the range its model is integrated well in (a joint
    faster than ARM_MAX_RATE rad/s, a point mass beyond PM_MAX_POS, or any
    non-finite value) starts a new episode from its initial state; `resets`
    counts those."""

    ARM_MAX_RATE = 50.0
    PM_MAX_POS = 100.0

    def __init__(self, specs, x0s):
        import numpy as np
        self.np = np
        self.specs = specs
        self.x = [np.asarray(x, np.float64).copy() for x in x0s]
        self.x_init = [x.copy() for x in self.x]
        self.resets = 0
        self.pending = {}
        self.groups = {}
        for r, s in enumerate(specs):
            key = ("pm", s["n"]) if s["dyn"] == "pointmass" else ("arm", s["n_links"])
            self.groups.setdefault(key, []).append(r)
        self.model = {}
        for r, s in enumerate(specs):
            if s["dyn"] != "chain":
                continue
            m = np.array(s["mass"], np.float64)
            l = np.array(s["length"], np.float64)
            L = len(m)
            tail = np.concatenate([np.cumsum(m[::-1])[::-1][1:], [0.0]])  # sum of masses beyond j
            D = np.empty((L, L))
            for j in range(L):
                for k in range(L):
                    a, c = min(j, k), max(j, k)
                    D[j, k] = (l[j] * l[j] * (m[j] / 3.0 + tail[j]) if j == k
                               else l[a] * l[c] * (m[c] / 2.0 + tail[c]))
            grav = s.get("gravity", 9.81) * l * (m / 2.0 + tail)
            self.model[r] = (D, grav)

    def defer(self, robots, U):
        for r, u in zip(robots, U):
            self.pending[int(r)] = u

    def state(self, r: int):
        if r in self.pending:
            self.flush()
        return self.x[r]

    def flush(self):
        np = self.np
        if not self.pending:
            return
        by_group = collections.defaultdict(list)
        for r in self.pending:
            s = self.specs[r]
            key = ("pm", s["n"]) if s["dyn"] == "pointmass" else ("arm", s["n_links"])
            by_group[key].append(r)
        for (kind, dim), rs in by_group.items():
            X = np.stack([self.x[r] for r in rs])
            U = np.stack([np.asarray(self.pending[r][:dim], np.float64) for r in rs])
            dt = np.array([self.specs[r]["dt"] for r in rs])[:, None]
            if kind == "pm":
                v = X[:, dim:] + dt * U
                X = np.concatenate([X[:, :dim] + dt * v, v], axis=1)
            else:
                q, qd = X[:, :dim], X[:, dim:]
                phi, w = np.cumsum(q, axis=1), np.cumsum(qd, axis=1)
                D = np.stack([self.model[r][0] for r in rs])
                grav = np.stack([self.model[r][1] for r in rs])
                dphi = phi[:, :, None] - phi[:, None, :]
                A = D * np.cos(dphi)
                vel = np.einsum("bjk,bk->bj", D * np.sin(dphi), w * w)
                tau_next = np.concatenate([U[:, 1:], np.zeros((len(rs), 1))], axis=1)
                rhs = U - tau_next - vel - grav * np.cos(phi)
                wd = np.linalg.solve(A, rhs[..., None])[..., 0]
                w = w + dt * wd
                phi = phi + dt * w
                q = np.diff(phi, axis=1, prepend=0.0)
                qd = np.diff(w, axis=1, prepend=0.0)
                X = np.concatenate([q, qd], axis=1)
            if kind == "pm":
                bad = np.abs(X[:, :dim]).max(axis=1) > self.PM_MAX_POS
            else:
                bad = np.abs(X[:, dim:]).max(axis=1) > self.ARM_MAX_RATE
            bad |= ~np.isfinite(X).all(axis=1)
            for i, r in enumerate(rs):
                if bad[i]:
                    self.x[r] = self.x_init[r].copy()
                    self.resets += 1
                else:
                    self.x[r] = X[i]
        self.pending.clear()


def served_open_loop(mtp, srv, ids, sim, steps_of, rate_hz, seconds, warmup, rng):
    """Poisson arrivals at rate_hz per robot for warmup + seconds; each
    request submitted with the robot's simulated state.  Latency runs from
    the scheduled arrival to the poll that sees the result.  Returns the
    window's completions, rollout steps, latencies and refusals."""
    import numpy as np
    R = len(ids)
    t0 = time.perf_counter()
    t_end = t0 + warmup + seconds
    w0 = t0 + warmup
    next_t = t0 + rng.exponential(1.0 / rate_hz, size=R)
    out_t, out_r, out_a = [], [], []   # outstanding tickets, robots, arrival times
    lat, done, steps, refused = [], 0, 0.0, 0
    waiting = collections.deque()      # (robot, arrival) not yet accepted
    while True:
        now = time.perf_counter()
        if now >= t_end and not out_t and not waiting:
            break
        if now < t_end:
            due = np.nonzero(next_t <= now)[0]
            if len(due):
                for r in due[np.argsort(next_t[due])]:
                    waiting.append((int(r), float(next_t[r])))
                next_t[due] += rng.exponential(1.0 / rate_hz, size=len(due))
        if waiting:
            rs = [r for r, _ in waiting]
            x0 = np.concatenate([sim.state(r) for r in rs]).astype(np.float32)
            try:
                ts = mtp.mtp_submit_many(srv, ids[rs], x0)
                k, skip = len(ts), 0
            except mtp.MtpError as e:   # a robot's queue is full: that arrival is refused
                if e.status != 4:
                    raise
                ts, k, skip = e.tickets, len(e.tickets), 1
            for j in range(k):
                r, a = waiting.popleft()
                out_t.append(int(ts[j]))
                out_r.append(r)
                out_a.append(a)
            if skip:
                r, a = waiting.popleft()
                refused += a >= w0
        if out_t:
            status, u, ready = mtp.mtp_poll_many(srv, np.array(out_t, np.uint64), 32, 0.0)
            if ready:
                t_obs = time.perf_counter()
                keep_t, keep_r, keep_a = [], [], []
                fin_r, fin_u = [], []
                for j, st in enumerate(status):
                    if st == 0:
                        fin_r.append(out_r[j])
                        fin_u.append(u[j])
                        if out_a[j] >= w0:
                            lat.append(t_obs - out_a[j])
                            done += 1
                            steps += steps_of[out_r[j]]
                    elif st in (5, 6):
                        keep_t.append(out_t[j])
                        keep_r.append(out_r[j])
                        keep_a.append(out_a[j])
                    else:
                        raise RuntimeError(f"serving poll failed: status {st}")
                sim.defer(fin_r, fin_u)
                sim.flush()
                out_t, out_r, out_a = keep_t, keep_r, keep_a
                continue
        time.sleep(50e-6)
    return done, steps, lat, refused


def plain_open_loop(mtp, handles, sim, steps_of, rate_hz, seconds, warmup, rng, drain_cap=3.0):
    """The same Poisson request stream served by the plain path: one request
    at a time, first come first served, through mtp_plan_step_host +
    mtp_shift on the robot's own handle."""
    import numpy as np
    R = len(handles)
    t0 = time.perf_counter()
    t_end = t0 + warmup + seconds
    w0 = t0 + warmup
    next_t = t0 + rng.exponential(1.0 / rate_hz, size=R)
    queue = collections.deque()
    u = np.empty(32, np.float32)
    lat, done, steps, unfinished = [], 0, 0.0, 0
    while True:
        now = time.perf_counter()
        if now >= t_end:
            if not queue:
                break
            if now >= t_end + drain_cap:   # overloaded: what is left counts as unserved
                unfinished = sum(1 for _, a in queue if a >= w0)
                break
        else:
            due = np.nonzero(next_t <= now)[0]
            if len(due):
                for r in due[np.argsort(next_t[due])]:
                    queue.append((int(r), float(next_t[r])))
                next_t[due] += rng.exponential(1.0 / rate_hz, size=len(due))
        if queue:
            r, a = queue.popleft()
            mtp.mtp_plan_step_host(handles[r], sim.state(r).astype(np.float32), 1, u)
            mtp.mtp_shift(handles[r], 1)
            t_obs = time.perf_counter()
            sim.defer([r], [u.copy()])
            if len(sim.pending) >= 64:
                sim.flush()
            if a >= w0:
                lat.append(t_obs - a)
                done += 1
                steps += steps_of[r]
            continue
        sim.flush()
        time.sleep(20e-6)
    return done, steps, lat, unfinished


def serve_point(done, steps, lat, seconds, offered, extra):
    lat_ms = sorted(1e3 * v for v in lat)
    unserved = extra.get("unfinished", 0) + extra.get("refused", 0)
    p99 = percentile(lat_ms, 0.99)
    if unserved > 0.01 * max(done + unserved, 1):
        p99 = float("inf")  # more than 1 % of the window's requests were never served
    return dict({"offered_requests_per_s": offered, "plan_steps_per_s": done / seconds,
                 "rollout_steps_per_s": steps / seconds, "p50_ms": percentile(lat_ms, 0.5),
                 "p99_ms": p99, "completed": done}, **extra)


def best_at_p99(points, target_ms):
    ok = [p for p in points if p["p99_ms"] is not None and p["p99_ms"] <= target_ms]
    return max(ok, key=lambda p: p["plan_steps_per_s"]) if ok else None


def run_serving(args, mtp, dev) -> dict:
    """The 1024-robot fleet (Poisson arrivals per robot) through the re-plan
    server at several offered rates, and the same request stream through the
    plain path; plan-steps/s compared at a matched p99 latency."""
    import numpy as np
    import torch
    from paper_2505_01059_gb300 import workloads as W

    specs = W.robots(count=args.robots)
    R = len(specs)
    rng = np.random.default_rng(4)
    x0s = [np.asarray(s["x0"], np.float64) + rng.uniform(-0.1, 0.1, size=s["d"]) for s in specs]
    steps_of = np.array([s["B"] * s["H"] for s in specs], dtype=np.float64)
    out = {"workload": f"{R} robots (2-D point masses and 3..9-link arms, H 64..128, B 1024..4096), "
                       f"each a Poisson stream of re-plans; 1 iteration + shift per request; "
                       f"host simulator advances every robot's own model in FP64",
           "latency": "scheduled arrival -> result seen by the client, host wall time"}

    # served
    srv = mtp.mtp_server_create(max_batch=args.max_batch, iters_per_request=1, shift_after=1,
                                max_queue=8, max_robots=R)
    ids = np.array([mtp.mtp_server_register(srv, s) for s in specs], dtype=np.int32)
    sim = HostSim(specs, x0s)
    served = []
    # the client's own pauses (Python's cyclic garbage collector) are kept
    # out of the latency windows; the first pass warms every robot
    gc.collect()
    gc.disable()
    # the clock sampler (nvidia-smi) starts before the warm-up pass: its
    # start-up holds the driver for a while
    with ClockSampler(dev.index) as clocks:
        served_open_loop(mtp, srv, ids, sim, steps_of, 50.0, 1.0, 0.0, rng)
        for rate in args.serve_rates:
            done, steps, lat, refused = served_open_loop(mtp, srv, ids, sim, steps_of, rate,
                                                         args.serve_seconds, args.serve_warmup, rng)
            served.append(serve_point(done, steps, lat, args.serve_seconds, R * rate,
                                      {"rate_hz_per_robot": rate, "refused": refused}))
    stats = mtp.mtp_server_get_stats(srv)
    srv.close()
    out["served_episode_resets"] = sim.resets
    out["served"] = served
    out["served_clocks"] = clocks.summary()
    out["server_cycles"] = stats["cycles"]
    out["mean_robots_per_cycle"] = stats["planned"] / max(stats["cycles"], 1)

    # plain: each robot's own handle, one request at a time
    handles = [mtp.mtp_create(dict(s)) for s in specs]
    sim = HostSim(specs, x0s)
    u = np.empty(32, np.float32)
    # capture every graph a handle replays: the first step makes its
    # candidates in full, and a pipelined handle then alternates between its
    # two candidate buffers, each with a graph of its own
    for r, h in enumerate(handles):
        for _ in range(3):
            mtp.mtp_plan_step_host(h, sim.state(r).astype(np.float32), 1, u)
            mtp.mtp_shift(h, 1)
    torch.cuda.synchronize()
    probe = rng.integers(0, R, size=256)
    t0 = time.perf_counter()
    for r in probe:
        mtp.mtp_plan_step_host(handles[r], sim.state(r).astype(np.float32), 1, u)
        mtp.mtp_shift(handles[r], 1)
    service = (time.perf_counter() - t0) / len(probe)
    capacity = 1.0 / service
    plain = []
    gc.collect()
    for frac in args.plain_loads:
        rate = frac * capacity / R
        done, steps, lat, unfinished = plain_open_loop(mtp, handles, sim, steps_of, rate,
                                                       args.serve_seconds, args.serve_warmup, rng)
        plain.append(serve_point(done, steps, lat, args.serve_seconds, R * rate,
                                 {"load_of_capacity": frac, "unfinished": unfinished}))
    gc.enable()
    for h in handles:
        mtp.mtp_destroy(h)
    out["plain"] = plain
    out["plain_episode_resets"] = sim.resets
    out["plain_service_ms"] = service * 1e3
    out["plain_capacity_requests_per_s"] = capacity

    # matched p99: the served p99 at the nominal 50 Hz fleet, and the 20 ms
    # control period of a 50 Hz re-plan loop
    nominal = next((p for p in served if p["rate_hz_per_robot"] == 50.0), served[0])
    comps = {}
    for name, target in (("served_p99_at_50hz", nominal["p99_ms"]), ("control_period_20ms", 20.0)):
        s_best, p_best = best_at_p99(served, target), best_at_p99(plain, target)
        comps[name] = {
            "p99_target_ms": target,
            "served_plan_steps_per_s": s_best["plan_steps_per_s"] if s_best else None,
            "plain_plan_steps_per_s": p_best["plan_steps_per_s"] if p_best else None,
            "served_over_plain": (s_best["plan_steps_per_s"] / p_best["plan_steps_per_s"]
                                  if s_best and p_best else None)}
    out["matched_p99"] = comps
    return out


# ----------------------------------------------------------------------------
# one instance per launch sequence: the 7-link arm and the 16-link legged chain
# ----------------------------------------------------------------------------

def run_single(args, mtp, dev, spec, name, steps, pg=None, world=1, rank=0, flush=None) -> dict:
    """mtp_plan_step (graph replay) of one instance: rollout-steps/s, the
    per-stage device times (direct launches with events between them) and
    the rollout kernel against the FP32 peak."""
    import numpy as np
    import torch
    spec = dict(spec, seed=spec["seed"] + 7919 * rank)
    h = mtp.mtp_create(spec)
    s = h.sizes
    x0 = torch.tensor(spec["x0"], dtype=torch.float32, device=dev)
    ustar = torch.empty(s["n"], dtype=torch.float32, device=dev)
    if flush is None:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        mtp.mtp_plan_step(h, x0, 1, ustar)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clocks:
        t_wall = time.perf_counter()
        ms = time_steps(lambda: mtp.mtp_plan_step(h, x0, 1, ustar), steps, flush, stream)
        t_wall = time.perf_counter() - t_wall
    if pg:
        pg.barrier()
    total_ms = max_over_ranks(sum(ms), pg, dev)
    steps_per_iter = s["B"] * s["H"]
    res = {"workload": workload_label(spec, name),
           "value": job_rate(world, steps_per_iter * steps, total_ms / 1e3),
           "plan_steps_per_s": job_rate(world, steps, total_ms / 1e3),
           "ms_per_step": total_ms / steps, "clocks": clocks.summary(), "wall_s_timed": t_wall,
           "gpu_launches": s["kernels_per_iteration"] * steps,
           "pipelined": {0: "no", 1: "graph rows", 2: "graph rows and draws"}[s["pipelined"]]}
    # stage pass: the same kernels launched directly, events between them
    hp = mtp.mtp_create(dict(spec, flags=spec.get("flags", 0) | mtp.FLAG_NO_GRAPH))
    for _ in range(3):
        mtp.mtp_plan_step(hp, x0, 1, ustar)
    mtp.mtp_set_profiling(hp, True)
    n_stage = min(steps, 200)
    for _ in range(n_stage):
        flush.zero_()
        mtp.mtp_plan_step(hp, x0, 1, ustar)
    torch.cuda.synchronize()
    stage5, n_it = mtp.mtp_stage_times5(hp)
    mtp.mtp_destroy(hp)
    stage_ms = [v / max(n_it, 1) for v in stage5[:4]]
    res["stage_ms_per_step"] = dict(zip(("generate", "rollout", "select", "update"), stage_ms))
    res["prepare_overlapped_ms_per_step"] = stage5[4] / max(n_it, 1)
    peak, note = fp32_peak(peaks().get("sm_max_mhz", 2070.0), device_sms(dev.index))
    fl = flops_per_step(spec) * steps_per_iter
    achieved = fl / (stage_ms[1] / 1e3) / 1e12
    kernel_file = KERNEL_FILE[spec["dyn"]]
    summary = {"chain": "rollout_chain7_arm_B4096.txt", "pointmass": "rollout_pointmass2_B512.txt",
               "legged": "rollout_legged16_B4096.txt"}[spec["dyn"]]
    res["roofline"] = {"bound": "alu", "kernel": ROLLOUT_KERNEL[spec["dyn"]], "achieved": achieved,
                       "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                       "traffic": profiled_traffic(kernel_file, summary),
                       "flops_per_launch": fl, "duration_us": stage_ms[1] * 1e3,
                       "timing": f"CUDA events around the rollout launch on its stream, {n_it} "
                                 f"direct-launch iterations, L2 flushed between steps",
                       "peak_note": note + " (of measured clock)"}
    # end to end through the host-pointer call: pinned x0 in, u* out
    x0_h = torch.tensor(spec["x0"], dtype=torch.float32).pin_memory()
    u_h = torch.empty(s["n"], dtype=torch.float32).pin_memory()
    lat = []
    for k in range(min(steps, 500) + 3):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mtp.mtp_plan_step_host(h, x0_h, 1, u_h)
        if k >= 3:
            lat.append(time.perf_counter() - t0)
    lat.sort()
    res["e2e"] = {"value": steps_per_iter * len(lat) / sum(lat), "unit": UNIT,
                  "h2d_bytes_per_step": 4 * s["d"], "d2h_bytes_per_step": 4 * s["n"],
                  "p50_ms": 1e3 * lat[len(lat) // 2], "p99_ms": 1e3 * percentile(lat, 0.99)}
    mtp.mtp_destroy(h)
    return res


# ----------------------------------------------------------------------------
# entry points
# ----------------------------------------------------------------------------

def base_line(args, world, value, ms_per_step, config, dtype="f32") -> dict:
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": config}


def run_headline(args):
    world, rank, local = dist_init()
    dev, pg, mtp = setup_gpu(local, world)
    res = run_batch_arms(args, mtp, dev, pg, world, rank)
    extras = {}
    if rank == 0 and not args.quick:
        import torch
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        extras["serving"] = run_serving(args, mtp, dev)
        for name in ("arm7", "legged16"):
            extras[name] = run_single(args, mtp, dev, workload(name), name, args.single_steps,
                                      flush=flush)
    if rank == 0:
        cfg = {"workload": BATCH_LABEL, "instances": len(res["specs"]),
               "rollout_steps_per_iteration": res["steps_per_iter"],
               "parallelism": f"replicas{world}", "iters_per_step": 1,
               "l2": "flushed between steps (256 MB write); the candidate tensors exceed L2",
               "timed_mode": "CUDA graph replay of mtp_batch_plan_step"}
        line = base_line(args, world, res["value"], res["ms_per_step"], cfg)
        line.update({
            "plan_steps_per_s": res["plan_steps_per_s"],
            "replan_latency_ms": res["latency_ms"],
            "plain": res.get("plain"),
            "batched_over_plain": res.get("batched_over_plain"),
            "serving": extras.get("serving"),
            "roofline": res.get("roofline"),
            "rollout_groups": res.get("rollout_groups"),
            "whole_step_fp32": res.get("whole_step_fp32"),
            "tiles": res["tiles"],
            "rollout_mode": res["rollout_mode"],
            "arm7": extras.get("arm7"),
            "legged16": extras.get("legged16"),
            "e2e": res.get("e2e"),
            "gpu_launches": res["gpu_launches"],
            "clocks": res["clocks"],
            "wall_s_timed": res["wall_s_timed"],
        })
        if world == 1 and not args.no_cpu_baseline:
            cpu = host_cpu()
            allc = cpu_oracle_batch(res["specs"], args.cpu_seconds, cpu["cores"])
            one = cpu_oracle_batch(res["specs"][:32], args.cpu_seconds / 3, 1)
            line["cpu_baseline"] = {
                "value": allc["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle",
                "cpu_model": cpu["model"],
                "sample": f"one Alg. 2 iteration of all {allc['instances']} instances on their "
                          f"first {allc['rows_per_instance']} candidates in {allc['seconds']:.1f} s "
                          f"(FP64 C oracle, rollouts on {cpu['cores']} threads)",
                "one_thread": {"value": one["value"], "unit": UNIT, "cores": 1,
                               "sample": f"32 instances on their first {one['rows_per_instance']} "
                                         f"candidates in {one['seconds']:.1f} s"}}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def run_serve_only(args):
    world, rank, local = dist_init()
    dev, pg, mtp = setup_gpu(local, world)
    if rank == 0:
        out = run_serving(args, mtp, dev)
        nominal = next((p for p in out["served"] if p["rate_hz_per_robot"] == 50.0), out["served"][0])
        line = base_line(args, world, nominal["rollout_steps_per_s"], 1e3 / max(nominal["plan_steps_per_s"], 1e-9),
                         {"workload": out["workload"], "step": "one completed re-plan"})
        line.update({"serving": out, "plan_steps_per_s": nominal["plan_steps_per_s"],
                     "clocks": out["served_clocks"],
                     "e2e": {"value": nominal["rollout_steps_per_s"], "unit": UNIT,
                             "h2d_bytes_per_step": 4 * 9, "d2h_bytes_per_step": 4 * 4,
                             "note": "the served path is end to end by construction"}})
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def run_single_only(args, name):
    world, rank, local = dist_init()
    dev, pg, mtp = setup_gpu(local, world)
    res = run_single(args, mtp, dev, workload(name, args.candidates), name, args.steps, pg, world,
                     rank)
    if rank == 0:
        line = base_line(args, world, res["value"], res["ms_per_step"],
                         {"workload": res["workload"], "parallelism": f"replicas{world}",
                          "iters_per_step": 1, "l2": "flushed between steps (256 MB write)",
                          "timed_mode": "CUDA graph replay of mtp_plan_step"})
        line.update({k: v for k, v in res.items() if k not in ("value", "ms_per_step", "workload")})
        if world == 1 and not args.no_cpu_baseline:
            cpu = host_cpu()
            c = cpu_oracle_single(workload(name, args.candidates), args.cpu_seconds, cpu["cores"])
            line["cpu_baseline"] = {"value": c["value"], "unit": UNIT, "cores": cpu["cores"],
                                    "kind": "oracle", "cpu_model": cpu["model"],
                                    "sample": f"one Alg. 2 iteration on {c['rows']} candidates in "
                                              f"{c['seconds']:.1f} s (FP64 C oracle)"}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def run_sweep(args):
    """The M, N ablation of the paper's Navigation study (Appendix, sweep of
    M and N with full tensor sampling, beta = 1, B = 256, 4 seeds) on the
    synthetic 2-D point mass with circular obstacles: for every (M, N) and
    interpolation, the best candidate cost after 10 planner iterations and
    the cost entropy of the last selection (Sec. 4.1), mean over 4 seeds."""
    import numpy as np
    import torch
    from paper_2505_01059_gb300 import workloads as W
    world, rank, local = dist_init()
    dev, pg, mtp = setup_gpu(local, world)
    Ms, Ns, seeds, iters = [2, 3, 4, 6, 8, 12, 16], [4, 8, 16, 32, 64], [11, 12, 13, 14], 10
    grid = {}
    t0 = time.perf_counter()
    for interp in ("bspline", "akima", "linear"):
        for M in Ms:
            for N in Ns:
                best, ent = [], []
                for seed in seeds:
                    spec = W.pointmass(seed=seed, M=M, N=N, B=256, beta=1.0, interp=interp,
                                       degree=min(3, M - 1), E=16,
                                       flags=mtp.FLAG_COST_ENTROPY)
                    h = mtp.mtp_create(spec)
                    x0 = torch.tensor(spec["x0"], dtype=torch.float32, device=dev)
                    u = torch.empty(spec["n"], device=dev)
                    mtp.mtp_plan_step(h, x0, iters, u)
                    buf = mtp.mtp_get_buffers(h)
                    cost = torch.as_tensor(buf["cost"], device=dev)
                    best.append(float(cost.min().item()))
                    ent.append(mtp.mtp_cost_entropy(h))
                    mtp.mtp_destroy(h)
                grid[f"{interp} M={M} N={N}"] = {"best_cost": float(np.mean(best)),
                                                 "best_cost_std": float(np.std(best)),
                                                 "entropy": float(np.mean(ent))}
    line = {"metric": "best candidate cost after 10 iterations (mean over 4 seeds)",
            "unit": "cost", "higher_is_better": False, "n_gpus": 1,
            "config": {"workload": "2-D point mass, 5 circular obstacles, beta 1 (tensor samples "
                                   "only), B 256, E 16, H 64, lambda 0.1", "M": Ms, "N": Ns,
                       "seeds": seeds, "iterations": iters},
            "grid": grid, "wall_s": time.perf_counter() - t0}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "serve", "arm7", "pointmass2", "legged16", "sweep"])
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--candidates", type=int, default=None,
                    help="arm7 / pointmass2 / legged16: candidates B instead of the workload's own")
    ap.add_argument("--robots", type=int, default=1024)
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[25.0, 50.0, 100.0, 125.0],
                    help="served: Poisson re-plan rates per robot (Hz)")
    ap.add_argument("--plain-loads", type=float, nargs="+", default=[0.3, 0.5, 0.7, 0.85],
                    help="plain: offered load as a fraction of its measured capacity")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-warmup", type=float, default=0.5)
    ap.add_argument("--single-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--reference-seconds", type=float, default=90.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="batched timed region only")
    ap.add_argument("--rollout-mode", default="auto", choices=["auto"] + list(ROLLOUT_MODES),
                    help="batched rollouts: the autotuner's pick, or one mode forced")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_headline(args)
    elif args.workload == "serve":
        run_serve_only(args)
    elif args.workload == "sweep":
        run_sweep(args)
    else:
        run_single_only(args, args.workload)


if __name__ == "__main__":
    main()

"""The N>1 path on CPU: two gloo ranks each plan their own instances
(replicas, no collective on the data path); the timing reduction takes the
slowest rank and the job rate counts the units of all ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2505_01059_gb300 import workloads as W
    specs = bench.rank_specs([W.pointmass(B=64, E=8, H=16), W.chain(links=3, B=32, E=4, H=8)],
                             rank)
    costs = []
    for spec in specs:
        mu, sigma = W.initial_distribution(spec)
        costs.append(oracle.plan_iteration(spec, 0, np.array(spec["x0"]), mu, sigma)["cost"])
    my_time = 1.0 + rank  # a stand-in per-rank time: rank 1 is the slowest
    t_max = bench.max_over_ranks(my_time, dist, torch.device("cpu"))
    rate = bench.job_rate(world, sum(s["B"] * s["H"] for s in specs), t_max)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), seed=specs[0]["seed"],
             cost=np.concatenate(costs), t_max=t_max, rate=rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_plan_independent_replicas(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    assert int(r0["seed"]) != int(r1["seed"])              # each rank its own instance
    assert not np.array_equal(r0["cost"], r1["cost"])      # independent work
    assert float(r0["t_max"]) == float(r1["t_max"]) == 2.0  # slowest rank's time on both
    assert float(r0["rate"]) == pytest.approx(2 * (64 * 16 + 32 * 8) / 2.0)

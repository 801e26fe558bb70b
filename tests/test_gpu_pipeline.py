"""Pipelined plan steps: a handle that prepares each next iteration's graph
rows and local draws during the rollout gives bitwise the results of one
that makes every iteration's candidates in full (MTP_FLAG_NO_PIPELINE),
across calls, shifts, checkpoint restores (which move the iteration counter
and so retire the prepared draws), host-pointer steps and batch runs, in
graph replay and eager launches."""
import numpy as np
import pytest

from paper_2505_01059_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mtp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_01059_gb300 import _build, mtp as m
    _build.build_library()
    m.load_library()
    torch.cuda.set_device(0)
    return m


SPECS = [
    W.chain(),                                             # 7-link arm, B 4096: graph rows only
    W.chain(B=2048),                                       # 7-link arm, Akima
    W.chain(links=5, B=2048, H=64, interp="linear"),       # straight lines
    W.pointmass(),                                         # C1: B 512, cubic B-spline
    W.pointmass(B=256, E=8, beta=1.0),                     # graph rows only (no local rows)
    W.pointmass(B=256, E=8, beta=0.0),                     # local rows only (no graph)
    W.chain(links=4, B=512, H=40, M=16, N=80, E=16),       # graph above 16 KB: Z in the
                                                           # preparing block's shared memory
    W.pointmass(k=5, B=333, H=37, E=9),                    # H n not a multiple of 4
]


def _run(mtp, spec, flags):
    h = mtp.mtp_create(dict(spec, flags=spec.get("flags", 0) | flags))
    s = h.sizes
    x0 = torch.tensor(spec["x0"], dtype=torch.float32, device=DEV)
    u = torch.empty(s["n"], device=DEV)
    outs = []

    def snap():
        torch.cuda.synchronize()
        buf = mtp.mtp_get_buffers(h)
        mu, sg, it = mtp.mtp_get_state(h)
        U = torch.as_tensor(buf["U"], device=DEV).cpu().numpy().copy()
        cost = torch.as_tensor(buf["cost"], device=DEV).cpu().numpy().copy()
        outs.append((mu, sg, it, u.cpu().numpy().copy(), U, cost))

    mtp.mtp_plan_step(h, x0, 1, u)
    snap()
    mtp.mtp_plan_step(h, x0, 1, u)
    mtp.mtp_shift(h, 1)
    mtp.mtp_plan_step(h, x0, 3, u)
    snap()
    mu, sg, _ = mtp.mtp_get_state(h)
    mtp.mtp_set_state(h, mu, sg, 11)  # the prepared draws are for iteration 5, not 11
    mtp.mtp_plan_step(h, x0, 2, u)
    snap()
    uh = np.empty(s["n"], np.float32)
    mtp.mtp_plan_step_host(h, np.asarray(spec["x0"], np.float32), 1, uh)
    u.copy_(torch.from_numpy(uh))
    snap()
    mtp.mtp_set_state(h, mu, sg, 14)  # the counter moved to the prepared iteration itself
    mtp.mtp_plan_step(h, x0, 1, u)
    snap()
    mtp.mtp_destroy(h)
    return s, outs


@pytest.mark.parametrize("graph_flags", [0, 0x2])
@pytest.mark.parametrize("spec", SPECS)
def test_pipelined_matches_unpipelined(mtp, spec, graph_flags):
    s_p, a = _run(mtp, spec, graph_flags)
    s_n, b = _run(mtp, spec, graph_flags | mtp.FLAG_NO_PIPELINE)
    # graph rows only: the 4096-candidate arm (24 idle SMs) and a problem without local rows
    only_graph = spec["B"] == 4096 or s_p["L"] == 0
    assert s_p["pipelined"] == (1 if only_graph else 2) and s_n["pipelined"] == 0
    assert s_p["kernels_per_iteration"] == 5
    for k, (x, y) in enumerate(zip(a, b)):
        for name, vx, vy in zip(("mu", "sigma", "iter", "ustar", "U", "cost"), x, y):
            assert np.array_equal(vx, vy), (k, name)


def test_legged_tiny_and_bf16_problems_are_not_pipelined(mtp):
    # the legged rollout fills the GPU; B 1 has no draws or graph rows; the
    # third one's rollout leaves no SM idle; the BF16 basis contraction runs
    # on the tensor cores in a launch of its own, which the preparation does
    # not make
    for spec in (W.legged(links=4, B=256, H=32, M=6, N=16, E=16), W.pointmass(B=1, E=1),
                 W.pointmass(B=8192, H=16, E=8), W.pointmass(k=3, B=600, flags=0x4)):
        h = mtp.mtp_create(spec)
        assert h.sizes["pipelined"] == 0, spec["B"]
        mtp.mtp_destroy(h)


def test_device_bytes_count_the_second_buffer(mtp):
    for spec in (W.chain(), W.chain(B=2048)):
        b_p = mtp.mtp_problem_device_bytes(spec)
        b_n = mtp.mtp_problem_device_bytes(dict(spec, flags=mtp.FLAG_NO_PIPELINE))
        assert b_p - b_n == spec["B"] * spec["H"] * spec["n"] * 4


@pytest.mark.parametrize("graph_flags", [0, 0x2])
@pytest.mark.parametrize("B", [4096, 2048])
def test_profiled_pipeline_reports_the_overlapped_preparation(mtp, graph_flags, B):
    spec = dict(W.chain(B=B), flags=graph_flags)
    h = mtp.mtp_create(spec)
    x0 = torch.tensor(spec["x0"], dtype=torch.float32, device=DEV)
    u = torch.empty(h.sizes["n"], device=DEV)
    mtp.mtp_set_profiling(h, True)
    mtp.mtp_plan_step(h, x0, 3, u)
    mtp.mtp_plan_step(h, x0, 1, u)
    ms, n_it = mtp.mtp_stage_times5(h)
    assert n_it == 4 and all(v > 0 for v in ms)
    mtp.mtp_destroy(h)


def test_batch_run_between_pipelined_steps(mtp):
    """A handle planned alone (pipelined), then in a batch, then alone again
    gets what a handle that never pipelines gets over the same sequence."""
    spec = W.chain(links=7, B=1024, E=32)
    other = W.pointmass(B=512)
    rng = np.random.default_rng(2)
    x0 = rng.uniform(-0.2, 0.2, size=spec["d"]).astype(np.float32)
    x1 = rng.uniform(-0.2, 0.2, size=other["d"]).astype(np.float32)
    res = []
    for flags in (0, mtp.FLAG_NO_PIPELINE):
        h = mtp.mtp_create(dict(spec, flags=flags))
        g = mtp.mtp_create(other)
        u = torch.empty(spec["n"], device=DEV)
        mtp.mtp_plan_step(h, torch.tensor(x0, device=DEV), 2, u)
        b = mtp.mtp_batch_create([h, g])
        us = torch.empty(b.ustar_offset[-1], device=DEV)
        mtp.mtp_batch_plan_step(b, torch.tensor(np.concatenate([x0, x1]), device=DEV), 2, us)
        mtp.mtp_batch_destroy(b)
        mtp.mtp_plan_step(h, torch.tensor(x0, device=DEV), 2, u)
        torch.cuda.synchronize()
        res.append((*mtp.mtp_get_state(h), u.cpu().numpy(), us.cpu().numpy()))
        mtp.mtp_destroy(h)
        mtp.mtp_destroy(g)
    for x, y in zip(res[0], res[1]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("flags,iters,profile", [
    (0, 1, False),       # one graph launch: staged start state, u* written to pinned memory
    (0, 3, False),
    (0, 70, False),      # more than 64 iterations: the copies around chunked graphs
    (0x2, 2, False),     # eager launches
    (0, 2, True),        # profiling: the copies around the profiled graphs
])
def test_host_step_paths_match_device_step(mtp, flags, iters, profile):
    """mtp_plan_step_host gives what mtp_plan_step gives a twin handle, call
    after call, whichever route it takes."""
    spec = dict(W.chain(links=3, B=1024, H=32, E=16), flags=flags)
    h, t = mtp.mtp_create(spec), mtp.mtp_create(spec)
    if profile:
        mtp.mtp_set_profiling(h, True)
    rng = np.random.default_rng(iters)
    u_dev = torch.empty(spec["n"], device=DEV)
    for call in range(3):
        x0 = (np.asarray(spec["x0"]) + rng.uniform(-0.1, 0.1, size=spec["d"])).astype(np.float32)
        u_host = np.full(spec["n"], np.nan, np.float32)
        mtp.mtp_plan_step_host(h, x0, iters, u_host)
        mtp.mtp_plan_step(t, torch.tensor(x0, device=DEV), iters, u_dev)
        torch.cuda.synchronize()
        assert np.array_equal(u_host, u_dev.cpu().numpy()), call
        for a, b in zip(mtp.mtp_get_state(h), mtp.mtp_get_state(t)):
            assert np.array_equal(a, b), call
    mtp.mtp_destroy(h)
    mtp.mtp_destroy(t)

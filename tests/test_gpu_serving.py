"""The re-plan server: every served u* is bitwise what the robot's own
handle gives alone (mtp_plan_step then mtp_shift, request by request);
poll reports NOT_READY / TIMEOUT while a request is in flight; admission
refuses robots over the memory budget or the robot limit and submits over
the queue limit; bad tickets and robots are errors."""
import numpy as np
import pytest

from paper_2505_01059_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
OK, ADMISSION, TIMEOUT, NOT_READY = 0, 4, 5, 6


@pytest.fixture(scope="module")
def mtp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_01059_gb300 import _build, mtp as m
    _build.build_library()
    m.load_library()
    torch.cuda.set_device(0)
    return m


def _fleet():
    specs = [s for s in W.robots(seed=21, count=6)]
    for s in specs:
        s["B"] = min(s["B"], 1024)
    specs.append(W.legged(links=4, B=256, H=32, M=6, N=16, E=16))
    return specs


def _x0(spec, rng):
    base = np.asarray(spec["x0"], dtype=np.float64)
    if spec["dyn"] != "legged":
        base = base + rng.uniform(-0.2, 0.2, size=spec["d"])
    return base.astype(np.float32)


@pytest.mark.parametrize("max_batch,iters,shift", [(3, 2, 1), (8, 1, 0)])
def test_served_results_match_each_robot_alone(mtp, max_batch, iters, shift):
    specs = _fleet()
    srv = mtp.mtp_server_create(max_batch=max_batch, iters_per_request=iters, shift_after=shift,
                                max_queue=4, max_robots=16)
    ids = [mtp.mtp_server_register(srv, s) for s in specs]
    assert ids == list(range(len(specs)))
    twins = [mtp.mtp_create(s) for s in specs]
    rng = np.random.default_rng(max_batch)
    rounds = 4
    # two requests per robot queued at once, in two waves: FIFO order per robot
    # is what makes the twin's sequential replay comparable
    for wave in range(rounds // 2):
        x0s = [[_x0(s, rng) for _ in range(2)] for s in specs]
        tickets = [[mtp.mtp_submit(srv, r, x0s[r][j]) for j in range(2)] for r in range(len(specs))]
        for r, s in enumerate(specs):
            for j in range(2):
                got = np.empty(s["n"], dtype=np.float32)
                assert mtp.mtp_poll(srv, tickets[r][j], got, timeout_s=30.0) == OK
                want = torch.empty(s["n"], device=DEV)
                mtp.mtp_plan_step(twins[r], torch.tensor(x0s[r][j], device=DEV), iters, want)
                if shift:
                    mtp.mtp_shift(twins[r], shift)
                assert np.array_equal(got, want.cpu().numpy()), (wave, r, j)
    st = mtp.mtp_server_get_stats(srv)
    n_req = rounds * len(specs)
    assert st["submitted"] == n_req and st["completed"] == n_req
    assert st["planned"] == n_req and 1 <= st["cycles"] <= n_req
    assert st["queued"] == 0 and st["in_flight"] == 0 and st["failed"] == 0
    assert 0.0 < st["p50_latency_s"] <= st["p99_latency_s"] < 30.0
    srv.close()
    for t in twins:
        mtp.mtp_destroy(t)


def _slow_server(mtp, **kw):
    """One robot whose request takes milliseconds (64 iterations of the
    7-link arm at B = 4096), so a poll right after submit finds it pending."""
    srv = mtp.mtp_server_create(max_batch=4, iters_per_request=64, shift_after=1, **kw)
    rid = mtp.mtp_server_register(srv, W.chain(links=7, B=4096, H=128))
    return srv, rid


def test_poll_not_ready_timeout_then_ready(mtp):
    srv, rid = _slow_server(mtp, max_queue=2, max_robots=2)
    x0 = np.zeros(14, dtype=np.float32)
    t = mtp.mtp_submit(srv, rid, x0)
    out = np.full(7, np.nan, dtype=np.float32)
    assert mtp.mtp_poll(srv, t, out, 0.0) == NOT_READY
    assert mtp.mtp_poll(srv, t, out, 1e-4) == TIMEOUT
    assert np.isnan(out).all()
    assert mtp.mtp_poll(srv, t, out, 60.0) == OK
    assert np.isfinite(out).all()
    with pytest.raises(mtp.MtpError) as ei:  # already collected
        mtp.mtp_poll(srv, t, out, 0.0)
    assert ei.value.status == 1
    with pytest.raises(mtp.MtpError) as ei:  # never issued
        mtp.mtp_poll(srv, 10 ** 9, out, 0.0)
    assert ei.value.status == 1
    with pytest.raises(mtp.MtpError) as ei:
        mtp.mtp_submit(srv, 5, x0)  # unknown robot
    assert ei.value.status == 1
    srv.close()


def test_queue_limit_refuses_submits(mtp):
    srv, rid = _slow_server(mtp, max_queue=1, max_robots=1)
    x0 = np.zeros(14, dtype=np.float32)
    tickets, refused = [], 0
    for _ in range(4):  # one goes in flight, one waits, the rest are refused
        try:
            tickets.append(mtp.mtp_submit(srv, rid, x0))
        except mtp.MtpError as e:
            assert e.status == ADMISSION
            refused += 1
    assert refused >= 2 and len(tickets) >= 1
    out = np.empty(7, dtype=np.float32)
    for t in tickets:
        assert mtp.mtp_poll(srv, t, out, 60.0) == OK
    with pytest.raises(mtp.MtpError) as ei:  # robot limit
        mtp.mtp_server_register(srv, W.pointmass(B=64, E=8))
    assert ei.value.status == ADMISSION
    srv.close()


def test_memory_budget_admission(mtp):
    small = W.pointmass(B=256, E=16)
    big = W.chain(links=7, B=8192, H=256)
    # the server plans its robots in batches, without the single-instance
    # pipeline's second candidate buffer
    b_small = mtp.mtp_problem_device_bytes(dict(small, flags=mtp.FLAG_NO_PIPELINE))
    b_big = mtp.mtp_problem_device_bytes(dict(big, flags=mtp.FLAG_NO_PIPELINE))
    assert mtp.mtp_problem_device_bytes(small) - b_small == 256 * 64 * 2 * 4
    assert b_big > 8192 * 256 * 7 * 4  # the candidate tensor alone
    srv = mtp.mtp_server_create(max_batch=4, memory_budget=2 * b_small + b_big // 2)
    assert mtp.mtp_server_register(srv, small) == 0
    with pytest.raises(mtp.MtpError) as ei:
        mtp.mtp_server_register(srv, big)
    assert ei.value.status == ADMISSION and "budget" in str(ei.value)
    assert mtp.mtp_server_register(srv, small) == 1  # a refusal allocates nothing
    st = mtp.mtp_server_get_stats(srv)
    assert st["robots"] == 2 and st["bytes_admitted"] == 2 * b_small
    with pytest.raises(mtp.MtpError) as ei:
        mtp.mtp_server_register(srv, dict(small, E=10 ** 6))  # does not validate
    assert ei.value.status == 1
    srv.close()


def test_submit_many_poll_many_match_single_calls(mtp):
    specs = _fleet()
    srv = mtp.mtp_server_create(max_batch=4, iters_per_request=1, shift_after=1, max_queue=2,
                                max_robots=16)
    ids = np.array([mtp.mtp_server_register(srv, s) for s in specs], dtype=np.int32)
    twins = [mtp.mtp_create(s) for s in specs]
    rng = np.random.default_rng(3)
    for _ in range(2):
        x0s = [_x0(s, rng) for s in specs]
        tickets = mtp.mtp_submit_many(srv, ids, np.concatenate(x0s))
        assert len(set(tickets.tolist())) == len(specs) and (tickets > 0).all()
        status, out, ready = mtp.mtp_poll_many(srv, tickets, 32, timeout_s=30.0)
        assert ready == len(specs) and (status == OK).all()
        for r, s in enumerate(specs):
            want = torch.empty(s["n"], device=DEV)
            mtp.mtp_plan_step(twins[r], torch.tensor(x0s[r], device=DEV), 1, want)
            mtp.mtp_shift(twins[r], 1)
            assert np.array_equal(out[r, :s["n"]], want.cpu().numpy()), r
        status, _, ready = mtp.mtp_poll_many(srv, tickets, 32, 0.0)  # all collected now
        assert ready == 0 and (status == 1).all()
    # a refusal part-way: the requests before it are queued
    with pytest.raises(mtp.MtpError) as ei:
        mtp.mtp_submit_many(srv, np.array([0, 99], dtype=np.int32), np.zeros(64, np.float32))
    assert ei.value.status == 1 and len(ei.value.tickets) == 1
    status, _, ready = mtp.mtp_poll_many(srv, ei.value.tickets, 32, 30.0)
    assert ready == 1
    srv.close()
    for t in twins:
        mtp.mtp_destroy(t)

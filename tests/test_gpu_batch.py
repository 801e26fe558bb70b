"""Batched planning: each instance's result in the mix is bitwise the result
it gets alone (random draws are keyed by (seed, iteration, index), never by
the slot or launch shape), before and after the rollout tiles are tuned."""
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


def _specs():
    specs = W.batch(seed=11, count=10)
    specs.append(W.pointmass(B=512))
    specs.append(W.chain(links=7, B=1000, E=50))
    specs.append(W.pointmass(k=3, B=600, flags=0x4))  # BF16 basis operands
    return specs


def _run_alone(mtp, specs, x0s, iters):
    out = []
    for spec, x0 in zip(specs, x0s):
        h = mtp.mtp_create(spec)
        u = torch.empty(spec["n"], device=DEV)
        mtp.mtp_plan_step(h, torch.tensor(x0, dtype=torch.float32, device=DEV), iters, u)
        mu, sg, it = mtp.mtp_get_state(h)
        buf = mtp.mtp_get_buffers(h)
        cost = torch.as_tensor(buf["cost"], device=DEV).cpu().numpy().copy()
        out.append((mu, sg, it, u.cpu().numpy(), cost))
        mtp.mtp_destroy(h)
    return out


@pytest.mark.parametrize("tune", [False, True])
def test_batch_matches_each_instance_alone(mtp, tune):
    specs = _specs()
    rng = np.random.default_rng(0)
    x0s = [rng.uniform(-0.2, 0.2, size=s["d"]).astype(np.float32) for s in specs]
    iters = 3
    handles = [mtp.mtp_create(s) for s in specs]
    b = mtp.mtp_batch_create(handles)
    if tune:
        tiles = mtp.mtp_batch_autotune(b)
        assert all(blk in (32, 64, 128) and chunk in (0, 4, 8) and spt in (1, 2)
                   for _, _, blk, chunk, spt in tiles)
    x0 = torch.tensor(np.concatenate(x0s), device=DEV)
    us = torch.empty(b.ustar_offset[-1], device=DEV)
    mtp.mtp_batch_plan_step(b, x0, 1, us)
    mtp.mtp_batch_plan_step(b, x0, iters - 1, us)
    torch.cuda.synchronize()
    ref = _run_alone(mtp, specs, x0s, iters)
    for i, (h, (mu, sg, it, u, cost)) in enumerate(zip(handles, ref)):
        mu_b, sg_b, it_b = mtp.mtp_get_state(h)
        assert it_b == it == iters
        assert np.array_equal(mu_b, mu), i
        assert np.array_equal(sg_b, sg), i
        lo, hi = b.ustar_offset[i], b.ustar_offset[i + 1]
        assert np.array_equal(us[lo:hi].cpu().numpy(), u), i
        cost_b = torch.as_tensor(mtp.mtp_get_buffers(h)["cost"], device=DEV).cpu().numpy()
        assert np.array_equal(cost_b, cost), i
    mtp.mtp_batch_destroy(b)
    for h in handles:
        mtp.mtp_destroy(h)


def _mode_specs():
    specs = _specs()
    specs.append(W.chain(links=11, B=300, H=48))            # longer than the persistent launch covers
    specs.append(W.legged(links=4, B=256, H=32, M=4, N=8))  # legged: its own launch
    specs.append(W.pointmass(k=3, H=33, B=100))             # H * n not a multiple of 4: direct loads
    return specs


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_persistent_rollouts_match_each_instance_alone(mtp, mode):
    """The point-mass and chain rollouts of the whole batch in one persistent
    launch (staged or direct tiles), beside the launches of the groups it
    does not cover: every instance's u*, costs and next state are the bits
    it gets alone."""
    specs = _mode_specs()
    rng = np.random.default_rng(1)
    x0s = [rng.uniform(-0.2, 0.2, size=s["d"]).astype(np.float32) for s in specs]
    iters = 3
    handles = [mtp.mtp_create(s) for s in specs]
    b = mtp.mtp_batch_create(handles)
    groups_launches = mtp.mtp_batch_launches(b, 1)
    mtp.mtp_batch_set_rollout_mode(b, mode)
    assert mtp.mtp_batch_rollout_mode(b)[0] == mode
    covered = len({(s["dyn"], s["n"] if s["dyn"] == "pointmass" else s["n_links"]) for s in specs
                   if (s["dyn"] == "pointmass" and s["n"] <= 16) or
                   (s["dyn"] == "chain" and s["n_links"] <= 9)})
    assert mtp.mtp_batch_launches(b, 1) == groups_launches - covered + (2 if mode == 3 else 1)
    x0 = torch.tensor(np.concatenate(x0s), device=DEV)
    us = torch.empty(b.ustar_offset[-1], device=DEV)
    mtp.mtp_batch_plan_step(b, x0, 1, us)          # direct launches
    mtp.mtp_batch_plan_step(b, x0, iters - 1, us)  # graph replay
    torch.cuda.synchronize()
    for h in handles:
        mtp.mtp_device_status(h)  # raises if a bounded wait gave up
    ref = _run_alone(mtp, specs, x0s, iters)
    for i, (h, (mu, sg, it, u, cost)) in enumerate(zip(handles, ref)):
        mu_b, sg_b, it_b = mtp.mtp_get_state(h)
        assert it_b == it == iters
        assert np.array_equal(mu_b, mu), i
        assert np.array_equal(sg_b, sg), i
        lo, hi = b.ustar_offset[i], b.ustar_offset[i + 1]
        assert np.array_equal(us[lo:hi].cpu().numpy(), u), i
        cost_b = torch.as_tensor(mtp.mtp_get_buffers(h)["cost"], device=DEV).cpu().numpy()
        assert np.array_equal(cost_b, cost), i
    # the persistent launch timed alone covers the point-mass and chain rollouts
    ms, steps = mtp.mtp_batch_persistent_time(b, reps=2)
    assert ms > 0
    assert steps == sum(s["B"] * s["H"] for s in specs
                        if (s["dyn"] == "pointmass" and s["n"] <= 16) or
                        (s["dyn"] == "chain" and s["n_links"] <= 9))
    with pytest.raises(mtp.MtpError):
        mtp.mtp_batch_set_rollout_mode(b, 4)
    mtp.mtp_batch_destroy(b)
    for h in handles:
        mtp.mtp_destroy(h)


@pytest.mark.parametrize("mode", [1, 3])
def test_persistent_modes_with_one_or_no_covered_group(mtp, mode):
    """Degenerate batches for the persistent modes: only legged robots (no
    instance is covered, the groups' own launches run) and a single covered
    group beside a legged robot (the two-launch mode has no group boundary to
    split at and runs one launch).  Bits as alone."""
    for specs in ([W.legged(links=4, B=256, H=32, M=4, N=8, seed=s) for s in (5, 6)],
                  [W.chain(links=5, B=700, H=40, seed=s) for s in (7, 8, 9)] +
                  [W.legged(links=4, B=256, H=32, M=4, N=8)]):
        rng = np.random.default_rng(len(specs))
        x0s = [rng.uniform(-0.2, 0.2, size=s["d"]).astype(np.float32) for s in specs]
        handles = [mtp.mtp_create(s) for s in specs]
        b = mtp.mtp_batch_create(handles)
        mtp.mtp_batch_set_rollout_mode(b, mode)
        x0 = torch.tensor(np.concatenate(x0s), device=DEV)
        us = torch.empty(b.ustar_offset[-1], device=DEV)
        mtp.mtp_batch_plan_step(b, x0, 1, us)
        mtp.mtp_batch_plan_step(b, x0, 1, us)
        torch.cuda.synchronize()
        ms, steps = mtp.mtp_batch_persistent_time(b, reps=1)
        covered = sum(s["B"] * s["H"] for s in specs if s["dyn"] == "chain")
        assert steps == covered and (ms > 0) == (covered > 0)
        ref = _run_alone(mtp, specs, x0s, 2)
        for i, (h, (mu, sg, it, u, cost)) in enumerate(zip(handles, ref)):
            mu_b, sg_b, it_b = mtp.mtp_get_state(h)
            assert it_b == 2 and np.array_equal(mu_b, mu) and np.array_equal(sg_b, sg), i
            lo, hi = b.ustar_offset[i], b.ustar_offset[i + 1]
            assert np.array_equal(us[lo:hi].cpu().numpy(), u), i
        mtp.mtp_batch_destroy(b)
        for h in handles:
            mtp.mtp_destroy(h)


def test_autotune_times_every_rollout_mode_and_restores_states(mtp):
    """The autotuner times whole iterations in each rollout mode from saved
    planner states and restores them: the tuned batch's next iterations are
    still the bits each instance gets alone."""
    specs = _mode_specs()
    rng = np.random.default_rng(2)
    x0s = [rng.uniform(-0.2, 0.2, size=s["d"]).astype(np.float32) for s in specs]
    handles = [mtp.mtp_create(s) for s in specs]
    b = mtp.mtp_batch_create(handles)
    x0 = torch.tensor(np.concatenate(x0s), device=DEV)
    us = torch.empty(b.ustar_offset[-1], device=DEV)
    mtp.mtp_batch_plan_step(b, x0, 1, us)
    mtp.mtp_batch_autotune(b)
    mode, ms = mtp.mtp_batch_rollout_mode(b)
    assert mode in (0, 1, 2, 3) and all(v > 0 for v in ms)
    assert ms[mode] == min(ms)
    mtp.mtp_batch_plan_step(b, x0, 2, us)
    torch.cuda.synchronize()
    ref = _run_alone(mtp, specs, x0s, 3)
    for i, (h, (mu, sg, it, u, cost)) in enumerate(zip(handles, ref)):
        mu_b, sg_b, it_b = mtp.mtp_get_state(h)
        assert it_b == 3
        assert np.array_equal(mu_b, mu), i
        assert np.array_equal(sg_b, sg), i
        lo, hi = b.ustar_offset[i], b.ustar_offset[i + 1]
        assert np.array_equal(us[lo:hi].cpu().numpy(), u), i
    mtp.mtp_batch_destroy(b)
    for h in handles:
        mtp.mtp_destroy(h)


def test_batch_rejects_bad_input(mtp):
    h = mtp.mtp_create(W.pointmass(B=64, E=8))
    with pytest.raises(mtp.MtpError):
        mtp.mtp_batch_create([h, h])
    mtp.mtp_destroy(h)


def test_batch_refill_in_place_and_shift(mtp):
    """A reserved batch refilled with different instance sets (legged robots
    included) and shifted in one launch gives every instance exactly what
    mtp_plan_step + mtp_shift give it alone, cycle after cycle."""
    specs = _specs() + [W.legged(links=4, B=256, H=32, M=6, N=16, E=16)]
    handles = [mtp.mtp_create(s) for s in specs]
    twins = [mtp.mtp_create(s) for s in specs]
    b = mtp.mtp_batch_reserve(8)
    rng = np.random.default_rng(5)
    for sel in ([0, 1, 2, 3, 4, 5], [6, 7, 8, 9, 10, 11, 12], [12, 0, 3]):
        mtp.mtp_batch_fill(b, [handles[i] for i in sel])
        # start states near each spec's own (the legged robot stands on the ground)
        x0s = [(np.asarray(specs[i]["x0"]) + (0.0 if specs[i]["dyn"] == "legged" else
                rng.uniform(-0.2, 0.2, size=specs[i]["d"]))).astype(np.float32) for i in sel]
        us = torch.empty(b.ustar_offset[-1], device=DEV)
        mtp.mtp_batch_plan_step(b, torch.tensor(np.concatenate(x0s), device=DEV), 2, us)
        mtp.mtp_batch_shift(b, 1)
        torch.cuda.synchronize()
        for j, i in enumerate(sel):
            u = torch.empty(specs[i]["n"], device=DEV)
            mtp.mtp_plan_step(twins[i], torch.tensor(x0s[j], device=DEV), 2, u)
            mtp.mtp_shift(twins[i], 1)
            lo, hi = b.ustar_offset[j], b.ustar_offset[j + 1]
            assert np.array_equal(us[lo:hi].cpu().numpy(), u.cpu().numpy()), (sel, i)
    for i, (h, t) in enumerate(zip(handles, twins)):
        mu_b, sg_b, it_b = mtp.mtp_get_state(h)
        mu_t, sg_t, it_t = mtp.mtp_get_state(t)
        assert it_b == it_t and np.array_equal(mu_b, mu_t) and np.array_equal(sg_b, sg_t), i
    with pytest.raises(mtp.MtpError) as ei:
        mtp.mtp_batch_fill(b, handles[:9])  # over capacity
    assert ei.value.status == 1
    mtp.mtp_batch_destroy(b)
    for h in handles + twins:
        mtp.mtp_destroy(h)


def _boundary_clear(cost, E, rtol=1e-4):
    srt = np.sort(np.where(np.isnan(cost), np.inf, cost))
    if E >= len(srt):
        return True
    a, b = srt[E - 1], srt[E]
    return (b - a) > 2 * rtol * max(abs(a), 1.0)


def test_batched_kernels_against_oracle(mtp):
    """The batched kernels (graph, candidate, local-row, rollout, selection
    and update launches over many instances) are separate code from the
    single-instance kernels, so each instance of a mixed batch is also held
    to the FP64 oracle, teacher-forced over two iterations (the first
    launched directly, the second a graph replay): candidates, costs of the
    GPU's candidates, elites exact on the GPU's costs, the FP64 update of
    the GPU's candidates, and u*."""
    import oracle as orc
    specs = [W.pointmass(k=5, H=64, M=7, N=16, B=1024, interp="bspline", degree=2, iters=1),
             W.chain(links=5, H=128, M=9, N=32, B=2048, interp="akima", iters=1),
             W.pointmass(k=3, B=600, flags=0x4),                       # BF16 basis operands
             W.chain(links=3, H=32, M=4, N=8, B=512, interp="bspline", E=16, iters=1),
             W.legged(links=4, B=256, H=32, M=6, N=16, E=16)]
    handles = [mtp.mtp_create(s) for s in specs]
    b = mtp.mtp_batch_create(handles)
    rng = np.random.default_rng(21)
    x0s = [(np.asarray(s["x0"]) + (0.0 if s["dyn"] == "legged" else
            rng.uniform(-0.2, 0.2, size=s["d"]))).astype(np.float32) for s in specs]
    x0 = torch.tensor(np.concatenate(x0s), device=DEV)
    us = torch.empty(b.ustar_offset[-1], device=DEV)
    threads = orc.host_threads()
    for it in range(2):
        before = [mtp.mtp_get_state(h) for h in handles]
        mtp.mtp_batch_plan_step(b, x0, 1, us)
        torch.cuda.synchronize()
        for i, (spec, h) in enumerate(zip(specs, handles)):
            mu, sigma, k = before[i]
            assert k == it
            buf = mtp.mtp_get_buffers(h)
            Ug = torch.as_tensor(buf["U"], device=DEV).cpu().numpy().astype(np.float64)
            cg = torch.as_tensor(buf["cost"], device=DEV).cpu().numpy().astype(np.float64)
            eg = torch.as_tensor(buf["elite"], device=DEV).cpu().numpy()
            xx = x0s[i].astype(np.float64)
            ref = orc.plan_iteration(spec, it, xx, mu, sigma, threads=threads)
            rng_span = (np.array(spec["u_max"]) - np.array(spec["u_min"])).max()
            assert np.abs(Ug - ref["U"]).max() <= 2e-5 * rng_span, (i, it)
            c_ref = orc.rollout_costs(spec, it, xx, Ug, threads=threads)
            err = np.abs(cg - c_ref) / np.maximum(np.abs(c_ref), 1.0)
            err[np.isinf(cg) & np.isinf(c_ref)] = 0.0
            assert err.max() <= 1e-4, (i, it, err.max())
            assert np.array_equal(eg, orc.top_e(cg, spec["E"])), (i, it)
            if _boundary_clear(c_ref, spec["E"]):
                assert set(eg.tolist()) == set(orc.top_e(c_ref, spec["E"]).tolist()), (i, it)
            mu_r, sg_r, us_r = orc.elite_update(spec, Ug, cg, eg, mu, sigma)
            mu_g, sg_g, _ = mtp.mtp_get_state(h)
            np.testing.assert_allclose(mu_g, mu_r, rtol=1e-9, atol=1e-12)
            np.testing.assert_allclose(sg_g, sg_r, rtol=1e-9, atol=1e-12)
            lo, hi = b.ustar_offset[i], b.ustar_offset[i + 1]
            assert np.array_equal(us[lo:hi].cpu().numpy().astype(np.float64), us_r), (i, it)
    mtp.mtp_batch_destroy(b)
    for h in handles:
        mtp.mtp_destroy(h)

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
        assert all(blk in (32, 64, 128) for _, _, blk in tiles)
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

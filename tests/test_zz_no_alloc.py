"""The handle-free, allocation-free elite update must agree with the
handle-based one.

mtp_elite_update_noalloc is for callers that cannot allocate device memory
(they cannot create a handle, whose buffers come from cudaMalloc).  Through
the C ABI it is called twice in a row with different costs, and each time
its elite indices, u*, new mean and new spread are compared with what
mtp_elite_update produces from the same inputs on a handle: both run the
same selection and update kernels, so the results must be the same bits.
The device's free memory and PyTorch's count of allocations are read around
the calls and must not change.  The file is collected last, so a run that stops
at its first failure has run every other test before this one.
"""
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


def _memory():
    """(free device bytes as the driver reports them, allocations PyTorch's
    caching allocator has made so far).  The second is a running count of
    allocation events, so a tensor the test itself frees in between does not
    move it."""
    torch.cuda.synchronize()
    return (torch.cuda.mem_get_info()[0],
            torch.cuda.memory_stats().get("allocation.all.allocated", 0))


@pytest.mark.parametrize("rule,alpha,E,B", [("softmax", 0.0, 64, 4096), ("softmax", 0.25, 512, 4096),
                                            ("plain_cem", 0.1, 16, 4096),
                                            # more elites than selection threads: each
                                            # thread keeps several elites' weights
                                            ("softmax", 0.0, 2048, 4096)])
def test_noalloc_matches_handle_update_twice(mtp, rule, alpha, E, B):
    spec = W.chain(links=7, B=B, E=E, H=128, alpha=alpha, update_rule=rule)
    h = mtp.mtp_create(spec)
    s = h.sizes
    rng = np.random.default_rng(E)
    lo, hi = np.array(spec["u_min"]), np.array(spec["u_max"])
    mu = rng.uniform(lo, hi, size=(s["H"], s["n"])) * 0.3
    sigma = rng.uniform(0.1, 1.0, size=(s["H"], s["n"]))
    mtp.mtp_set_state(h, mu, sigma, 0)
    mu_d = torch.tensor(mu, dtype=torch.float64, device=DEV)
    sg_d = torch.tensor(sigma, dtype=torch.float64, device=DEV)
    el = torch.full((E,), -1, dtype=torch.int32, device=DEV)
    us = torch.zeros(s["n"], dtype=torch.float32, device=DEV)
    el_ref = torch.empty(E, dtype=torch.int32, device=DEV)
    us_ref = torch.empty(s["n"], dtype=torch.float32, device=DEV)
    mem = []
    for call in range(2):
        U = torch.tensor(rng.uniform(lo, hi, size=(s["B"], s["H"], s["n"])), dtype=torch.float32,
                         device=DEV)
        cost = torch.tensor(rng.uniform(100.0, 200.0, size=s["B"]), dtype=torch.float32, device=DEV)
        # existing entry point on a handle
        mtp.mtp_elite_update(h, cost, U, el_ref, us_ref)
        mu_ref, sg_ref, _ = mtp.mtp_get_state(h)
        # the allocation-free entry point on caller-owned state
        el.fill_(-1)
        us.zero_()
        before = _memory()
        mtp.mtp_elite_update_noalloc(cost, U, E, spec["lambda"], alpha, spec["sigma_min"], rule,
                                     mu_d, sg_d, el, us)
        after = _memory()
        mem.append((before, after))
        assert torch.equal(el, el_ref), f"call {call}: elite indices differ"
        assert torch.equal(us, us_ref), f"call {call}: u* differs"
        assert np.array_equal(mu_d.cpu().numpy(), mu_ref), f"call {call}: mean differs"
        assert np.array_equal(sg_d.cpu().numpy(), sg_ref), f"call {call}: spread differs"
    # the second call allocates nothing at all; the first may only have
    # loaded code (the driver's free count moves in whole pages, if at all)
    assert mem[1][0] == mem[1][1], f"device memory changed over the second call: {mem[1]}"
    assert mem[0][0][1] == mem[0][1][1], "PyTorch allocated during the first call"
    mtp.mtp_destroy(h)


def test_noalloc_without_optional_outputs(mtp):
    """elite and u* may be left out: the mean and spread are still updated."""
    spec = W.pointmass(B=2048, E=32, H=64)
    h = mtp.mtp_create(spec)
    s = h.sizes
    rng = np.random.default_rng(3)
    mu = rng.uniform(-0.5, 0.5, size=(s["H"], s["n"]))
    sigma = rng.uniform(0.1, 1.0, size=(s["H"], s["n"]))
    mtp.mtp_set_state(h, mu, sigma, 0)
    U = torch.tensor(rng.uniform(-1, 1, size=(s["B"], s["H"], s["n"])), dtype=torch.float32,
                     device=DEV)
    cost = torch.tensor(rng.uniform(0.0, 5.0, size=s["B"]), dtype=torch.float32, device=DEV)
    mtp.mtp_elite_update(h, cost, U, None, None)
    mu_ref, sg_ref, _ = mtp.mtp_get_state(h)
    mu_d = torch.tensor(mu, dtype=torch.float64, device=DEV)
    sg_d = torch.tensor(sigma, dtype=torch.float64, device=DEV)
    mtp.mtp_elite_update_noalloc(cost, U, 32, spec["lambda"], 0.0, spec["sigma_min"], "softmax",
                                 mu_d, sg_d)
    torch.cuda.synchronize()
    assert np.array_equal(mu_d.cpu().numpy(), mu_ref)
    assert np.array_equal(sg_d.cpu().numpy(), sg_ref)
    mtp.mtp_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_limits(mtp):
    B, H, n = 4096, 128, 7
    U = torch.zeros(B, H, n, device=DEV)
    cost = torch.zeros(B, device=DEV)
    mu = torch.zeros(H, n, dtype=torch.float64, device=DEV)
    sg = torch.ones(H, n, dtype=torch.float64, device=DEV)
    with pytest.raises(mtp.MtpError) as ei:
        mtp.mtp_elite_update_noalloc(cost, U, 4000, 1.0, 0.0, 0.1, "softmax", mu, sg)
    assert ei.value.status == 1 and "MAX_ELITES" in str(ei.value)
    Ub = torch.zeros(8, 1024, 5, device=DEV)
    mub = torch.zeros(1024, 5, dtype=torch.float64, device=DEV)
    with pytest.raises(mtp.MtpError) as ei:
        mtp.mtp_elite_update_noalloc(cost[:8], Ub, 4, 1.0, 0.0, 0.1, "softmax", mub, mub.clone())
    assert ei.value.status == 1 and "MAX_HN" in str(ei.value)

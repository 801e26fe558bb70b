"""Pins of the oracle's elite selection and CEM update (Sec. 2.1, Alg. 2,
Sec. 4.3 corners) and of one full planner iteration."""
import numpy as np
import pytest
from scipy.special import softmax

from paper_2505_01059_gb300 import workloads as W


def test_top_e_brute_force(orc):
    rng = np.random.default_rng(0)
    for B in (1, 2, 7, 64, 1000):
        cost = rng.integers(0, 5, B).astype(float)  # many ties
        for E in {1, min(3, B), B}:
            got = orc.top_e(cost, E)
            ref = np.lexsort((np.arange(B), cost))[:E]
            np.testing.assert_array_equal(got, ref)


def test_top_e_nan_is_inf_and_permutation(orc):
    cost = np.array([3.0, np.nan, 1.0, np.inf, 1.0, -2.0])
    np.testing.assert_array_equal(orc.top_e(cost, 6), [5, 2, 4, 0, 1, 3])
    rng = np.random.default_rng(1)
    cost = rng.normal(size=300)
    perm = rng.permutation(300)
    a = orc.top_e(cost, 20)
    b = orc.top_e(cost[perm], 20)
    np.testing.assert_array_equal(perm[b], a)


def test_softmax_weights(orc):
    rng = np.random.default_rng(2)
    cost = rng.uniform(0, 10, 50)
    elite = orc.top_e(cost, 10)
    for lam in (0.01, 0.1, 1.0, 10.0):
        w = orc.softmax_weights(cost, elite, lam)
        np.testing.assert_allclose(w, softmax(-cost[elite] / lam), rtol=1e-12)
        assert w.sum() == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(orc.softmax_weights(cost, elite, 1e12), 0.1, rtol=1e-9)
    w0 = orc.softmax_weights(cost, elite, 1e-6)
    assert w0[0] == pytest.approx(1.0) and w0[1:].max() < 1e-12


def _setup(E, B=12, H=5, n=2, alpha=0.0, rule="softmax", lam=0.5, sigma_min=0.1):
    spec = W.pointmass(k=n, H=H, B=B, E=E, alpha=alpha, update_rule=rule, sigma_min=sigma_min)
    spec["lambda"] = lam
    rng = np.random.default_rng(E)
    U = rng.uniform(-1, 1, size=(B, H, n))
    cost = rng.uniform(0, 3, B)
    mu = rng.uniform(-1, 1, size=(H, n))
    sigma = rng.uniform(0.2, 1, size=(H, n))
    return spec, U, cost, mu, sigma


def test_softmax_update_moments(orc):
    spec, U, cost, mu, sigma = _setup(E=6)
    elite = orc.top_e(cost, 6)
    mu1, s1, ustar = orc.elite_update(spec, U, cost, elite, mu, sigma)
    w = softmax(-cost[elite] / 0.5)
    Ue = U[elite]
    m = np.tensordot(w, Ue, axes=1)
    s = np.sqrt(np.tensordot(w, (Ue - m) ** 2, axes=1))
    np.testing.assert_allclose(mu1, m, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(s1, np.maximum(s, 0.1), rtol=1e-12)
    assert np.all(s1 >= 0.1)
    np.testing.assert_array_equal(ustar, U[np.argmin(cost), 0])


def test_smoothing(orc):
    spec, U, cost, mu, sigma = _setup(E=4, alpha=0.3)
    elite = orc.top_e(cost, 4)
    mu_a, s_a, _ = orc.elite_update(spec, U, cost, elite, mu, sigma)
    spec0 = dict(spec, alpha=0.0)
    mu_0, s_0, _ = orc.elite_update(spec0, U, cost, elite, mu, sigma)
    np.testing.assert_allclose(mu_a, mu_0 + 0.3 * (mu - mu_0), rtol=1e-14)
    np.testing.assert_allclose(s_a, s_0 + 0.3 * (sigma - s_0), rtol=1e-14)


def test_ps_corner_single_elite(orc):
    # E = 1 (PS corner, Sec. 4.3): the new mean is the best candidate, spread at sigma_min
    spec, U, cost, mu, sigma = _setup(E=1)
    elite = orc.top_e(cost, 1)
    mu1, s1, _ = orc.elite_update(spec, U, cost, elite, mu, sigma)
    np.testing.assert_array_equal(mu1, U[np.argmin(cost)])
    np.testing.assert_array_equal(s1, 0.1)


def test_plain_cem_update_equals_sec21(orc):
    """update_rule plain CEM: mean and 1/(E-1) variance of the elites
    (Sec. 2.1, CEM update) with alpha*old + (1-alpha)*new smoothing."""
    spec, U, cost, mu, sigma = _setup(E=5, alpha=0.25, rule="plain_cem")
    elite = orc.top_e(cost, 5)
    mu1, s1, _ = orc.elite_update(spec, U, cost, elite, mu, sigma)
    m = U[elite].mean(axis=0)
    s = U[elite].std(axis=0, ddof=1)
    np.testing.assert_allclose(mu1, 0.25 * mu + 0.75 * m, rtol=1e-13)
    np.testing.assert_allclose(s1, 0.25 * sigma + 0.75 * s, rtol=1e-13)


def test_mppi_corner_uniform_at_large_lambda(orc):
    # E = B with a huge temperature: weights uniform, the mean is the batch mean
    spec, U, cost, mu, sigma = _setup(E=12, lam=1e15)
    elite = orc.top_e(cost, 12)
    mu1, _, _ = orc.elite_update(spec, U, cost, elite, mu, sigma)
    np.testing.assert_allclose(mu1, U.mean(axis=0), rtol=1e-9, atol=1e-12)


def test_shift_warm_start(orc):
    mu = np.arange(10.0).reshape(5, 2)
    sg = mu + 100
    m2, s2 = orc.shift(mu, sg, 2)
    np.testing.assert_array_equal(m2, [[4, 5], [6, 7], [8, 9], [8, 9], [8, 9]])
    np.testing.assert_array_equal(s2, m2 + 100)


def test_iteration_layout_full_tensor(orc):
    """beta = 1: no local samples; every row but the last is an interpolated
    graph path, the last row is the clamped nominal mean (Alg. 2 stacking)."""
    spec = W.pointmass(k=2, H=16, M=4, N=8, B=33, beta=1.0, E=4)
    pr = orc.make_problem(spec)
    assert pr.P == 32
    mu, sigma = W.initial_distribution(spec)
    x0 = np.zeros(4)
    out = orc.plan_iteration(spec, 0, x0, mu, sigma)
    Z = orc.graph_Z(spec, 0)
    I = orc.path_indices(spec, 0)
    UG = orc.interpolate(spec, orc.gather_C(spec, Z, I))
    np.testing.assert_array_equal(out["U"][:32], np.clip(UG, -1, 1))
    np.testing.assert_array_equal(out["U"][32], mu)


def test_local_only_corner_reduces_to_plain_cem(orc):
    """beta = 0 (local samples only) with the plain CEM update is Sec. 2.1's
    CEM: the iteration's new mean / std are the elite mean and 1/(E-1) std
    of its own candidates, which are Gaussian draws around mu."""
    spec = W.pointmass(k=2, H=10, B=64, beta=0.0, E=8, update_rule="plain_cem")
    pr = orc.make_problem(spec)
    assert pr.P == 0
    mu, sigma = W.initial_distribution(spec)
    mu = mu + 0.1
    sigma = sigma * 0.3
    x0 = np.array([0.1, -0.2, 0.0, 0.0])
    out = orc.plan_iteration(spec, 4, x0, mu, sigma)
    UL = orc.local_samples(spec, 4, mu, sigma)
    np.testing.assert_array_equal(out["U"][:63], np.clip(UL, -1, 1))
    elite = np.lexsort((np.arange(64), out["cost"]))[:8]
    np.testing.assert_array_equal(out["elite"], elite)
    np.testing.assert_allclose(out["mu"], out["U"][elite].mean(axis=0), rtol=1e-13)
    np.testing.assert_allclose(out["sigma"], out["U"][elite].std(axis=0, ddof=1), rtol=1e-12)


def test_planner_improves_pointmass(orc):
    # behavioural check (not parity): the best cost falls over the iterations
    spec = W.pointmass(B=256, iters=8)
    mu, sigma = W.initial_distribution(spec)
    x0 = np.array(spec["x0"])
    best = []
    for it in range(8):
        out = orc.plan_iteration(spec, it, x0, mu, sigma)
        mu, sigma = out["mu"], out["sigma"]
        best.append(out["cost"].min())
    assert best[-1] <= best[0]
    assert np.all(np.isfinite(best))


def test_cost_entropy(orc):
    assert orc.cost_entropy(np.zeros(64), 0.1) == pytest.approx(np.log(64))
    assert orc.cost_entropy(np.array([0.0, 1e6, 1e6]), 0.1) == pytest.approx(0.0, abs=1e-12)


def test_cost_entropy_two_levels(orc):
    """k candidates at cost 0 and m at cost d: with q = exp(-d / lambda) each
    cheap candidate has p = 1 / (k + m q) and each dear one p q, so
    H = log(k + m q) + m q (d / lambda) / (k + m q); the cheap ones weigh
    more (the exp(-J / lambda) reading)."""
    k, m, d, lam = 5, 3, 0.7, 0.25
    q = np.exp(-d / lam)
    Z = k + m * q
    want = np.log(Z) + m * q * (d / lam) / Z
    cost = np.array([0.0] * k + [d] * m)
    assert orc.cost_entropy(cost, lam) == pytest.approx(want, rel=1e-13)
    assert orc.cost_entropy(cost + 17.0, lam) == pytest.approx(want, rel=1e-12)  # shift invariant

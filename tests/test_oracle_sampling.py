"""Pins of the oracle's random draws: Philox, Def. 1 graph, Alg. 1 paths,
the Gaussian local sampler and the beta-mixing layout (Alg. 2)."""
import itertools
import os

import numpy as np
import pytest
from scipy import stats

from paper_2505_01059_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert orc.philox4x32_10(ctr, key) == out


def test_graph_samples_count_and_corners(orc):
    # Alg. 2: P = floor(beta B) graph paths, B-P-1 local samples, mu last.
    assert orc.num_graph_samples(0.5, 512) == 256
    assert orc.num_graph_samples(0.3, 16384) == 4915
    assert orc.num_graph_samples(0.0, 128) == 0        # local-only corner (PS / MPPI)
    assert orc.num_graph_samples(1.0, 128) == 127      # full tensor sampling: 0 local
    assert orc.num_graph_samples(0.999, 4) == 3


def test_graph_Z_uniform_in_box(orc):
    # Def. 1: every layer's waypoints are uniform over the control box.
    spec = W.pointmass(k=3, M=64, N=64, u_min=[-1.0, 0.0, -5.0], u_max=[1.0, 2.0, 5.0])
    Z = orc.graph_Z(spec, 7)
    assert Z.shape == (64, 64, 3)
    lo = np.array(spec["u_min"])
    hi = np.array(spec["u_max"])
    assert np.all(Z >= lo) and np.all(Z < hi)
    for i in range(3):
        u = (Z[:, :, i].ravel() - lo[i]) / (hi[i] - lo[i])
        assert stats.kstest(u, "uniform").pvalue > 1e-3
    # a different iteration gives a different graph (Alg. 2 resamples it)
    assert not np.array_equal(Z, orc.graph_Z(spec, 8))


def test_alg1_brute_force_2x3_graph(orc):
    """Alg. 1 on G(2, 3): every sampled C row is one of the 9 enumerated paths,
    the 9 paths are equally likely (chi-square, 8 dof) and the empirical
    entropy approaches M log N = 2 log 3 (Appendix, tensor-sampling entropy)."""
    spec = W.pointmass(k=2, M=2, N=3, B=900_001, beta=0.9)
    P = 900_000
    it = 3
    Z = orc.graph_Z(spec, it)
    I = orc.path_indices(spec, it, P)
    assert I.shape == (P, 2)
    assert I.min() == 0 and I.max() == 2
    C = orc.gather_C(spec, Z, I)
    # every C row is one of the N^M enumerated paths
    paths = np.array([[Z[0, a], Z[1, b]] for a, b in itertools.product(range(3), range(3))])
    which = np.full(P, -1)
    for p, path in enumerate(paths):
        hit = np.all(np.isclose(C, path[None], rtol=0, atol=0), axis=(1, 2))
        which[hit] = p
    assert np.all(which >= 0)
    counts = np.bincount(which, minlength=9)
    chi2 = float(((counts - P / 9.0) ** 2 / (P / 9.0)).sum())
    assert chi2 < 26.12, chi2  # p = 0.001 critical value for 8 degrees of freedom
    p_emp = counts / P
    H_emp = float(-(p_emp * np.log(p_emp)).sum())
    assert abs(H_emp - 2 * np.log(3)) < 1e-4


def test_path_index_layers_independent(orc):
    spec = W.pointmass(k=2, M=6, N=5, B=200_001, beta=0.9)
    I = orc.path_indices(spec, 0, 200_000)
    for m in range(6):
        c = np.bincount(I[:, m], minlength=5)
        chi2 = float(((c - 40_000) ** 2 / 40_000).sum())
        assert chi2 < 18.47  # 4 dof, p = 0.001
    # joint distribution of two layers is uniform over 25 cells (independence)
    c2 = np.bincount(I[:, 1] * 5 + I[:, 4], minlength=25)
    chi2 = float(((c2 - 8000) ** 2 / 8000).sum())
    assert chi2 < 51.18  # 24 dof, p = 0.001


def test_gaussian_local_samples(orc):
    spec = W.pointmass(k=4, H=250, B=2001, beta=0.0)
    L = 2000
    mu = np.zeros((250, 4))
    sigma = np.ones((250, 4))
    eps = orc.local_samples(spec, 5, mu, sigma, L).ravel()
    n = eps.size  # 2e6 draws
    assert abs(eps.mean()) < 5 / np.sqrt(n)
    assert abs(eps.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert stats.kstest(eps[:200_000], "norm").pvalue > 1e-3
    # the draws of one generator call are independent pairs (Box-Muller)
    e0, e1 = eps[0::4], eps[1::4]
    assert abs(np.corrcoef(e0, e1)[0, 1]) < 5 / np.sqrt(e0.size)


def test_gaussian_affine_map_exact(orc):
    spec = W.pointmass(k=2, H=8, B=11, E=4, beta=0.0)
    rng = np.random.default_rng(0)
    mu = rng.normal(size=(8, 2))
    sigma = rng.uniform(0.1, 2.0, size=(8, 2))
    UL = orc.local_samples(spec, 2, mu, sigma, 10)
    for b in range(10):
        for t in range(8):
            for i in range(2):
                eps = orc.standard_normal(spec["seed"], 2, b, t * 2 + i)
                assert UL[b, t, i] == mu[t, i] + sigma[t, i] * eps


def test_stack_layout_and_clamp(orc):
    # Alg. 2 stacking order: local rows, graph rows, then the nominal mu.
    spec = W.pointmass(k=2, H=5, B=10, E=4, beta=0.5)
    pr = orc.make_problem(spec)
    P, L = pr.P, 10 - pr.P - 1
    assert (P, L) == (5, 4)
    UL = np.full((L, 5, 2), 0.25)
    UG = np.full((P, 5, 2), -0.5)
    mu = np.full((5, 2), 3.0)  # outside the box: must be clamped
    U = orc.stack_clamp(spec, UL, UG, mu)
    assert np.all(U[:L] == 0.25)
    assert np.all(U[L:L + P] == -0.5)
    assert np.all(U[-1] == 1.0)


def test_dr_scales(orc):
    spec = W.chain(links=3, dr_lo=0.8, dr_hi=1.2)
    v = np.array([orc.dr_scale(spec, 0, b, j) for b in range(2000) for j in range(3)])
    assert np.all(v >= 0.8) and np.all(v < 1.2)
    assert abs(v.mean() - 1.0) < 0.01
    spec["dr_mode"] = "none"
    assert orc.dr_scale(spec, 0, 5, 1) == 1.0

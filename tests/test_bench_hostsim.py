"""The serving benchmark's host simulator (the robots' true motion between
re-plans) steps each robot's own nominal model: one step of it agrees with
one step of the FP64 oracle's rollout (recursive Newton-Euler there, the
Lagrangian in absolute angles here) for point masses and arms."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2505_01059_gb300 import workloads as W  # noqa: E402


@pytest.mark.parametrize("links", [1, 3, 7, 9])
def test_hostsim_arm_step_matches_oracle(orc, links):
    rng = np.random.default_rng(links)
    specs = [W.chain(seed=40 + i, links=links, H=1, B=4, E=2, mass_dr=0.0) for i in range(3)]
    x0s = [np.concatenate([rng.uniform(-1, 1, links), rng.uniform(-2, 2, links)]) for _ in specs]
    U = [rng.uniform(-2, 2, links) for _ in specs]
    sim = bench.HostSim(specs, x0s)
    sim.defer(range(3), U)
    sim.flush()
    for r, s in enumerate(specs):
        X, _ = orc.rollout_states(s, 0, x0s[r], U[r][None, :], 0)
        np.testing.assert_allclose(sim.state(r), X[1], rtol=1e-10, atol=1e-12)


def test_hostsim_pointmass_and_mixed_groups(orc):
    rng = np.random.default_rng(1)
    specs = [W.pointmass(seed=3, k=2, H=1, B=4, E=2), W.chain(seed=4, links=4, H=1, B=4, E=2,
                                                                mass_dr=0.0),
             W.pointmass(seed=5, k=5, H=1, B=4, E=2)]
    x0s = [rng.normal(size=s["d"]) for s in specs]
    U = [rng.uniform(-1, 1, s["n"]) for s in specs]
    sim = bench.HostSim(specs, x0s)
    sim.defer([2, 0, 1], [U[2], U[0], U[1]])
    for r, s in enumerate(specs):
        X, _ = orc.rollout_states(s, 0, x0s[r], U[r][None, :], 0)
        np.testing.assert_allclose(sim.state(r), X[1], rtol=1e-10, atol=1e-12)

"""Pins of the oracle's rollout (Eq. 2 with the synthetic task models):
closed forms, textbook two-link dynamics, power balance, energy drift and
contact statics."""
import numpy as np
import pytest

from paper_2505_01059_gb300 import workloads as W


def test_double_integrator_closed_form(orc):
    """Semi-implicit Euler v += dt u, p += dt v has the closed form
    v_T = v_0 + dt sum u_t,  p_T = p_0 + T dt v_0 + dt^2 sum_t (T - t) u_t."""
    k, H, dt = 3, 40, 0.02
    spec = W.pointmass(k=k, H=H, dt=dt, n_obstacles=0, u_min=[-5] * k, u_max=[5] * k)
    rng = np.random.default_rng(0)
    U = rng.uniform(-1, 1, size=(H, k))
    x0 = rng.normal(size=2 * k)
    X, J = orc.rollout_states(spec, 0, x0, U, 0)
    p0, v0 = x0[:k], x0[k:]
    for T in range(H + 1):
        vT = v0 + dt * U[:T].sum(axis=0)
        pT = p0 + T * dt * v0 + dt * dt * ((T - np.arange(T))[:, None] * U[:T]).sum(axis=0)
        np.testing.assert_allclose(X[T, k:], vT, rtol=0, atol=1e-13)
        np.testing.assert_allclose(X[T, :k], pT, rtol=0, atol=1e-13)
    # Eq. 2 with the goal term only: sum over t < T plus the weighted terminal term
    g = np.array(spec["target"])
    d2 = ((X[:, :k] - g) ** 2).sum(axis=1)
    assert J == pytest.approx(d2[:H].sum() + spec["w_term"] * d2[H], rel=1e-13)


def test_pointmass_obstacle_penetration(orc):
    spec = W.pointmass(k=2, H=1, dt=0.02, n_obstacles=0, w_term=0.0, target=[0, 0])
    spec.update(obs_c=[[0.0, 0.0]], obs_r=[0.5], w_obs=1000.0, w_target=0.0)
    x0 = np.array([0.2, 0.0, 0.0, 0.0])
    _, J = orc.rollout_states(spec, 0, x0, np.zeros((1, 2)), 0)
    assert J == pytest.approx(1000.0 * 0.3, rel=1e-14)
    x0 = np.array([0.7, 0.0, 0.0, 0.0])
    _, J = orc.rollout_states(spec, 0, x0, np.zeros((1, 2)), 0)
    assert J == 0.0


def test_pendulum_one_link(orc):
    # thin rod about its end: phi'' = 3 tau/(m l^2) - (3 g / 2 l) cos(phi)
    m, l, g = 1.7, 0.45, 9.81
    for phi, tau in [(0.0, 0.0), (0.3, 1.2), (-2.0, -0.7), (1.5707963, 0.0)]:
        qdd = orc.chain_forward_dynamics([m], [l], g, [phi], [0.9], [tau])
        assert qdd[0] == pytest.approx(3 * tau / (m * l * l) - 1.5 * g / l * np.cos(phi), rel=1e-12,
                                       abs=1e-12)


def test_two_link_textbook(orc):
    """Two-link planar arm (e.g. Spong, Robot Modeling and Control, Sec. 7.4):
    M(q) qdd + c(q, qd) + g(q) = tau with thin rods (lc = l/2, I = m l^2/12)."""
    rng = np.random.default_rng(5)
    g0 = 9.81
    for _ in range(20):
        m1, m2 = rng.uniform(0.5, 2, 2)
        l1, l2 = rng.uniform(0.2, 0.6, 2)
        q = rng.uniform(-3, 3, 2)
        qd = rng.uniform(-2, 2, 2)
        tau = rng.uniform(-5, 5, 2)
        lc1, lc2 = l1 / 2, l2 / 2
        I1, I2 = m1 * l1 * l1 / 12, m2 * l2 * l2 / 12
        c2 = np.cos(q[1])
        M = np.array([
            [m1 * lc1 ** 2 + m2 * (l1 ** 2 + lc2 ** 2 + 2 * l1 * lc2 * c2) + I1 + I2,
             m2 * (lc2 ** 2 + l1 * lc2 * c2) + I2],
            [m2 * (lc2 ** 2 + l1 * lc2 * c2) + I2, m2 * lc2 ** 2 + I2]])
        h = -m2 * l1 * lc2 * np.sin(q[1])
        cvec = np.array([h * qd[1] ** 2 + 2 * h * qd[0] * qd[1], -h * qd[0] ** 2])
        gvec = np.array([(m1 * lc1 + m2 * l1) * g0 * np.cos(q[0]) + m2 * lc2 * g0 * np.cos(q[0] + q[1]),
                         m2 * lc2 * g0 * np.cos(q[0] + q[1])])
        ref = np.linalg.solve(M, tau - cvec - gvec)
        got = orc.chain_forward_dynamics([m1, m2], [l1, l2], g0, q, qd, tau)
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("nl", [1, 2, 3, 5, 7, 9, 12])
def test_chain_power_balance(orc, nl):
    """dE/dt = qd . tau: the forward dynamics (recursive Newton-Euler) agrees
    with the separately written kinetic + potential energy."""
    rng = np.random.default_rng(nl)
    mass = rng.uniform(0.5, 2, nl)
    length = rng.uniform(0.2, 0.4, nl)
    for _ in range(5):
        q = rng.uniform(-np.pi, np.pi, nl)
        qd = rng.uniform(-2, 2, nl)
        tau = rng.uniform(-10, 10, nl)
        qdd = orc.chain_forward_dynamics(mass, length, 9.81, q, qd, tau)
        h = 1e-6
        Ep = orc.chain_energy(mass, length, 9.81, q + h * qd, qd + h * qdd)
        Em = orc.chain_energy(mass, length, 9.81, q - h * qd, qd - h * qdd)
        dE = (Ep - Em) / (2 * h)
        assert dE == pytest.approx(float(qd @ tau), rel=1e-6, abs=1e-6)


def test_chain_energy_drift_zero_torque(orc):
    """Zero torque, no friction: the energy of semi-implicit Euler is exact up
    to O(dt).  Over 1 s of a falling 7-link chain the largest energy error
    halves when dt halves (first-order convergence; a wrong force term would
    leave an O(1) error) and stays small against the kinetic energy reached."""
    nl = 7
    rng = np.random.default_rng(9)
    x0 = np.concatenate([rng.uniform(-0.5, 0.5, nl), np.zeros(nl)])
    errs = []
    for dt in (1e-3, 5e-4, 2.5e-4):
        steps = int(round(1.0 / dt))
        spec = W.chain(links=nl, H=steps, dt=dt, mass_dr=0.0, tau_max=1.0)
        X, _ = orc.rollout_states(spec, 0, x0, np.zeros((steps, nl)), 0)
        E = np.array([orc.chain_energy(spec["mass"], spec["length"], 9.81, x[:nl], x[nl:])
                      for x in X])
        KE = E - np.array([orc.chain_energy(spec["mass"], spec["length"], 9.81, x[:nl], 0 * x[nl:])
                           for x in X])
        errs.append(np.abs(E - E[0]).max())
        assert errs[-1] < 0.06 * KE.max() * (dt / 1e-3)
    assert 1.6 < errs[0] / errs[1] < 2.5
    assert 1.6 < errs[1] / errs[2] < 2.5


def test_legged_free_fall_and_momentum(orc):
    """Far above the ground the floating chain is a free body: with zero joint
    torques at rest it falls at g without rotating; with g = 0 and arbitrary
    joint torques its centre of mass does not accelerate."""
    spec = W.legged(links=4, H=2)
    nl = 4
    mass = np.array(spec["mass"][:nl])
    q = np.array([0.3, 5.0, 0.4, 0.2, -0.5, 0.1])
    qd = np.zeros(6)
    qdd = orc.legged_forward_dynamics(spec, mass, 1.0, q, qd, np.zeros(3))
    np.testing.assert_allclose(qdd, [0, -9.81, 0, 0, 0, 0], atol=1e-10)

    spec0 = dict(spec, gravity=0.0)
    rng = np.random.default_rng(2)
    qd = rng.normal(size=6)
    tau = rng.normal(size=3) * 5
    qdd = orc.legged_forward_dynamics(spec0, mass, 1.0, q, qd, tau)
    L = np.array(spec["length"][:nl])

    def com_rel(qq):
        # centre of mass relative to the base point (small numbers: less roundoff)
        x, y, phi = 0.0, 0.0, 0.0
        acc = np.zeros(2)
        for j in range(nl):
            phi += qq[2 + j]
            e = np.array([np.cos(phi), np.sin(phi)])
            acc += mass[j] * (np.array([x, y]) + 0.5 * L[j] * e)
            x, y = x + L[j] * e[0], y + L[j] * e[1]
        return acc / mass.sum()

    # a_com = base acceleration + J qdd + (d/dt J) qd, the last two as
    # directional differences of the relative centre of mass
    h1 = 1e-5 / np.linalg.norm(qdd)
    h2 = 1e-4 / np.linalg.norm(qd)
    j_qdd = (com_rel(q + h1 * qdd) - com_rel(q - h1 * qdd)) / (2 * h1)
    jd_qd = (com_rel(q + h2 * qd) - 2 * com_rel(q) + com_rel(q - h2 * qd)) / (h2 * h2)
    a_com = qdd[:2] + j_qdd + jd_qd
    scale = np.abs(qdd[:2]).max() + np.abs(j_qdd).max() + np.abs(jd_qd).max()
    np.testing.assert_allclose(a_com, 0.0, atol=1e-6 * scale)


def test_legged_rests_on_ground(orc):
    """One link lying flat with both ends pressed in by m g / (2 k): the two
    spring forces carry the weight, friction is zero at rest, so the body
    stays put (qdd = 0)."""
    spec = W.legged(links=1, H=2)
    m = 1.3
    spec.update(mass=[m], length=[0.5])
    pen = m * 9.81 / (2 * spec["k_contact"])
    q = np.array([0.0, -pen, 0.0])
    qdd = orc.legged_forward_dynamics(spec, np.array([m]), 1.0, q, np.zeros(3), np.zeros(0))
    np.testing.assert_allclose(qdd, 0.0, atol=1e-9)


def test_dr_per_sample_changes_cost(orc):
    spec = W.chain(links=3, H=20, B=4, E=2, mass_dr=0.2)
    U = np.full((2, 20, 3), 2.0)
    x0 = np.zeros(6)
    c = orc.rollout_costs(spec, 0, x0, U, row0=0)
    assert c[0] != c[1]  # same controls, different randomised masses
    spec["dr_mode"] = "none"
    c = orc.rollout_costs(spec, 0, x0, U, row0=0)
    assert c[0] == c[1]


def test_dr_shared_models_average(orc):
    spec = W.chain(links=3, H=20, B=4, E=2, mass_dr=0.2, dr_mode="shared", R=3)
    U = np.full((1, 20, 3), 1.5)
    x0 = np.zeros(6)
    c = orc.rollout_costs(spec, 0, x0, U, row0=0)[0]
    per = []
    for r in range(3):
        s = dict(spec, dr_mode="none", mass=[spec["mass"][j] * orc.dr_scale(spec, 0, r, j)
                                           for j in range(3)])
        per.append(orc.rollout_costs(s, 0, x0, U, row0=0)[0])
    assert c == pytest.approx(np.mean(per), rel=1e-13)

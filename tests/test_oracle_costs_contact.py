"""Pins of the oracle's task costs and ground contact against closed forms.

The reach cost of the serial arm, the Walker-like cost of the legged chain
(Eq. 2's stage and terminal terms, with the task models of the Walker task in
the paper's appendix on task details) and the spring-damper contact with
smoothed Coulomb friction are each fixed here by mechanics or by a hand
calculation, never by the oracle's own formula: forward kinematics of
straight and folded arms, a body sliding on the ground (deceleration mu g),
the vertical force balance of a pressed-in body and the trajectory of the
damped oscillator it forms.
"""
import numpy as np
import pytest

from paper_2505_01059_gb300 import workloads as W


def _stage_cost(orc, spec, x0, u=None):
    """Eq. 2 with H = 1 and no terminal weight: the stage cost at x0."""
    U = np.zeros((1, spec["n"])) if u is None else np.asarray(u, float).reshape(1, -1)
    _, J = orc.rollout_states(spec, 0, x0, U, 0)
    return J


def _arm(nl, lengths, **over):
    spec = W.chain(links=nl, H=1, B=4, E=2, mass_dr=0.0, w_term=0.0, w_ctrl=0.0, **over)
    spec["length"] = list(lengths)
    return spec


def _tip_from_costs(orc, nl, lengths, q, w_target=2.5):
    """Recovers the tip position from the reach cost at three targets:
    J_a = w |tip - a|^2 for a = (0, 0), (1, 0), (0, 1) fixes (x, y)."""
    x0 = np.concatenate([q, np.zeros(nl)])
    J = []
    for tgt in ([0.0, 0.0], [1.0, 0.0], [0.0, 1.0]):
        J.append(_stage_cost(orc, _arm(nl, lengths, target=tgt, w_target=w_target), x0) / w_target)
    return np.array([(J[0] - J[1] + 1.0) / 2.0, (J[0] - J[2] + 1.0) / 2.0]), J[0]


@pytest.mark.parametrize("q, tip", [
    # straight arm along +x: tip at the summed length
    ([0.0, 0.0, 0.0], lambda l: (l.sum(), 0.0)),
    # straight arm pointing up
    ([np.pi / 2, 0.0, 0.0], lambda l: (0.0, l.sum())),
    # straight arm hanging down
    ([-np.pi / 2, 0.0, 0.0], lambda l: (0.0, -l.sum())),
    # first link up, elbow bent back by -90 degrees: the rest points along +x
    # (relative joint angles; absolute ones would give (0, l0 - l1 - l2))
    ([np.pi / 2, -np.pi / 2, 0.0], lambda l: (l[1] + l[2], l[0])),
    # folded at the elbow: the second link, and the third that continues it,
    # come back over the first
    ([0.0, np.pi, 0.0], lambda l: (l[0] - l[1] - l[2], 0.0)),
    # folded twice: out, back, out again
    ([0.0, np.pi, np.pi], lambda l: (l[0] - l[1] + l[2], 0.0)),
    # zig-zag: +x, +y, +x
    ([0.0, np.pi / 2, -np.pi / 2], lambda l: (l[0] + l[2], l[1])),
])
def test_chain_tip_closed_form(orc, q, tip):
    lengths = np.array([0.31, 0.27, 0.22])
    got, _ = _tip_from_costs(orc, 3, lengths, np.array(q))
    np.testing.assert_allclose(got, tip(lengths), rtol=0, atol=1e-12)


def test_chain_reach_cost_value(orc):
    """Hand value: two links (0.5, 0.25) at q = (0, pi/2) put the tip at
    (0.5, 0.25); target (0.1, -0.05) is at distance^2 0.4^2 + 0.3^2 = 0.25,
    so with w_target 4 the stage cost is 1.0, plus w_ctrl |tau|^2 =
    0.5 * (1 + 4) = 2.5 for tau = (1, -2)."""
    spec = _arm(2, [0.5, 0.25], target=[0.1, -0.05], w_target=4.0)
    x0 = np.array([0.0, np.pi / 2, 0.3, -0.7])  # velocities do not enter the reach cost
    assert _stage_cost(orc, spec, x0) == pytest.approx(1.0, rel=1e-13)
    spec["w_ctrl"] = 0.5
    assert _stage_cost(orc, spec, x0, u=[1.0, -2.0]) == pytest.approx(3.5, rel=1e-13)


def test_chain_terminal_term(orc):
    """Without gravity or torque an arm at rest stays put, so Eq. 2 with one
    step is c(x0) (1 + w_term)."""
    spec = _arm(2, [0.5, 0.25], target=[0.1, -0.05], w_target=4.0, gravity=0.0)
    spec["w_term"] = 10.0
    x0 = np.array([0.0, np.pi / 2, 0.0, 0.0])
    assert _stage_cost(orc, spec, x0) == pytest.approx(11.0, rel=1e-13)


def _legged(links=1, **over):
    spec = W.legged(links=links, H=1, B=4, E=2, dr_mode="none", w_term=0.0, w_ctrl=0.0)
    spec.update(over)
    return spec


def test_legged_state_cost_hand_value(orc):
    """Walker-like cost at a hand-set state of a two-link floating chain:
    height y_b = 0.5 (target 0.8), pitch phi_0 = 0.3 (target 0.1), forward
    velocity of the base point 0.4 (target 1.0), weights 10 / 2 / 3:
    10 * 0.09 + 2 * 0.04 + 3 * 0.36 = 2.06.  The other coordinates are set to
    values that would change the sum if they entered it."""
    spec = _legged(links=2, target=[0.8, 1.0, 0.1], w_height=10.0, w_pitch=2.0, w_vel=3.0)
    x0 = np.array([7.0, 0.5, 0.3, 1.1,      # x_b, y_b, phi_0, q_1
                   0.4, -2.0, 3.0, -1.0])   # their rates
    assert _stage_cost(orc, spec, x0) == pytest.approx(2.06, rel=1e-13)
    spec["w_ctrl"] = 0.25
    assert _stage_cost(orc, spec, x0, u=[2.0]) == pytest.approx(3.06, rel=1e-13)


def _flat_body(spec, m=1.3, length=0.5):
    spec.update(mass=[m], length=[length])
    return np.array([m])


@pytest.mark.parametrize("v, mu_scale", [(1.0, 1.0), (0.5, 1.1), (-2.0, 0.85)])
def test_sliding_body_decelerates_at_mu_g(orc, v, mu_scale):
    """A flat link resting on both contact points (each pressed in by
    m g / (2 k), so the springs carry the weight) slides at |v| >> v_slip:
    the smoothed Coulomb force is mu s m g opposite to v, so the body
    decelerates at mu s g, with no vertical or angular acceleration (the
    friction forces act on the line through the centre of mass)."""
    spec = _legged()
    mass = _flat_body(spec)
    m, g, k, mu = 1.3, spec["gravity"], spec["k_contact"], spec["mu_friction"]
    pen = m * g / (2 * k)
    q = np.array([0.0, -pen, 0.0])
    qd = np.array([v, 0.0, 0.0])
    qdd = orc.legged_forward_dynamics(spec, mass, mu_scale, q, qd, np.zeros(0))
    np.testing.assert_allclose(qdd, [-np.sign(v) * mu * mu_scale * g, 0.0, 0.0], atol=1e-10)


def test_friction_smoothing_at_slip_speed(orc):
    """At the slip speed itself the smoothed Coulomb force is tanh(1) of the
    full one; at zero speed it vanishes."""
    spec = _legged()
    mass = _flat_body(spec)
    m, g, k, mu, vs = 1.3, spec["gravity"], spec["k_contact"], spec["mu_friction"], spec["v_slip"]
    q = np.array([0.0, -m * g / (2 * k), 0.0])
    qdd = orc.legged_forward_dynamics(spec, mass, 1.0, q, np.array([vs, 0, 0]), np.zeros(0))
    assert qdd[0] == pytest.approx(-mu * g * np.tanh(1.0), rel=1e-12)
    qdd = orc.legged_forward_dynamics(spec, mass, 1.0, q, np.array([-3 * vs, 0, 0]), np.zeros(0))
    assert qdd[0] == pytest.approx(mu * g * np.tanh(3.0), rel=1e-12)


def test_sliding_trajectory(orc):
    """Rolled out (semi-implicit Euler, constant deceleration is integrated
    exactly in the velocity): v_T = v_0 - mu g T dt while v >> v_slip, and
    the body neither sinks nor tilts."""
    dt, H = 1e-4, 500
    spec = _legged(dt=dt)
    spec["H"] = H
    _flat_body(spec)
    m, g, k, mu = 1.3, spec["gravity"], spec["k_contact"], spec["mu_friction"]
    pen = m * g / (2 * k)
    v0 = 0.8
    x0 = np.array([0.0, -pen, 0.0, v0, 0.0, 0.0])
    X, _ = orc.rollout_states(spec, 0, x0, np.zeros((H, 0)), 0)
    t = np.arange(H + 1) * dt
    np.testing.assert_allclose(X[:, 3], v0 - mu * g * t, atol=1e-9)
    np.testing.assert_allclose(X[:, 1], -pen, atol=1e-12)
    np.testing.assert_allclose(X[:, 2], 0.0, atol=1e-12)


@pytest.mark.parametrize("pen_scale, vy", [(1.0, 0.0), (2.0, 0.0), (1.5, -0.03), (0.5, 0.02),
                                            (1.0, 0.5)])
def test_contact_vertical_balance(orc, pen_scale, vy):
    """Vertical acceleration of a flat link on two contact points, each
    pushing with f_n = max(0, k pen + c d(pen)/dt) = max(0, k pen - c v_y):
    y'' = 2 f_n / m - g.  The last case pulls out of the ground faster than
    the spring pushes, so f_n clips to zero and the body falls freely."""
    spec = _legged()
    mass = _flat_body(spec)
    m, g, k, c = 1.3, spec["gravity"], spec["k_contact"], spec["c_contact"]
    pen = pen_scale * m * g / (2 * k)
    q = np.array([0.0, -pen, 0.0])
    qd = np.array([0.0, vy, 0.0])
    qdd = orc.legged_forward_dynamics(spec, mass, 1.0, q, qd, np.zeros(0))
    f_n = max(0.0, k * pen - c * vy)
    np.testing.assert_allclose(qdd, [0.0, 2 * f_n / m - g, 0.0], atol=1e-9)


def test_damped_bounce_matches_oscillator(orc):
    """Small vertical motion about the resting penetration is the damped
    oscillator z'' + 2 gamma z' + w0^2 z = 0 with w0^2 = 2k/m and
    gamma = c/m (two contact points, each with k and c).  From z0 and rest:
    z(t) = exp(-gamma t) (z0 cos(wd t) + gamma z0 / wd sin(wd t)),
    wd = sqrt(w0^2 - gamma^2).  Semi-implicit Euler at dt 1e-5 follows it to
    well under one percent of the amplitude over 50 ms (several periods)."""
    dt, H = 1e-5, 5000
    spec = _legged(dt=dt)
    spec["H"] = H
    _flat_body(spec)
    m, g, k, c = 1.3, spec["gravity"], spec["k_contact"], spec["c_contact"]
    y_eq = -m * g / (2 * k)
    z0 = -1e-4
    x0 = np.array([0.0, y_eq + z0, 0.0, 0.0, 0.0, 0.0])
    X, _ = orc.rollout_states(spec, 0, x0, np.zeros((H, 0)), 0)
    t = np.arange(H + 1) * dt
    w0sq, gam = 2 * k / m, c / m
    wd = np.sqrt(w0sq - gam * gam)
    z = np.exp(-gam * t) * (z0 * np.cos(wd * t) + gam * z0 / wd * np.sin(wd * t))
    np.testing.assert_allclose(X[:, 1] - y_eq, z, atol=5e-3 * abs(z0))
    # the decay is really there: after 50 ms the amplitude is exp(-gamma t) small
    assert abs(X[-1, 1] - y_eq) < 0.05 * abs(z0)


def test_tilted_spinning_rod_newton_euler(orc):
    """A single rod (mass m, length l, centre of mass at l/2, I = m l^2/12)
    whose ends touch the ground, tilted and spinning, solved by hand:
    contact points r_0 = base, r_1 = base + l e(phi); their velocities by
    rigid-body kinematics v = v_b + w z x (r - r_b); the contact law at each
    (normal max(0, k pen - c v_y), tangential -mu s f_n tanh(v_x / v_slip));
    then Newton's and Euler's equations about the centre of mass, and the
    base point's acceleration a_b = a_c - alpha z x r_c + w^2 r_c."""
    spec = _legged()
    m, length = 1.3, 0.5
    mass = _flat_body(spec, m=m, length=length)
    g, k, c = spec["gravity"], spec["k_contact"], spec["c_contact"]
    mu, vs = spec["mu_friction"], spec["v_slip"]
    rng = np.random.default_rng(11)
    for _ in range(12):
        phi = rng.uniform(-2e-3, 2e-3)
        yb = -rng.uniform(2e-4, 8e-4)
        vb = rng.uniform(-0.05, 0.05, 2)
        w = rng.uniform(-0.3, 0.3)
        s = rng.uniform(0.8, 1.2)
        e = np.array([np.cos(phi), np.sin(phi)])
        pts = [np.array([0.0, yb]), np.array([0.0, yb]) + length * e]
        force = np.zeros(2)
        torque_c = 0.0
        rc = 0.5 * length * e                       # centre of mass from the base
        for r in pts:
            rel = r - pts[0]
            v = vb + w * np.array([-rel[1], rel[0]])
            fn = max(0.0, k * (-r[1]) - c * v[1]) if r[1] < 0 else 0.0
            f = np.array([-mu * s * fn * np.tanh(v[0] / vs), fn])
            force += f
            arm = rel - rc
            torque_c += arm[0] * f[1] - arm[1] * f[0]
        a_c = force / m + np.array([0.0, -g])
        alpha = torque_c / (m * length * length / 12.0)
        a_b = a_c - alpha * np.array([-rc[1], rc[0]]) + w * w * rc
        q = np.array([0.0, yb, phi])
        qd = np.array([vb[0], vb[1], w])
        qdd = orc.legged_forward_dynamics(spec, mass, s, q, qd, np.zeros(0))
        np.testing.assert_allclose(qdd, [a_b[0], a_b[1], alpha], rtol=1e-9, atol=1e-9)

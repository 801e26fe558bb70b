"""Seeded synthetic planning problems shaped like the paper's tasks.

This module holds no step of the planner: it only draws task parameters
(link masses and lengths, obstacle circles, targets) from numpy's seeded
generator and writes them into plain dicts.  Both the CUDA library binding
and the FP64 oracle take these dicts, so every input of a parity test comes
from here; the random numbers the planner itself draws (graph knots, path
indices, Gaussian noise, per-sample model scales) are made by Philox inside
each implementation.

The paper's MuJoCo tasks are not available; these stand in for them:

* ``pointmass`` - the Navigation task's shape (Sec. 4.1, Table 1: state 4,
  control 2) as a double integrator with circular obstacles.
* ``chain`` - a torque-controlled planar serial arm (reach task).
* ``legged`` - a floating-base planar chain with spring-damper ground
  contact, cost modelled on the Walker task (Sec. A, task details).
"""
from __future__ import annotations

import numpy as np


def _base(**kw) -> dict:
    spec = dict(
        time_mapping="valid_span", update_rule="softmax", dr_mode="none", R=1,
        dr_lo=1.0, dr_hi=1.0, alpha=0.0, degree=2, w_obs=0.0, w_ctrl=0.0,
        w_term=1.0, obs_c=[], obs_r=[], n_links=0, mass=[], length=[], gravity=9.81,
        mu_init=0.0,
    )
    spec.update(kw)
    return spec


def pointmass(seed: int = 1, k: int = 2, H: int = 64, M: int = 4, N: int = 8, B: int = 512,
              beta: float = 0.5, interp: str = "bspline", degree: int = 3, E: int = 32,
              n_obstacles: int = 5, iters: int = 10, dt: float = 0.02, **over) -> dict:
    """k-D point-mass double integrator; with the defaults this is the 2-D
    workload: |u| <= 1, dt 0.02, H 64, graph 4 x 8, 512 candidates (256 graph
    paths), cubic B-spline, 5 circular obstacles of radius U[0.1, 0.3] with
    centres U[0, 0.6]^k, goal (0.6, ..., 0.6), top-32 elites, 10 iterations."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 0.6, size=(n_obstacles, k))
    radii = rng.uniform(0.1, 0.3, size=n_obstacles)
    spec = _base(
        dyn="pointmass", n=k, d=2 * k, H=H, dt=dt,
        u_min=[-1.0] * k, u_max=[1.0] * k,
        M=M, N=N, B=B, beta=beta, E=E, interp=interp, degree=degree,
        sigma_init=1.0, sigma_min=0.1, alpha=0.0,
        seed=seed, target=[0.6] * k, w_target=1.0, w_obs=1e3, w_ctrl=0.0, w_term=10.0,
        obs_c=centres.tolist(), obs_r=radii.tolist(),
        x0=[0.0] * (2 * k), iters=iters,
    )
    spec["lambda"] = 0.1
    spec.update(over)
    return spec


def chain(seed: int = 2, links: int = 7, H: int = 128, M: int = 8, N: int = 32, B: int = 4096,
          beta: float = 0.5, interp: str = "akima", E: int = 64, iters: int = 20,
          dt: float = 0.005, tau_max: float = 2.0, mass_dr: float = 0.2, **over) -> dict:
    """Torque-controlled planar serial arm; with the defaults this is the
    7-link workload: masses U[0.5, 2] kg, lengths U[0.2, 0.4] m, per-sample
    mass scale U[0.8, 1.2], semi-implicit Euler dt 0.005, H 128, graph 8 x 32,
    4096 candidates, Akima, reach + torque cost, 20 iterations.  The arm hangs
    in the vertical plane (g = 9.81) with joint torques in [-2, 2] N m: with
    larger boxes random torque profiles whip the light distal links and the
    explicit integrator diverges at dt 0.005."""
    rng = np.random.default_rng(seed)
    mass = rng.uniform(0.5, 2.0, size=links)
    length = rng.uniform(0.2, 0.4, size=links)
    reach = float(length.sum())
    radius = rng.uniform(0.3, 0.8) * reach
    angle = rng.uniform(0.0, 2.0 * np.pi)
    target = [radius * float(np.cos(angle)), radius * float(np.sin(angle))]
    spec = _base(
        dyn="chain", n=links, d=2 * links, H=H, dt=dt,
        u_min=[-tau_max] * links, u_max=[tau_max] * links,
        M=M, N=N, B=B, beta=beta, E=E, interp=interp, degree=2,
        sigma_init=tau_max, sigma_min=0.1 * tau_max, alpha=0.0,
        seed=seed, target=target, w_target=1.0, w_ctrl=1e-2, w_term=10.0,
        n_links=links, mass=mass.tolist(), length=length.tolist(), gravity=9.81,
        dr_mode="per_sample" if mass_dr > 0 else "none",
        dr_lo=1.0 - mass_dr, dr_hi=1.0 + mass_dr,
        x0=[0.0] * (2 * links), iters=iters,
    )
    spec["lambda"] = 5.0
    spec.update(over)
    return spec


def legged(seed: int = 5, links: int = 16, H: int = 256, M: int = 16, N: int = 64,
           B: int = 16384, beta: float = 0.3, interp: str = "bspline", E: int = 64,
           iters: int = 1, dt: float = 0.002, tau_max: float = 5.0, **over) -> dict:
    """Floating-base planar chain with ground contact; with the defaults this
    is the 16-link workload: k 1e4, c 100, friction 0.8 (per-sample scale
    U[0.8, 1.2], also on every link mass), dt 0.002, H 256, graph 16 x 64,
    16384 candidates, beta 0.3, quadratic B-spline with BF16 operands in the
    basis contraction (flags 0x4, FP32 sums).  Links are U[2, 4] kg and
    U[0.15, 0.3] m and the chain starts flat, 2 cm above the ground: with lighter links the
    explicit spring-damper contact at dt 0.002 is unstable (the damper needs
    an effective mass above c dt / 2 = 0.1 kg at each contact point)."""
    rng = np.random.default_rng(seed)
    mass = rng.uniform(2.0, 4.0, size=links)
    length = rng.uniform(0.15, 0.3, size=links)
    nq = links + 2
    q0 = np.zeros(nq)
    q0[1] = 0.02
    spec = _base(
        dyn="legged", n=links - 1, d=2 * nq, H=H, dt=dt,
        u_min=[-tau_max] * (links - 1), u_max=[tau_max] * (links - 1),
        M=M, N=N, B=B, beta=beta, E=E, interp=interp, degree=2,
        sigma_init=tau_max, sigma_min=0.1 * tau_max, alpha=0.0,
        seed=seed, target=[0.8, 1.0, 0.0], w_ctrl=1e-3, w_term=10.0,
        w_height=10.0, w_pitch=1.0, w_vel=1.0,
        n_links=links, mass=mass.tolist(), length=length.tolist(), gravity=9.81,
        k_contact=1e4, c_contact=100.0, mu_friction=0.8, v_slip=0.01,
        dr_mode="per_sample", dr_lo=0.8, dr_hi=1.2,
        x0=q0.tolist() + [0.0] * nq, iters=iters,
        flags=0x4 if interp == "bspline" else 0,
    )
    spec["lambda"] = 1.0
    spec.update(over)
    return spec


def initial_distribution(spec: dict):
    """The nominal mean and spread the planner starts from (Alg. 2 init):
    constant mu_init and sigma_init over the (H, n) horizon."""
    H, n = spec["H"], spec["n"]
    mu = np.full((H, n), float(spec.get("mu_init", 0.0)))
    sigma = np.full((H, n), float(spec["sigma_init"]))
    return mu, sigma


def batch(seed: int = 3, count: int = 256, bf16: bool = False) -> list[dict]:
    """Uneven instances: half k-D point masses (k in 2..12), half chains of
    3..9 links; H in {32, 64, 128, 256}, B in 512..8192 (powers of two),
    M in 4..16, N in {8, 16, 32, 64}, B-spline or Akima at random.  With
    bf16, the B-spline instances contract their basis with BF16 operands
    (flags 0x4); the drawn sizes are the same either way."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        H = int(rng.choice([32, 64, 128, 256]))
        B = int(rng.choice([512, 1024, 2048, 4096, 8192]))
        M = int(rng.integers(4, 17))
        N = int(rng.choice([8, 16, 32, 64]))
        interp = "bspline" if rng.random() < 0.5 else "akima"
        E = 32
        if i % 2 == 0:
            k = int(rng.integers(2, 13))
            spec = pointmass(seed=1000 + i, k=k, H=H, M=M, N=N, B=B, interp=interp, degree=2,
                             E=E, iters=1)
        else:
            links = int(rng.integers(3, 10))
            spec = chain(seed=2000 + i, links=links, H=H, M=M, N=N, B=B, interp=interp, E=E,
                         iters=1)
        if bf16 and interp == "bspline":
            spec["flags"] = spec.get("flags", 0) | 0x4
        out.append(spec)
    return out


def robots(seed: int = 4, count: int = 1024) -> list[dict]:
    """Serving fleet: half 2-D point masses, half 3..9-link arms; H in
    64..128, B in 1024..4096."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        H = int(rng.choice([64, 96, 128]))
        B = int(rng.choice([1024, 2048, 4096]))
        if i % 2 == 0:
            spec = pointmass(seed=5000 + i, H=H, B=B, iters=1, degree=2)
        else:
            spec = chain(seed=6000 + i, links=int(rng.integers(3, 10)), H=H, B=B, iters=1)
        out.append(spec)
    return out

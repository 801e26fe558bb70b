"""ctypes binding of the FP64 C oracle (test infrastructure only).

Build: ``build_oracle()`` compiles ``mtp_oracle.c`` with gcc into
``_liboracle.so`` next to it.  Each wrapper takes and returns numpy arrays in
the paper's logical layouts: Z (M, N, n), I (P, M), C (P, M, n), U (B, H, n),
costs (B,), mu/sigma (H, n).

A problem is given as a plain dict (see ``paper_2505_01059_gb300.workloads``);
``make_problem`` turns it into the oracle's own C struct.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mtp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

MAXN = 32
MAXL = 18
MAXOBS = 8

DYN = {"pointmass": 0, "chain": 1, "legged": 2}
INTERP = {"linear": 0, "bspline": 1, "akima": 2}
TIME_MAPPING = {"valid_span": 0, "paper_literal": 1}
UPDATE = {"softmax": 0, "plain_cem": 1}
DR = {"none": 0, "per_sample": 1, "shared": 2}


class OrProblem(C.Structure):
    _fields_ = [
        ("dyn", C.c_int32), ("n", C.c_int32), ("d", C.c_int32), ("H", C.c_int32),
        ("M", C.c_int32), ("N", C.c_int32), ("B", C.c_int32), ("P", C.c_int32), ("E", C.c_int32),
        ("interp", C.c_int32), ("degree", C.c_int32), ("time_mapping", C.c_int32),
        ("update_rule", C.c_int32),
        ("dr_mode", C.c_int32), ("R", C.c_int32),
        ("seed", C.c_uint64),
        ("dt", C.c_double), ("lam", C.c_double), ("alpha", C.c_double), ("sigma_min", C.c_double),
        ("u_min", C.c_double * MAXN), ("u_max", C.c_double * MAXN),
        ("target", C.c_double * MAXN),
        ("w_target", C.c_double), ("w_obs", C.c_double), ("w_ctrl", C.c_double),
        ("w_term", C.c_double),
        ("n_obs", C.c_int32),
        ("obs_c", (C.c_double * MAXN) * MAXOBS),
        ("obs_r", C.c_double * MAXOBS),
        ("dr_lo", C.c_double), ("dr_hi", C.c_double),
        ("n_links", C.c_int32),
        ("mass", C.c_double * MAXL), ("length", C.c_double * MAXL),
        ("gravity", C.c_double),
        ("k_contact", C.c_double), ("c_contact", C.c_double), ("mu_friction", C.c_double),
        ("v_slip", C.c_double),
        ("w_height", C.c_double), ("w_pitch", C.c_double), ("w_vel", C.c_double),
        ("bf16_basis", C.c_int32),
    ]


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no target-specific flags)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-pthread",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = C.CDLL(_LIB_PATH)
        P = C.POINTER
        dp, ip, up = P(C.c_double), P(C.c_int32), P(C.c_uint32)
        pp = P(OrProblem)
        sig = {
            "or_philox4x32_10": (None, [up, up, up]),
            "or_num_graph_samples": (C.c_int32, [C.c_double, C.c_int32]),
            "or_graph_Z": (None, [pp, C.c_uint32, dp]),
            "or_path_indices": (None, [pp, C.c_uint32, C.c_int32, ip]),
            "or_gather_C": (None, [pp, dp, ip, C.c_int32, dp]),
            "or_bspline_time": (C.c_double, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
            "or_bspline_basis": (None, [C.c_int, C.c_int, C.c_int, C.c_int, dp]),
            "or_interp_bspline": (None, [pp, dp, C.c_int32, dp]),
            "or_bf16_round": (C.c_double, [C.c_double]),
            "or_akima_knot": (C.c_double, [C.c_int, C.c_int, C.c_int]),
            "or_akima_time": (C.c_double, [C.c_int, C.c_int, C.c_int]),
            "or_akima_coeffs": (None, [C.c_int, dp, dp, dp]),
            "or_akima_eval": (C.c_double, [C.c_int, dp, dp, C.c_double]),
            "or_interp_akima": (None, [pp, dp, C.c_int32, dp]),
            "or_interp_linear": (None, [pp, dp, C.c_int32, dp]),
            "or_interpolate": (None, [pp, dp, C.c_int32, dp]),
            "or_standard_normal": (C.c_double, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]),
            "or_local_samples": (None, [pp, C.c_uint32, dp, dp, C.c_int32, dp]),
            "or_stack_clamp": (None, [pp, dp, dp, dp, dp]),
            "or_dr_scale": (C.c_double, [pp, C.c_uint32, C.c_uint32, C.c_uint32]),
            "or_chain_forward_dynamics": (C.c_int, [C.c_int, dp, dp, C.c_double, dp, dp, dp, dp]),
            "or_chain_energy": (C.c_double, [C.c_int, dp, dp, C.c_double, dp, dp]),
            "or_legged_forward_dynamics": (C.c_int, [pp, dp, C.c_double, dp, dp, dp, dp]),
            "or_rollout_costs": (None, [pp, C.c_uint32, dp, dp, C.c_int32, C.c_int32, dp]),
            "or_rollout_costs_threads": (None, [pp, C.c_uint32, dp, dp, C.c_int32, C.c_int32, dp,
                                                C.c_int32]),
            "or_rollout_states": (C.c_double, [pp, C.c_uint32, dp, dp, C.c_int32, dp]),
            "or_top_e": (None, [dp, C.c_int32, C.c_int32, ip]),
            "or_softmax_weights": (None, [dp, ip, C.c_int32, C.c_double, dp]),
            "or_elite_update": (None, [pp, dp, dp, ip, dp, dp, dp]),
            "or_shift": (None, [C.c_int, C.c_int, C.c_int, dp, dp]),
            "or_plan_iteration": (C.c_int, [pp, C.c_uint32, dp, dp, dp, dp, dp, ip, dp]),
            "or_plan_iteration_threads": (C.c_int, [pp, C.c_uint32, dp, dp, dp, dp, dp, ip, dp,
                                                    C.c_int32]),
            "or_cost_entropy": (C.c_double, [dp, C.c_int32, C.c_double]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


# ----------------------------------------------------------------------------
# problem description
# ----------------------------------------------------------------------------

def num_graph_samples(beta: float, B: int) -> int:
    return int(_load().or_num_graph_samples(float(beta), int(B)))


def make_problem(spec: dict) -> OrProblem:
    """Fill the oracle's C struct from a workload dict."""
    if not 1 <= spec["E"] <= spec["B"]:
        raise ValueError("the oracle needs 1 <= E <= B")
    pr = OrProblem()
    pr.dyn = DYN[spec["dyn"]]
    pr.n = spec["n"]
    pr.d = spec["d"]
    pr.H = spec["H"]
    pr.M = spec["M"]
    pr.N = spec["N"]
    pr.B = spec["B"]
    pr.P = num_graph_samples(spec["beta"], spec["B"])
    pr.E = spec["E"]
    pr.interp = INTERP[spec["interp"]]
    pr.degree = spec.get("degree", 2)
    pr.time_mapping = TIME_MAPPING[spec.get("time_mapping", "valid_span")]
    pr.update_rule = UPDATE[spec.get("update_rule", "softmax")]
    pr.dr_mode = DR[spec.get("dr_mode", "none")]
    pr.R = spec.get("R", 1)
    pr.seed = spec["seed"]
    pr.dt = spec["dt"]
    pr.lam = spec["lambda"]
    pr.alpha = spec["alpha"]
    pr.sigma_min = spec["sigma_min"]
    for i in range(spec["n"]):
        pr.u_min[i] = spec["u_min"][i]
        pr.u_max[i] = spec["u_max"][i]
    for i, v in enumerate(spec.get("target", [])):
        pr.target[i] = v
    pr.w_target = spec.get("w_target", 1.0)
    pr.w_obs = spec.get("w_obs", 0.0)
    pr.w_ctrl = spec.get("w_ctrl", 0.0)
    pr.w_term = spec.get("w_term", 1.0)
    obs_c = spec.get("obs_c", [])
    pr.n_obs = len(obs_c)
    for o, (c, r) in enumerate(zip(obs_c, spec.get("obs_r", []))):
        for a, v in enumerate(c):
            pr.obs_c[o][a] = v
        pr.obs_r[o] = r
    pr.dr_lo = spec.get("dr_lo", 1.0)
    pr.dr_hi = spec.get("dr_hi", 1.0)
    pr.n_links = spec.get("n_links", 0)
    for j, v in enumerate(spec.get("mass", [])):
        pr.mass[j] = v
    for j, v in enumerate(spec.get("length", [])):
        pr.length[j] = v
    pr.gravity = spec.get("gravity", 9.81)
    pr.k_contact = spec.get("k_contact", 0.0)
    pr.c_contact = spec.get("c_contact", 0.0)
    pr.mu_friction = spec.get("mu_friction", 0.0)
    pr.v_slip = spec.get("v_slip", 0.01)
    pr.w_height = spec.get("w_height", 0.0)
    pr.w_pitch = spec.get("w_pitch", 0.0)
    pr.w_vel = spec.get("w_vel", 0.0)
    pr.bf16_basis = 1 if (spec.get("flags", 0) & 0x4) else 0
    return pr


def _pr(spec_or_pr):
    return spec_or_pr if isinstance(spec_or_pr, OrProblem) else make_problem(spec_or_pr)


# ----------------------------------------------------------------------------
# wrappers
# ----------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    lib = _load()
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (C.c_uint32 * 4)()
    lib.or_philox4x32_10(c, k, out)
    return [int(v) for v in out]


def graph_Z(spec, it: int) -> np.ndarray:
    pr = _pr(spec)
    Z = np.empty((pr.M, pr.N, pr.n), np.float64)
    _load().or_graph_Z(C.byref(pr), it, _dp(Z))
    return Z


def path_indices(spec, it: int, P: int | None = None) -> np.ndarray:
    pr = _pr(spec)
    P = pr.P if P is None else P
    I = np.empty((max(P, 0), pr.M), np.int32)
    _load().or_path_indices(C.byref(pr), it, P, _ip(I))
    return I


def gather_C(spec, Z, I) -> np.ndarray:
    pr = _pr(spec)
    Z = _f64(Z)
    I = np.ascontiguousarray(I, dtype=np.int32)
    P = I.shape[0]
    Cc = np.empty((P, pr.M, pr.n), np.float64)
    _load().or_gather_C(C.byref(pr), _dp(Z), _ip(I), P, _dp(Cc))
    return Cc


def bspline_time(M, p, H, mapping, j) -> float:
    return float(_load().or_bspline_time(M, p, H, TIME_MAPPING.get(mapping, mapping), j))


def bspline_basis(M: int, p: int, H: int, mapping="valid_span") -> np.ndarray:
    """Def. 2 basis matrix (M, H) by the Cox-de Boor recursion (Eq. 4)."""
    Bm = np.empty((M, H), np.float64)
    _load().or_bspline_basis(M, p, H, TIME_MAPPING.get(mapping, mapping), _dp(Bm))
    return Bm


def akima_knot(M, mapping, i) -> float:
    return float(_load().or_akima_knot(M, TIME_MAPPING.get(mapping, mapping), i))


def akima_time(H, mapping, j) -> float:
    return float(_load().or_akima_time(H, TIME_MAPPING.get(mapping, mapping), j))


def akima_coeffs(tk, z) -> np.ndarray:
    """Eqs. 6-7: (M-1, 4) coefficients (a, b, c, d) for knots tk and values z."""
    tk = _f64(tk)
    z = _f64(z)
    M = tk.shape[0]
    coef = np.empty((M - 1, 4), np.float64)
    _load().or_akima_coeffs(M, _dp(tk), _dp(z), _dp(coef))
    return coef


def akima_eval(tk, coef, t: float) -> float:
    tk = _f64(tk)
    coef = _f64(coef)
    return float(_load().or_akima_eval(tk.shape[0], _dp(tk), _dp(coef), float(t)))


def bf16_round(x) -> np.ndarray:
    """bfloat16 rounding of each value (the oracle's definition, FP64 in/out)."""
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    lib = _load()
    return np.array([lib.or_bf16_round(float(v)) for v in x.ravel()]).reshape(x.shape)


def interpolate(spec, Cc, kind: str | None = None) -> np.ndarray:
    pr = _pr(spec)
    Cc = _f64(Cc)
    P = Cc.shape[0]
    U = np.empty((P, pr.H, pr.n), np.float64)
    lib = _load()
    fn = {None: lib.or_interpolate, "bspline": lib.or_interp_bspline,
          "akima": lib.or_interp_akima, "linear": lib.or_interp_linear}[kind]
    fn(C.byref(pr), _dp(Cc), P, _dp(U))
    return U


def standard_normal(seed: int, it: int, b: int, e: int) -> float:
    return float(_load().or_standard_normal(seed, it, b, e))


def local_samples(spec, it: int, mu, sigma, L: int | None = None) -> np.ndarray:
    pr = _pr(spec)
    L = pr.B - pr.P - 1 if L is None else L
    mu = _f64(mu, (pr.H, pr.n))
    sigma = _f64(sigma, (pr.H, pr.n))
    UL = np.empty((max(L, 0), pr.H, pr.n), np.float64)
    _load().or_local_samples(C.byref(pr), it, _dp(mu), _dp(sigma), L, _dp(UL))
    return UL


def stack_clamp(spec, UL, UG, mu) -> np.ndarray:
    pr = _pr(spec)
    UL = _f64(UL)
    UG = _f64(UG)
    mu = _f64(mu, (pr.H, pr.n))
    if UL.size == 0:
        UL = np.zeros((1, pr.H, pr.n))
    if UG.size == 0:
        UG = np.zeros((1, pr.H, pr.n))
    U = np.empty((pr.B, pr.H, pr.n), np.float64)
    _load().or_stack_clamp(C.byref(pr), _dp(UL), _dp(UG), _dp(mu), _dp(U))
    return U


def dr_scale(spec, it: int, unit: int, slot: int) -> float:
    pr = _pr(spec)
    return float(_load().or_dr_scale(C.byref(pr), it, unit, slot))


def chain_forward_dynamics(mass, length, g, q, qd, tau) -> np.ndarray:
    mass, length, q, qd, tau = (_f64(a) for a in (mass, length, q, qd, tau))
    nl = mass.shape[0]
    qdd = np.empty(nl, np.float64)
    rc = _load().or_chain_forward_dynamics(nl, _dp(mass), _dp(length), float(g), _dp(q),
                                           _dp(qd), _dp(tau), _dp(qdd))
    if rc != 0:
        raise FloatingPointError("mass matrix not positive definite")
    return qdd


def chain_energy(mass, length, g, q, qd) -> float:
    mass, length, q, qd = (_f64(a) for a in (mass, length, q, qd))
    return float(_load().or_chain_energy(mass.shape[0], _dp(mass), _dp(length), float(g),
                                         _dp(q), _dp(qd)))


def legged_forward_dynamics(spec, mass, mu_scale, q, qd, tau) -> np.ndarray:
    pr = _pr(spec)
    mass, q, qd, tau = (_f64(a) for a in (mass, q, qd, tau))
    qdd = np.empty(pr.n_links + 2, np.float64)
    rc = _load().or_legged_forward_dynamics(C.byref(pr), _dp(mass), float(mu_scale), _dp(q),
                                            _dp(qd), _dp(tau), _dp(qdd))
    if rc != 0:
        raise FloatingPointError("mass matrix not positive definite")
    return qdd


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def rollout_costs(spec, it: int, x0, U, row0: int = 0, threads: int = 1) -> np.ndarray:
    """Costs of candidates row0 .. row0+len(U)-1 (U holds only those rows);
    threads > 1 splits the candidates over that many host threads (same
    per-candidate arithmetic, so the same values)."""
    pr = _pr(spec)
    x0 = _f64(x0)
    U = _f64(U, (-1, pr.H, pr.n))
    cost = np.empty(U.shape[0], np.float64)
    if threads > 1:
        _load().or_rollout_costs_threads(C.byref(pr), it, _dp(x0), _dp(U), row0, U.shape[0],
                                         _dp(cost), int(threads))
    else:
        _load().or_rollout_costs(C.byref(pr), it, _dp(x0), _dp(U), row0, U.shape[0], _dp(cost))
    return cost


def rollout_states(spec, it: int, x0, Ub, b: int):
    pr = _pr(spec)
    x0 = _f64(x0)
    Ub = _f64(Ub, (pr.H, pr.n))
    X = np.empty((pr.H + 1, pr.d), np.float64)
    J = _load().or_rollout_states(C.byref(pr), it, _dp(x0), _dp(Ub), b, _dp(X))
    return X, float(J)


def top_e(cost, E: int) -> np.ndarray:
    cost = _f64(cost)
    if not 1 <= E <= cost.shape[0]:
        raise ValueError("top_e needs 1 <= E <= B")
    elite = np.empty(E, np.int32)
    _load().or_top_e(_dp(cost), cost.shape[0], E, _ip(elite))
    return elite


def softmax_weights(cost, elite, lam: float) -> np.ndarray:
    cost = _f64(cost)
    elite = np.ascontiguousarray(elite, dtype=np.int32)
    w = np.empty(elite.shape[0], np.float64)
    _load().or_softmax_weights(_dp(cost), _ip(elite), elite.shape[0], float(lam), _dp(w))
    return w


def elite_update(spec, U, cost, elite, mu, sigma):
    """Returns (mu_new, sigma_new, ustar); inputs are not modified."""
    pr = _pr(spec)
    U = _f64(U, (pr.B, pr.H, pr.n))
    cost = _f64(cost)
    elite = np.ascontiguousarray(elite, dtype=np.int32)
    mu = _f64(mu, (pr.H, pr.n)).copy()
    sigma = _f64(sigma, (pr.H, pr.n)).copy()
    ustar = np.empty(pr.n, np.float64)
    _load().or_elite_update(C.byref(pr), _dp(U), _dp(cost), _ip(elite), _dp(mu), _dp(sigma),
                            _dp(ustar))
    return mu, sigma, ustar


def shift(mu, sigma, k: int):
    mu = _f64(mu).copy()
    sigma = _f64(sigma).copy()
    H, n = mu.shape
    _load().or_shift(H, n, k, _dp(mu), _dp(sigma))
    return mu, sigma


def plan_iteration(spec, it: int, x0, mu, sigma, threads: int = 1):
    """One Alg. 2 iteration.  Returns dict(U, cost, elite, mu, sigma, ustar).
    threads > 1 rolls the candidates out on that many host threads."""
    pr = _pr(spec)
    x0 = _f64(x0)
    mu = _f64(mu, (pr.H, pr.n)).copy()
    sigma = _f64(sigma, (pr.H, pr.n)).copy()
    U = np.empty((pr.B, pr.H, pr.n), np.float64)
    cost = np.empty(pr.B, np.float64)
    elite = np.empty(pr.E, np.int32)
    ustar = np.empty(pr.n, np.float64)
    _load().or_plan_iteration_threads(C.byref(pr), it, _dp(x0), _dp(mu), _dp(sigma), _dp(U),
                                      _dp(cost), _ip(elite), _dp(ustar), int(threads))
    return {"U": U, "cost": cost, "elite": elite, "mu": mu, "sigma": sigma, "ustar": ustar}


def cost_entropy(cost, lam: float) -> float:
    cost = _f64(cost)
    return float(_load().or_cost_entropy(_dp(cost), cost.shape[0], float(lam)))


__all__ = [n for n in dir() if not n.startswith("_") and n not in ("annotations", "C", "np", "os",
                                                                  "subprocess", "threading")]

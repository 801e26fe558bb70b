"""Thin ctypes binding of libmtp.so (include/mtp.h), same names as the C ABI.

Only argument marshalling lives here: every step of the planner runs in the
library's CUDA kernels.  Device arrays are torch CUDA tensors (their
``data_ptr()`` is passed through), streams default to torch's current
stream.  If libmtp.so has not been built this module raises on first use;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmtp.so")

MAX_CTRL = 32
MAX_LINKS = 16
MAX_OBS = 8

MTP_OK = 0
STATUS = {0: "MTP_OK", 1: "MTP_ERR_INVALID_ARG", 2: "MTP_ERR_OUT_OF_MEMORY", 3: "MTP_ERR_CUDA",
          4: "MTP_ERR_ADMISSION", 5: "MTP_ERR_TIMEOUT", 6: "MTP_ERR_NOT_READY",
          7: "MTP_ERR_UNSUPPORTED"}
DYN = {"pointmass": 0, "chain": 1, "legged": 2}
INTERP = {"linear": 0, "bspline": 1, "akima": 2}
TIME_MAPPING = {"valid_span": 0, "paper_literal": 1}
UPDATE = {"softmax": 0, "plain_cem": 1}
DR = {"none": 0, "per_sample": 1, "shared": 2}
FLAG_NO_KAHAN = 0x1
FLAG_NO_GRAPH = 0x2
FLAG_COST_ENTROPY = 0x10
FLAG_BF16_BASIS = 0x4
FLAG_NO_PIPELINE = 0x8

# every function include/mtp.h declares
EXPORTS = [
    "mtp_problem_bytes", "mtp_create", "mtp_destroy", "mtp_last_error", "mtp_get_sizes",
    "mtp_get_buffers", "mtp_sample_tensor", "mtp_interpolate", "mtp_sample_local",
    "mtp_generate_candidates", "mtp_rollout_cost", "mtp_rollout_states", "mtp_elite_update",
    "mtp_plan_step", "mtp_plan_step_host", "mtp_shift", "mtp_get_state", "mtp_set_state",
    "mtp_set_profiling", "mtp_stage_times", "mtp_stage_times5", "mtp_elite_update_noalloc",
    "mtp_batch_create", "mtp_batch_destroy", "mtp_batch_layout", "mtp_batch_plan_step",
    "mtp_batch_autotune", "mtp_batch_reserve", "mtp_batch_fill", "mtp_batch_shift",
    "mtp_batch_launches", "mtp_batch_rollout_times", "mtp_batch_set_rollout_mode",
    "mtp_batch_rollout_mode", "mtp_batch_persistent_time", "mtp_device_status", "mtp_cost_entropy",
    "mtp_selftest_bounded_wait",
    "mtp_problem_device_bytes", "mtp_server_create", "mtp_server_destroy", "mtp_server_register",
    "mtp_submit", "mtp_poll", "mtp_server_get_stats", "mtp_server_last_error",
    "mtp_submit_many", "mtp_poll_many",
]


class MtpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MtpProblem(C.Structure):
    _fields_ = [
        ("dyn", C.c_int32), ("ctrl_dim", C.c_int32), ("state_dim", C.c_int32),
        ("horizon", C.c_int32), ("dt", C.c_float),
        ("u_min", C.c_float * MAX_CTRL), ("u_max", C.c_float * MAX_CTRL),
        ("M", C.c_int32), ("N", C.c_int32), ("B", C.c_int32), ("E", C.c_int32),
        ("beta", C.c_double), ("lam", C.c_double), ("alpha", C.c_double),
        ("sigma_min", C.c_double), ("mu_init", C.c_double), ("sigma_init", C.c_double),
        ("interp", C.c_int32), ("bspline_degree", C.c_int32), ("time_mapping", C.c_int32),
        ("update_rule", C.c_int32), ("dr_mode", C.c_int32), ("R", C.c_int32),
        ("dr_lo", C.c_float), ("dr_hi", C.c_float), ("seed", C.c_uint64),
        ("target", C.c_float * MAX_CTRL),
        ("w_target", C.c_float), ("w_obs", C.c_float), ("w_ctrl", C.c_float),
        ("w_term", C.c_float),
        ("n_obstacles", C.c_int32),
        ("obs_center", (C.c_float * MAX_CTRL) * MAX_OBS),
        ("obs_radius", C.c_float * MAX_OBS),
        ("n_links", C.c_int32),
        ("link_mass", C.c_float * MAX_LINKS), ("link_length", C.c_float * MAX_LINKS),
        ("gravity", C.c_float), ("k_contact", C.c_float), ("c_contact", C.c_float),
        ("mu_friction", C.c_float), ("v_slip", C.c_float),
        ("w_height", C.c_float), ("w_pitch", C.c_float), ("w_vel", C.c_float),
        ("flags", C.c_uint32),
    ]


class MtpSizes(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("B", "P", "L", "E", "H", "n", "d", "M", "N",
                                         "kernels_per_iteration", "pipelined")]


class MtpBuffers(C.Structure):
    _fields_ = [("U", C.c_void_p), ("cost", C.c_void_p), ("elite", C.c_void_p),
                ("weight", C.c_void_p), ("mu", C.c_void_p), ("sigma", C.c_void_p),
                ("ustar", C.c_void_p), ("iter", C.c_void_p)]


class MtpServerConfig(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("iters_per_request", C.c_int32),
                ("shift_after", C.c_int32), ("max_queue", C.c_int32), ("max_robots", C.c_int32),
                ("memory_budget", C.c_uint64)]


class MtpServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("cycles", C.c_uint64),
                ("planned", C.c_uint64), ("queued", C.c_int32), ("in_flight", C.c_int32),
                ("robots", C.c_int32), ("failed", C.c_int32), ("bytes_admitted", C.c_uint64),
                ("p50_latency_s", C.c_double), ("p99_latency_s", C.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmtp.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(nvcc, sm_103a); there is no CPU fallback")
    lib = C.CDLL(path)
    vp, i32, u32 = C.c_void_p, C.c_int32, C.c_uint32
    sig = {
        "mtp_problem_bytes": (C.c_size_t, []),
        "mtp_create": (i32, [C.POINTER(MtpProblem), C.POINTER(vp)]),
        "mtp_destroy": (i32, [vp]),
        "mtp_last_error": (C.c_char_p, [vp]),
        "mtp_get_sizes": (i32, [vp, C.POINTER(MtpSizes)]),
        "mtp_get_buffers": (i32, [vp, C.POINTER(MtpBuffers)]),
        "mtp_sample_tensor": (i32, [vp, u32, vp, vp, vp, vp]),
        "mtp_interpolate": (i32, [vp, vp, i32, vp, vp]),
        "mtp_sample_local": (i32, [vp, u32, vp, vp]),
        "mtp_generate_candidates": (i32, [vp, u32, vp, vp]),
        "mtp_rollout_cost": (i32, [vp, u32, vp, vp, i32, i32, vp, vp]),
        "mtp_rollout_states": (i32, [vp, u32, vp, vp, i32, vp, vp, vp]),
        "mtp_elite_update": (i32, [vp, vp, vp, vp, vp, vp]),
        "mtp_plan_step": (i32, [vp, vp, i32, vp, vp]),
        "mtp_plan_step_host": (i32, [vp, vp, i32, vp, vp]),
        "mtp_shift": (i32, [vp, i32, vp]),
        "mtp_get_state": (i32, [vp, vp, vp, vp]),
        "mtp_device_status": (i32, [vp]),
        "mtp_selftest_bounded_wait": (i32, [C.c_double, vp]),
        "mtp_cost_entropy": (i32, [vp, vp]),
        "mtp_set_state": (i32, [vp, vp, vp, u32]),
        "mtp_set_profiling": (i32, [vp, i32]),
        "mtp_stage_times": (i32, [vp, vp, vp]),
        "mtp_stage_times5": (i32, [vp, vp, vp]),
        "mtp_elite_update_noalloc": (i32, [vp, vp, i32, i32, i32, i32, C.c_double, C.c_double,
                                           C.c_double, i32, vp, vp, vp, vp, vp]),
        "mtp_batch_create": (i32, [C.POINTER(vp), i32, C.POINTER(vp)]),
        "mtp_batch_destroy": (i32, [vp]),
        "mtp_batch_layout": (i32, [vp, vp, vp]),
        "mtp_batch_plan_step": (i32, [vp, vp, i32, vp, vp]),
        "mtp_batch_autotune": (i32, [vp, vp, vp, vp]),
        "mtp_batch_launches": (i32, [vp, i32, vp]),
        "mtp_batch_set_rollout_mode": (i32, [vp, i32]),
        "mtp_batch_rollout_mode": (i32, [vp, vp, vp]),
        "mtp_batch_persistent_time": (i32, [vp, i32, vp, vp, vp]),
        "mtp_batch_rollout_times": (i32, [vp, i32, vp, vp, i32, vp, vp]),
        "mtp_batch_reserve": (i32, [i32, C.POINTER(vp)]),
        "mtp_batch_fill": (i32, [vp, C.POINTER(vp), i32, vp]),
        "mtp_batch_shift": (i32, [vp, i32, vp]),
        "mtp_problem_device_bytes": (i32, [C.POINTER(MtpProblem), C.POINTER(C.c_uint64)]),
        "mtp_server_create": (i32, [C.POINTER(MtpServerConfig), C.POINTER(vp)]),
        "mtp_server_destroy": (i32, [vp]),
        "mtp_server_register": (i32, [vp, C.POINTER(MtpProblem), C.POINTER(i32)]),
        "mtp_submit": (i32, [vp, i32, vp, C.POINTER(C.c_uint64)]),
        "mtp_poll": (i32, [vp, C.c_uint64, vp, C.c_double]),
        "mtp_server_get_stats": (i32, [vp, C.POINTER(MtpServerStats)]),
        "mtp_server_last_error": (C.c_char_p, [vp]),
        "mtp_submit_many": (i32, [vp, i32, vp, vp, vp, vp]),
        "mtp_poll_many": (i32, [vp, i32, vp, vp, i32, C.c_double, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.mtp_problem_bytes() != C.sizeof(MtpProblem):
        raise RuntimeError("mtp_problem layout mismatch between libmtp.so and the binding")
    _lib = lib
    return lib


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------

def problem_from_spec(spec: dict) -> MtpProblem:
    """Fill the C struct from a workload dict (see ``workloads``)."""
    p = MtpProblem()
    p.dyn = DYN[spec["dyn"]]
    p.ctrl_dim = spec["n"]
    p.state_dim = spec["d"]
    p.horizon = spec["H"]
    p.dt = spec["dt"]
    for i in range(spec["n"]):
        p.u_min[i] = spec["u_min"][i]
        p.u_max[i] = spec["u_max"][i]
    p.M, p.N, p.B, p.E = spec["M"], spec["N"], spec["B"], spec["E"]
    p.beta = spec["beta"]
    p.lam = spec["lambda"]
    p.alpha = spec["alpha"]
    p.sigma_min = spec["sigma_min"]
    p.mu_init = spec.get("mu_init", 0.0)
    p.sigma_init = spec["sigma_init"]
    p.interp = INTERP[spec["interp"]]
    p.bspline_degree = spec.get("degree", 2)
    p.time_mapping = TIME_MAPPING[spec.get("time_mapping", "valid_span")]
    p.update_rule = UPDATE[spec.get("update_rule", "softmax")]
    p.dr_mode = DR[spec.get("dr_mode", "none")]
    p.R = spec.get("R", 1)
    p.dr_lo = spec.get("dr_lo", 1.0)
    p.dr_hi = spec.get("dr_hi", 1.0)
    p.seed = spec["seed"]
    for i, v in enumerate(spec.get("target", [])):
        p.target[i] = v
    p.w_target = spec.get("w_target", 1.0)
    p.w_obs = spec.get("w_obs", 0.0)
    p.w_ctrl = spec.get("w_ctrl", 0.0)
    p.w_term = spec.get("w_term", 1.0)
    obs_c = spec.get("obs_c", [])
    p.n_obstacles = len(obs_c)
    for o, (c, r) in enumerate(zip(obs_c, spec.get("obs_r", []))):
        for a, v in enumerate(c):
            p.obs_center[o][a] = v
        p.obs_radius[o] = r
    p.n_links = spec.get("n_links", 0)
    for j, v in enumerate(spec.get("mass", [])):
        p.link_mass[j] = v
    for j, v in enumerate(spec.get("length", [])):
        p.link_length[j] = v
    p.gravity = spec.get("gravity", 9.81)
    p.k_contact = spec.get("k_contact", 0.0)
    p.c_contact = spec.get("c_contact", 0.0)
    p.mu_friction = spec.get("mu_friction", 0.0)
    p.v_slip = spec.get("v_slip", 0.01)
    p.w_height = spec.get("w_height", 0.0)
    p.w_pitch = spec.get("w_pitch", 0.0)
    p.w_vel = spec.get("w_vel", 0.0)
    p.flags = spec.get("flags", 0)
    return p


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t, dtype=None, numel: int | None = None, name: str = "tensor"):
    """Device pointer of a contiguous CUDA tensor (or 0 for None)."""
    if t is None:
        return None
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, needs {numel}")
    return t.data_ptr()


def _check(status: int, handle=None):
    if status != MTP_OK:
        lib = load_library()
        msg = lib.mtp_last_error(handle)
        raise MtpError(status, msg.decode() if msg else "")


class DeviceArray:
    """A handle-owned device buffer exposed through __cuda_array_interface__
    (wrap it with torch.as_tensor(x, device='cuda') for a zero-copy view)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


class Handle:
    """An mtp_handle* plus its sizes; destroyed with mtp_destroy (or on GC)."""

    def __init__(self, ptr: int, spec: dict):
        self.ptr = C.c_void_p(ptr)
        self.spec = spec
        s = MtpSizes()
        _check(load_library().mtp_get_sizes(self.ptr, C.byref(s)), self.ptr)
        self.sizes = {k: getattr(s, k) for k, _ in MtpSizes._fields_}

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            try:
                load_library().mtp_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = C.c_void_p(0)


# ----------------------------------------------------------------------------
# the ABI, one wrapper per entry point
# ----------------------------------------------------------------------------

def mtp_create(spec_or_problem) -> Handle:
    lib = load_library()
    prob = spec_or_problem if isinstance(spec_or_problem, MtpProblem) else problem_from_spec(spec_or_problem)
    out = C.c_void_p()
    st = lib.mtp_create(C.byref(prob), C.byref(out))
    if st != MTP_OK:
        raise MtpError(st, lib.mtp_last_error(None).decode())
    return Handle(out.value, spec_or_problem if isinstance(spec_or_problem, dict) else {})


def mtp_destroy(h: Handle):
    if h.ptr.value:
        _check(load_library().mtp_destroy(h.ptr))
        h.ptr = C.c_void_p(0)


def mtp_get_buffers(h: Handle) -> dict:
    b = MtpBuffers()
    _check(load_library().mtp_get_buffers(h.ptr, C.byref(b)), h.ptr)
    s = h.sizes
    return {
        "U": DeviceArray(b.U, (s["B"], s["H"], s["n"]), "<f4"),
        "cost": DeviceArray(b.cost, (s["B"],), "<f4"),
        "elite": DeviceArray(b.elite, (s["E"],), "<i4"),
        "weight": DeviceArray(b.weight, (s["E"],), "<f8"),
        "mu": DeviceArray(b.mu, (s["H"], s["n"]), "<f8"),
        "sigma": DeviceArray(b.sigma, (s["H"], s["n"]), "<f8"),
        "ustar": DeviceArray(b.ustar, (s["n"],), "<f4"),
        "iter": DeviceArray(b.iter, (1,), "<u4"),
    }


def _f32():
    import torch
    return torch.float32


def _i32():
    import torch
    return torch.int32


def mtp_sample_tensor(h: Handle, it: int, Z=None, idx=None, Cw=None, stream=None):
    s = h.sizes
    _check(load_library().mtp_sample_tensor(
        h.ptr, it, _dptr(Z, _f32(), s["M"] * s["N"] * s["n"], "Z"),
        _dptr(idx, _i32(), s["P"] * s["M"], "idx"),
        _dptr(Cw, _f32(), s["P"] * s["M"] * s["n"], "C"), _stream(stream)), h.ptr)


def mtp_interpolate(h: Handle, Cw, U, stream=None):
    s = h.sizes
    P = Cw.shape[0]
    _check(load_library().mtp_interpolate(
        h.ptr, _dptr(Cw, _f32(), P * s["M"] * s["n"], "C"), P,
        _dptr(U, _f32(), P * s["H"] * s["n"], "U"), _stream(stream)), h.ptr)


def mtp_sample_local(h: Handle, it: int, U, stream=None):
    s = h.sizes
    _check(load_library().mtp_sample_local(
        h.ptr, it, _dptr(U, _f32(), s["B"] * s["H"] * s["n"], "U"), _stream(stream)), h.ptr)


def mtp_generate_candidates(h: Handle, it: int, U, stream=None):
    s = h.sizes
    _check(load_library().mtp_generate_candidates(
        h.ptr, it, _dptr(U, _f32(), s["B"] * s["H"] * s["n"], "U"), _stream(stream)), h.ptr)


def mtp_rollout_cost(h: Handle, it: int, x0, U, cost, row0: int = 0, rows: int | None = None,
                     stream=None):
    s = h.sizes
    rows = U.shape[0] if rows is None else rows
    _check(load_library().mtp_rollout_cost(
        h.ptr, it, _dptr(x0, _f32(), s["d"], "x0"),
        _dptr(U, _f32(), rows * s["H"] * s["n"], "U"), row0, rows,
        _dptr(cost, _f32(), rows, "cost"), _stream(stream)), h.ptr)


def mtp_rollout_states(h: Handle, it: int, x0, Urow, row: int, X, cost, stream=None):
    s = h.sizes
    _check(load_library().mtp_rollout_states(
        h.ptr, it, _dptr(x0, _f32(), s["d"], "x0"), _dptr(Urow, _f32(), s["H"] * s["n"], "U"),
        row, _dptr(X, _f32(), (s["H"] + 1) * s["d"], "X"), _dptr(cost, _f32(), 1, "cost"),
        _stream(stream)), h.ptr)


def mtp_elite_update(h: Handle, cost, U, elite=None, ustar=None, stream=None):
    s = h.sizes
    _check(load_library().mtp_elite_update(
        h.ptr, _dptr(cost, _f32(), s["B"], "cost"), _dptr(U, _f32(), s["B"] * s["H"] * s["n"], "U"),
        _dptr(elite, _i32(), s["E"], "elite"), _dptr(ustar, _f32(), s["n"], "ustar"),
        _stream(stream)), h.ptr)


def mtp_plan_step(h: Handle, x0, iters: int, ustar, stream=None):
    s = h.sizes
    _check(load_library().mtp_plan_step(
        h.ptr, _dptr(x0, _f32(), s["d"], "x0"), iters, _dptr(ustar, _f32(), s["n"], "ustar"),
        _stream(stream)), h.ptr)


def mtp_plan_step_host(h: Handle, x0: np.ndarray, iters: int, ustar: np.ndarray, stream=None):
    """x0 / ustar are float32 host arrays (numpy, or pinned torch CPU tensors)."""
    s = h.sizes

    def hptr(a, n, name):
        if hasattr(a, "data_ptr"):
            if a.is_cuda or a.dtype != _f32() or not a.is_contiguous() or a.numel() < n:
                raise ValueError(f"{name}: need a contiguous float32 host tensor of {n}")
            return a.data_ptr()
        if a.dtype != np.float32 or not a.flags.c_contiguous or a.size < n:
            raise ValueError(f"{name}: need a contiguous float32 array of {n}")
        return a.ctypes.data

    _check(load_library().mtp_plan_step_host(h.ptr, hptr(x0, s["d"], "x0"), iters,
                                             hptr(ustar, s["n"], "ustar"), _stream(stream)), h.ptr)


def mtp_shift(h: Handle, k: int, stream=None):
    _check(load_library().mtp_shift(h.ptr, k, _stream(stream)), h.ptr)


def mtp_cost_entropy(h: Handle) -> float:
    """Sec. 4.1 cost entropy of the latest selection (problems created with
    FLAG_COST_ENTROPY)."""
    v = C.c_double()
    _check(load_library().mtp_cost_entropy(h.ptr, C.addressof(v)), h.ptr)
    return float(v.value)


def mtp_selftest_bounded_wait(limit_s: float):
    """Runs the bounded-wait self-test; returns (status, host-measured seconds).
    A working library gives MTP_ERR_TIMEOUT (5) after about limit_s."""
    waited = C.c_double()
    st = load_library().mtp_selftest_bounded_wait(float(limit_s), C.addressof(waited))
    return int(st), float(waited.value)


def mtp_device_status(h: Handle):
    """Raises MtpError (MTP_ERR_TIMEOUT) if a bounded device wait of the
    handle's rollouts gave up since the last check; synchronises."""
    _check(load_library().mtp_device_status(h.ptr), h.ptr)


def mtp_get_state(h: Handle):
    s = h.sizes
    mu = np.empty((s["H"], s["n"]), np.float64)
    sg = np.empty((s["H"], s["n"]), np.float64)
    it = C.c_uint32()
    _check(load_library().mtp_get_state(h.ptr, mu.ctypes.data, sg.ctypes.data, C.addressof(it)),
           h.ptr)
    return mu, sg, int(it.value)


def mtp_set_state(h: Handle, mu, sigma, it: int):
    s = h.sizes
    mu = np.ascontiguousarray(mu, np.float64).reshape(s["H"], s["n"])
    sg = np.ascontiguousarray(sigma, np.float64).reshape(s["H"], s["n"])
    _check(load_library().mtp_set_state(h.ptr, mu.ctypes.data, sg.ctypes.data, it), h.ptr)


def mtp_set_profiling(h: Handle, enable: bool):
    _check(load_library().mtp_set_profiling(h.ptr, 1 if enable else 0), h.ptr)


def mtp_stage_times(h: Handle):
    """(ms per stage [generate, rollout, select, update], iterations)."""
    ms = (C.c_double * 4)()
    n = C.c_int32()
    _check(load_library().mtp_stage_times(h.ptr, C.addressof(ms), C.addressof(n)), h.ptr)
    return [float(v) for v in ms], int(n.value)


def mtp_stage_times5(h: Handle):
    """(ms per stage [generate, rollout, select, update, prepare], iterations);
    "prepare" is the next iteration's generation that a pipelined handle runs
    on a second stream during the rollout."""
    ms = (C.c_double * 5)()
    n = C.c_int32()
    _check(load_library().mtp_stage_times5(h.ptr, C.addressof(ms), C.addressof(n)), h.ptr)
    return [float(v) for v in ms], int(n.value)


def mtp_elite_update_noalloc(cost, U, E: int, lam: float, alpha: float, sigma_min: float,
                             update_rule: str, mu, sigma, elite=None, ustar=None, stream=None):
    """The handle-free elite update: cost (B), U (B, H, n) float32; mu, sigma
    (H, n) float64 CUDA tensors updated in place; elite (E) int32 and ustar
    (n) float32 optional outputs.  Allocates nothing.  The library runs the
    call on the current CUDA device, so every tensor must live there."""
    import torch
    B, H, n = U.shape
    dev = torch.cuda.current_device()
    for name, t in (("cost", cost), ("U", U), ("mu", mu), ("sigma", sigma), ("elite", elite),
                    ("ustar", ustar)):
        if t is not None and getattr(t, "is_cuda", False) and t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, but the current device is "
                             f"cuda:{dev}")
    _check(load_library().mtp_elite_update_noalloc(
        _dptr(cost, _f32(), B, "cost"), _dptr(U, _f32(), B * H * n, "U"), B, E, H, n,
        float(lam), float(alpha), float(sigma_min), UPDATE[update_rule],
        _dptr(mu, torch.float64, H * n, "mu"), _dptr(sigma, torch.float64, H * n, "sigma"),
        _dptr(elite, _i32(), E, "elite"), _dptr(ustar, _f32(), n, "ustar"), _stream(stream)))


class Batch:
    """An mtp_batch* over handles (kept alive here) and its packed layout."""

    def __init__(self, ptr: int, handles):
        self.ptr = C.c_void_p(ptr)
        self.handles = []
        self.x0_offset = [0]
        self.ustar_offset = [0]
        if handles:
            self._set(handles)

    def _set(self, handles):
        self.handles = list(handles)
        n = len(self.handles) + 1
        x0 = (C.c_int32 * n)()
        us = (C.c_int32 * n)()
        _check(load_library().mtp_batch_layout(self.ptr, C.addressof(x0), C.addressof(us)))
        self.x0_offset = list(x0)
        self.ustar_offset = list(us)

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            try:
                load_library().mtp_batch_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = C.c_void_p(0)


def _handle_array(handles):
    return (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])


def mtp_batch_create(handles) -> Batch:
    lib = load_library()
    out = C.c_void_p()
    st = lib.mtp_batch_create(_handle_array(handles), len(handles), C.byref(out))
    if st != MTP_OK:
        raise MtpError(st, lib.mtp_last_error(None).decode())
    return Batch(out.value, handles)


def mtp_batch_reserve(capacity: int) -> Batch:
    lib = load_library()
    out = C.c_void_p()
    st = lib.mtp_batch_reserve(int(capacity), C.byref(out))
    if st != MTP_OK:
        raise MtpError(st, lib.mtp_last_error(None).decode())
    return Batch(out.value, [])


def mtp_batch_fill(b: Batch, handles, stream=None):
    lib = load_library()
    st = lib.mtp_batch_fill(b.ptr, _handle_array(handles), len(handles), _stream(stream))
    if st != MTP_OK:
        raise MtpError(st, lib.mtp_last_error(None).decode())
    b._set(handles)


def mtp_batch_shift(b: Batch, k: int, stream=None):
    st = load_library().mtp_batch_shift(b.ptr, int(k), _stream(stream))
    if st != MTP_OK:
        raise MtpError(st, load_library().mtp_last_error(None).decode())


def mtp_problem_device_bytes(spec_or_problem) -> int:
    lib = load_library()
    pr = spec_or_problem if isinstance(spec_or_problem, MtpProblem) else problem_from_spec(spec_or_problem)
    out = C.c_uint64()
    st = lib.mtp_problem_device_bytes(C.byref(pr), C.byref(out))
    if st != MTP_OK:
        raise MtpError(st, lib.mtp_last_error(None).decode())
    return out.value


def mtp_batch_destroy(b: Batch):
    if b.ptr.value:
        _check(load_library().mtp_batch_destroy(b.ptr))
        b.ptr = C.c_void_p(0)


def mtp_batch_plan_step(b: Batch, x0, iters: int, ustar, stream=None):
    _check(load_library().mtp_batch_plan_step(
        b.ptr, _dptr(x0, _f32(), b.x0_offset[-1], "x0"), iters,
        _dptr(ustar, _f32(), b.ustar_offset[-1], "ustar"), _stream(stream)))


def mtp_batch_autotune(b: Batch, stream=None):
    """Returns [(dyn, dim, block, chunk, samples_per_thread), ...] per rollout group."""
    groups = len(b.handles)
    out = (C.c_int32 * (5 * groups))()
    ng = C.c_int32()
    _check(load_library().mtp_batch_autotune(b.ptr, C.addressof(out), C.addressof(ng),
                                             _stream(stream)))
    return [tuple(out[5 * i + k] for k in range(5)) for i in range(ng.value)]


# how a batch runs its rollouts (mtp_batch_set_rollout_mode)
BATCH_ROLLOUT_GROUPS = 0
BATCH_ROLLOUT_PERSISTENT_STAGED = 1
BATCH_ROLLOUT_PERSISTENT_DIRECT = 2
BATCH_ROLLOUT_PERSISTENT_SPLIT = 3
BATCH_ROLLOUT_NAMES = {0: "groups", 1: "persistent, staged", 2: "persistent, direct",
                       3: "persistent, two launches"}


def mtp_batch_set_rollout_mode(b: Batch, mode: int) -> None:
    _check(load_library().mtp_batch_set_rollout_mode(b.ptr, int(mode)))


def mtp_batch_rollout_mode(b: Batch):
    """(mode, [the autotuner's iteration ms per mode, 0 where not timed])."""
    mode = C.c_int32()
    ms = (C.c_double * 4)()
    _check(load_library().mtp_batch_rollout_mode(b.ptr, C.addressof(mode), C.addressof(ms)))
    return int(mode.value), [float(v) for v in ms]


def mtp_batch_persistent_time(b: Batch, reps: int = 5, stream=None):
    """(ms, rollout steps) of the persistent rollout launch timed alone."""
    ms = C.c_double()
    steps = C.c_int64()
    _check(load_library().mtp_batch_persistent_time(b.ptr, int(reps), C.addressof(ms),
                                                    C.addressof(steps), _stream(stream)))
    return float(ms.value), int(steps.value)


def mtp_batch_launches(b: Batch, iters: int = 1) -> int:
    """Kernel launches of one mtp_batch_plan_step(b, ..., iters, ...)."""
    n = C.c_int32()
    _check(load_library().mtp_batch_launches(b.ptr, int(iters), C.addressof(n)))
    return int(n.value)


def mtp_batch_rollout_times(b: Batch, reps: int = 3, stream=None):
    """Each group's rollout launch timed alone: a list of dicts with dyn,
    dim, block, instances, candidates, steps and ms (average device time)."""
    groups = max(1, len(b.handles))
    ms = (C.c_double * groups)()
    info = (C.c_int32 * (8 * groups))()
    ng = C.c_int32()
    _check(load_library().mtp_batch_rollout_times(b.ptr, int(reps), C.addressof(ms),
                                                  C.addressof(info), groups, C.addressof(ng),
                                                  _stream(stream)))
    keys = ("dyn", "dim", "block", "instances", "candidates", "steps", "chunk", "samples")
    return [dict(zip(keys, (int(info[8 * g + k]) for k in range(8))), ms=float(ms[g]))
            for g in range(ng.value)]


# ----------------------------------------------------------------------------
# re-plan server
# ----------------------------------------------------------------------------

class Server:
    """An mtp_server*: robots registered with their problems, requests
    submitted with host start states, results polled by ticket."""

    def __init__(self, ptr: int):
        self.ptr = C.c_void_p(ptr)

    def _err(self):
        return load_library().mtp_server_last_error(self.ptr).decode()

    def close(self):
        if self.ptr.value:
            _check(load_library().mtp_server_destroy(self.ptr))
            self.ptr = C.c_void_p(0)

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            try:
                load_library().mtp_server_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = C.c_void_p(0)


def mtp_server_create(max_batch: int = 64, iters_per_request: int = 1, shift_after: int = 1,
                      max_queue: int = 4, max_robots: int = 1024, memory_budget: int = 0) -> Server:
    lib = load_library()
    cfg = MtpServerConfig(int(max_batch), int(iters_per_request), int(shift_after), int(max_queue),
                          int(max_robots), int(memory_budget))
    out = C.c_void_p()
    st = lib.mtp_server_create(C.byref(cfg), C.byref(out))
    if st != MTP_OK:
        raise MtpError(st, lib.mtp_last_error(None).decode())
    return Server(out.value)


def mtp_server_destroy(srv: Server):
    srv.close()


def mtp_server_register(srv: Server, spec_or_problem) -> int:
    pr = spec_or_problem if isinstance(spec_or_problem, MtpProblem) else problem_from_spec(spec_or_problem)
    rid = C.c_int32()
    st = load_library().mtp_server_register(srv.ptr, C.byref(pr), C.byref(rid))
    if st != MTP_OK:
        raise MtpError(st, srv._err())
    return rid.value


def mtp_submit(srv: Server, robot: int, x0: np.ndarray) -> int:
    x = np.ascontiguousarray(x0, dtype=np.float32)
    t = C.c_uint64()
    st = load_library().mtp_submit(srv.ptr, int(robot), x.ctypes.data, C.byref(t))
    if st != MTP_OK:
        raise MtpError(st, srv._err())
    return t.value


def mtp_poll(srv: Server, ticket: int, out: np.ndarray, timeout_s: float = 0.0) -> int:
    """Returns the status: MTP_OK (u* in `out`), NOT_READY (6) or TIMEOUT (5);
    raises for the other errors."""
    assert out.dtype == np.float32 and out.flags.c_contiguous
    st = load_library().mtp_poll(srv.ptr, C.c_uint64(int(ticket)), out.ctypes.data, float(timeout_s))
    if st not in (MTP_OK, 5, 6):
        raise MtpError(st, srv._err())
    return st


def mtp_server_get_stats(srv: Server) -> dict:
    s = MtpServerStats()
    _check(load_library().mtp_server_get_stats(srv.ptr, C.byref(s)))
    return {k: getattr(s, k) for k, _ in MtpServerStats._fields_}


def mtp_submit_many(srv: Server, robots: np.ndarray, x0_packed: np.ndarray) -> np.ndarray:
    """Queues one request per entry of `robots` (start states packed in
    order); returns the tickets.  Raises on the first refusal, after the
    requests before it were queued (their tickets are in the error's
    `tickets` attribute)."""
    r = np.ascontiguousarray(robots, dtype=np.int32)
    x = np.ascontiguousarray(x0_packed, dtype=np.float32)
    t = np.zeros(len(r), dtype=np.uint64)
    acc = C.c_int32()
    st = load_library().mtp_submit_many(srv.ptr, len(r), r.ctypes.data, x.ctypes.data,
                                        t.ctypes.data, C.byref(acc))
    if st != MTP_OK:
        err = MtpError(st, srv._err())
        err.tickets = t[:acc.value]
        raise err
    return t


def mtp_poll_many(srv: Server, tickets: np.ndarray, stride: int, timeout_s: float = 0.0):
    """Returns (status per ticket, u* rows (count, stride), number ready)."""
    t = np.ascontiguousarray(tickets, dtype=np.uint64)
    out = np.zeros((len(t), stride), dtype=np.float32)
    status = np.zeros(len(t), dtype=np.int32)
    ready = C.c_int32()
    _check(load_library().mtp_poll_many(srv.ptr, len(t), t.ctypes.data, out.ctypes.data, int(stride),
                                        float(timeout_s), status.ctypes.data, C.byref(ready)))
    return status, out, ready.value

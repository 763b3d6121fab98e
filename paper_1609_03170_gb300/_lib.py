"""ctypes binding of libgrape.so: the C ABI of include/grape.h, same names.

Argument marshalling only; every step of the propagation and of the gradient
runs in the library's CUDA kernels.  Loading fails loudly when the library is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32, c_double, c_void_p, c_size_t = ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
P = ctypes.POINTER

GRAPE_OK, GRAPE_EINVAL, GRAPE_ENOMEM, GRAPE_ECUDA, GRAPE_ETIMEOUT, GRAPE_EBUSY, \
    GRAPE_ENOTREADY, GRAPE_EINTERNAL = range(8)
GRAPE_GRAD_EXACT, GRAPE_GRAD_FIRST_ORDER = 0, 1
GRAPE_PREC_DF64, GRAPE_PREC_FP64 = 0, 1

STATUS_NAMES = {0: "GRAPE_OK", 1: "GRAPE_EINVAL", 2: "GRAPE_ENOMEM", 3: "GRAPE_ECUDA",
                4: "GRAPE_ETIMEOUT", 5: "GRAPE_EBUSY", 6: "GRAPE_ENOTREADY", 7: "GRAPE_EINTERNAL"}


class grape_band_op(ctypes.Structure):
    _fields_ = [("n_diag", c_int32), ("offsets", P(c_int32)), ("values", P(c_double))]


class grape_problem_desc(ctypes.Structure):
    _fields_ = [("d", c_int32), ("n_controls", c_int32), ("n_jumps", c_int32),
                ("n_states", c_int32), ("n_slices", c_int32), ("n_rk", c_int32),
                ("T", c_double),
                ("H0", grape_band_op), ("Hc", P(grape_band_op)), ("jumps", P(grape_band_op)),
                ("rates", P(c_double)), ("rho0", P(c_double)), ("sigma", P(c_double)),
                ("sigma_broadcast", c_int32), ("grad_mode", c_int32), ("ckpt_stride", c_int32),
                ("precision", c_int32), ("jump_control", P(c_int32))]


class grape_opt_params(ctypes.Structure):
    _fields_ = [("max_iters", c_int32), ("lbfgs_m", c_int32), ("u_min", c_double),
                ("u_max", c_double), ("step0", c_double), ("tol", c_double)]


class grape_job_info(ctypes.Structure):
    _fields_ = [("evaluations", c_int32), ("queued_us", c_double), ("latency_us", c_double)]


class GrapeError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

EXPORTS = ["grape_problem_create", "grape_problem_destroy", "grape_forward", "grape_gradient",
           "grape_filter_apply", "grape_filter_adjoint", "grape_gradient_filtered",
           "grape_problem_memory", "grape_problem_geometry", "grape_problem_set_tile",
           "grape_problem_set_penalty", "grape_set_profiling",
           "grape_phase_times", "grape_gradient_launches", "grape_gradient_static",
           "grape_batch_create", "grape_batch_destroy", "grape_batch_gradient", "grape_batch_info",
           "grape_problem_kernel", "grape_problem_status", "grape_server_create",
           "grape_server_destroy", "grape_submit", "grape_poll",
           "grape_fma_peak", "grape_last_error", "grape_version"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgrape.so (building it with nvcc when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libgrape.so not found at {path}; run paper_1609_03170_gb300.build")
    lib = ctypes.CDLL(path)
    lib.grape_problem_create.argtypes = [P(grape_problem_desc), P(c_void_p)]
    lib.grape_problem_create.restype = c_int32
    lib.grape_problem_destroy.argtypes = [c_void_p]
    lib.grape_problem_destroy.restype = c_int32
    lib.grape_forward.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.grape_forward.restype = c_int32
    lib.grape_gradient.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.grape_gradient.restype = c_int32
    for name in ("grape_filter_apply", "grape_filter_adjoint"):
        getattr(lib, name).argtypes = [c_int32, c_int32, c_int32, c_double, c_double, P(c_double),
                                       c_void_p, c_void_p, c_void_p]
        getattr(lib, name).restype = c_int32
    lib.grape_gradient_filtered.argtypes = [c_void_p, c_int32, P(c_double), c_void_p, c_void_p,
                                            c_void_p, c_void_p]
    lib.grape_gradient_filtered.restype = c_int32
    lib.grape_server_create.argtypes = [c_size_t, c_int32, P(c_void_p)]
    lib.grape_server_create.restype = c_int32
    lib.grape_server_destroy.argtypes = [c_void_p]
    lib.grape_server_destroy.restype = c_int32
    lib.grape_submit.argtypes = [c_void_p, c_void_p, P(c_double), P(grape_opt_params),
                                 P(ctypes.c_uint64)]
    lib.grape_submit.restype = c_int32
    lib.grape_poll.argtypes = [c_void_p, ctypes.c_uint64, ctypes.c_int64, P(c_double),
                               P(c_double), P(grape_job_info)]
    lib.grape_poll.restype = c_int32
    lib.grape_problem_kernel.argtypes = [c_void_p, P(c_int32)]
    lib.grape_problem_kernel.restype = c_int32
    lib.grape_problem_status.argtypes = [c_void_p]
    lib.grape_problem_status.restype = c_int32
    lib.grape_batch_create.argtypes = [P(c_void_p), c_int32, c_int32, P(c_void_p)]
    lib.grape_batch_create.restype = c_int32
    lib.grape_batch_destroy.argtypes = [c_void_p]
    lib.grape_batch_destroy.restype = c_int32
    lib.grape_batch_gradient.argtypes = [c_void_p, P(c_void_p), c_void_p, P(c_void_p), c_void_p]
    lib.grape_batch_gradient.restype = c_int32
    lib.grape_batch_info.argtypes = [c_void_p, P(c_int32), P(c_size_t), P(c_int32)]
    lib.grape_batch_info.restype = c_int32
    lib.grape_gradient_static.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.grape_gradient_static.restype = c_int32
    lib.grape_problem_memory.argtypes = [c_void_p, P(c_size_t)]
    lib.grape_problem_memory.restype = c_int32
    lib.grape_problem_geometry.argtypes = [c_void_p, P(c_int32), P(c_int32), P(c_int32)]
    lib.grape_problem_geometry.restype = c_int32
    lib.grape_problem_set_penalty.argtypes = [c_void_p, P(c_double), c_double]
    lib.grape_problem_set_penalty.restype = c_int32
    lib.grape_problem_set_tile.argtypes = [c_void_p, c_int32, c_int32]
    lib.grape_problem_set_tile.restype = c_int32
    lib.grape_set_profiling.argtypes = [c_void_p, c_int32]
    lib.grape_set_profiling.restype = c_int32
    lib.grape_phase_times.argtypes = [c_void_p, P(c_double), P(c_int32)]
    lib.grape_phase_times.restype = c_int32
    lib.grape_gradient_launches.argtypes = [c_void_p]
    lib.grape_gradient_launches.restype = c_int32
    lib.grape_last_error.argtypes = []
    lib.grape_last_error.restype = ctypes.c_char_p
    lib.grape_version.argtypes = []
    lib.grape_version.restype = ctypes.c_char_p
    lib.grape_fma_peak.argtypes = [c_int32, P(c_double), P(c_double)]
    lib.grape_fma_peak.restype = c_int32
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != GRAPE_OK:
        msg = load().grape_last_error().decode(errors="replace")
        raise GrapeError(status, where, msg)


def grape_problem_create(desc: grape_problem_desc) -> c_void_p:
    h = c_void_p()
    check(load().grape_problem_create(ctypes.byref(desc), ctypes.byref(h)), "grape_problem_create")
    return h


def grape_problem_destroy(h) -> None:
    check(load().grape_problem_destroy(h), "grape_problem_destroy")


def grape_forward(h, u_ptr: int, F_ptr: int, rhoT_ptr: int, stream_ptr: int) -> None:
    check(load().grape_forward(h, u_ptr or None, F_ptr or None, rhoT_ptr or None,
                               stream_ptr or None), "grape_forward")


def grape_gradient(h, u_ptr: int, F_ptr: int, grad_ptr: int, stream_ptr: int) -> None:
    check(load().grape_gradient(h, u_ptr or None, F_ptr or None, grad_ptr or None,
                                stream_ptr or None), "grape_gradient")


def _omega0(omega0, n):
    w = (c_double * n)()
    vals = list(omega0) if hasattr(omega0, "__len__") else [omega0] * n
    if len(vals) != n:
        raise ValueError(f"omega0 needs {n} values")
    for k, v in enumerate(vals):
        w[k] = float(v)
    return w


def grape_filter_apply(n_steps, n_sub, n_controls, Dt, dt, omega0, u_ptr, s_ptr, stream_ptr):
    check(load().grape_filter_apply(n_steps, n_sub, n_controls, Dt, dt, _omega0(omega0, n_controls),
                                    u_ptr or None, s_ptr or None, stream_ptr or None),
          "grape_filter_apply")


def grape_filter_adjoint(n_steps, n_sub, n_controls, Dt, dt, omega0, gs_ptr, gu_ptr, stream_ptr):
    check(load().grape_filter_adjoint(n_steps, n_sub, n_controls, Dt, dt, _omega0(omega0, n_controls),
                                      gs_ptr or None, gu_ptr or None, stream_ptr or None),
          "grape_filter_adjoint")


def grape_gradient_filtered(h, n_steps, n_controls, omega0, u_ptr, F_ptr, grad_ptr, stream_ptr):
    check(load().grape_gradient_filtered(h, n_steps, _omega0(omega0, n_controls), u_ptr or None,
                                         F_ptr or None, grad_ptr or None, stream_ptr or None),
          "grape_gradient_filtered")


def grape_gradient_static(h, u_ptr: int, F_ptr: int, grad_ptr: int, stream_ptr: int) -> None:
    """grape_gradient with every scratch buffer in the library's static device
    array (no device allocation); u, F and grad must be device pointers."""
    check(load().grape_gradient_static(h, u_ptr or None, F_ptr or None, grad_ptr or None,
                                       stream_ptr or None), "grape_gradient_static")


def grape_server_create(budget_bytes: int = 0, max_slots: int = 16):
    srv = c_void_p()
    check(load().grape_server_create(int(budget_bytes), int(max_slots), ctypes.byref(srv)),
          "grape_server_create")
    return srv


def grape_server_destroy(srv) -> None:
    check(load().grape_server_destroy(srv), "grape_server_destroy")


def grape_submit(srv, problem_handle, u0, params: grape_opt_params) -> int:
    t = ctypes.c_uint64()
    check(load().grape_submit(srv, problem_handle, u0.ctypes.data_as(P(c_double)),
                              ctypes.byref(params), ctypes.byref(t)), "grape_submit")
    return int(t.value)


def grape_poll(srv, ticket: int, timeout_us: int, u_out, F_out, info: grape_job_info) -> bool:
    """True when the job is done (results written), False while it runs."""
    st = load().grape_poll(srv, ctypes.c_uint64(ticket), ctypes.c_int64(int(timeout_us)),
                           u_out.ctypes.data_as(P(c_double)), F_out.ctypes.data_as(P(c_double)),
                           ctypes.byref(info))
    if st == GRAPE_ENOTREADY:
        return False
    check(st, "grape_poll")
    return True


KERNEL_NAMES = {0: "hermitian-cluster", 1: "full-cluster", 2: "grid"}


def grape_problem_kernel(h) -> str:
    k = c_int32()
    check(load().grape_problem_kernel(h, ctypes.byref(k)), "grape_problem_kernel")
    return KERNEL_NAMES[int(k.value)]


def grape_problem_status(h) -> None:
    check(load().grape_problem_status(h), "grape_problem_status")


def grape_batch_create(handles, n_lanes: int = 0):
    arr = (c_void_p * len(handles))(*[h.value if isinstance(h, c_void_p) else h for h in handles])
    b = c_void_p()
    check(load().grape_batch_create(arr, len(handles), int(n_lanes), ctypes.byref(b)),
          "grape_batch_create")
    return b


def grape_batch_destroy(b) -> None:
    check(load().grape_batch_destroy(b), "grape_batch_destroy")


def grape_batch_gradient(b, u_ptrs, F_ptr: int, grad_ptrs, stream_ptr: int) -> None:
    n = len(u_ptrs)
    ua = (c_void_p * n)(*u_ptrs)
    ga = (c_void_p * n)(*grad_ptrs)
    check(load().grape_batch_gradient(b, ua, F_ptr or None, ga, stream_ptr or None),
          "grape_batch_gradient")


def grape_batch_info(b):
    nl, by, la = c_int32(), c_size_t(), c_int32()
    check(load().grape_batch_info(b, ctypes.byref(nl), ctypes.byref(by), ctypes.byref(la)),
          "grape_batch_info")
    return int(nl.value), int(by.value), int(la.value)


def grape_problem_memory(h) -> int:
    n = c_size_t()
    check(load().grape_problem_memory(h, ctypes.byref(n)), "grape_problem_memory")
    return int(n.value)


def grape_problem_geometry(h):
    c, t, e = c_int32(), c_int32(), c_int32()
    check(load().grape_problem_geometry(h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(e)),
          "grape_problem_geometry")
    return int(c.value), int(t.value), int(e.value)


def grape_problem_set_penalty(h, diag, beta: float) -> None:
    if diag is None:
        check(load().grape_problem_set_penalty(h, None, 0.0), "grape_problem_set_penalty")
        return
    a = (c_double * len(diag))(*[float(x) for x in diag])
    check(load().grape_problem_set_penalty(h, a, float(beta)), "grape_problem_set_penalty")


def grape_problem_set_tile(h, cluster: int, threads: int) -> None:
    check(load().grape_problem_set_tile(h, int(cluster), int(threads)), "grape_problem_set_tile")


def grape_set_profiling(h, on: bool) -> None:
    check(load().grape_set_profiling(h, 1 if on else 0), "grape_set_profiling")


PHASES = ("forward", "cost", "adjoint", "trace")


def grape_phase_times(h):
    """{phase: (milliseconds, launches)} since the previous call."""
    ms = (c_double * 4)()
    n = (c_int32 * 4)()
    check(load().grape_phase_times(h, ms, n), "grape_phase_times")
    return {PHASES[i]: (float(ms[i]), int(n[i])) for i in range(4)}


def grape_gradient_launches(h) -> int:
    return int(load().grape_gradient_launches(h))


def grape_version() -> str:
    return load().grape_version().decode()


def grape_fma_peak(precision: int):
    """Measured FMA throughput of the current device: (TFLOP/s, ms of the
    timed run) of the FP32 pipes (GRAPE_PREC_DF64) or the FP64 pipe
    (GRAPE_PREC_FP64)."""
    t, ms = c_double(), c_double()
    check(load().grape_fma_peak(int(precision), ctypes.byref(t), ctypes.byref(ms)), "grape_fma_peak")
    return float(t.value), float(ms.value)

"""ctypes front end of grape_oracle.c (the plain-C FP64 oracle).

Test infrastructure only.  The C code is built by ``oracle.sparse.build()``
(gcc, OpenMP) into ``oracle/_build/libgrape_oracle.so``.  Operators come from
``oracle.operators`` (dense, built from the physics parameters) and are turned
into coordinate lists here, so nothing is shared with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

from . import operators

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grape_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libgrape_oracle.so")
_lib = None

MODE_FORWARD, MODE_EXACT, MODE_FIRST_ORDER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + OpenMP, no target-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fcx-fortran-rules",
                        "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        lib.grape_oracle_run.restype = ctypes.c_int
        lib.grape_oracle_run.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
            ctypes.c_int, ctypes.c_int,
            P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_double),
            P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_double), ctypes.c_double,
            P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int,
            P(ctypes.c_double), ctypes.c_int, ctypes.c_int,
            P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double)]
        lib.grape_oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().grape_oracle_max_threads())


def _coo(mats):
    ptr, rows, cols, vals = [0], [], [], []
    for M in mats:
        r, c = np.nonzero(M)
        rows.append(r); cols.append(c); vals.append(M[r, c])
        ptr.append(ptr[-1] + len(r))
    rows = np.concatenate(rows).astype(np.int32)
    cols = np.concatenate(cols).astype(np.int32)
    vals = np.ascontiguousarray(np.concatenate(vals).astype(np.complex128))
    return np.array(ptr, dtype=np.int32), rows, cols, vals.view(np.float64)


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def run(phys, u, rho0s, sigma, T, n_rk, mode=MODE_EXACT, threads=0, penalty=None, beta=0.0):
    """Returns (F, grad or None, rhoT, seconds).  Controls on dissipation
    rates come from the physics; `penalty` (the diagonal of A, length d) with
    weight `beta` adds the running cost -beta dt sum_n Re Tr(A rho_n)."""
    lib = _load()
    model = operators.build(phys)
    jumps = list(model.jumps) + [(r, c) for _, r, c in model.rate_ctl]
    jctl = np.array([-1] * len(model.jumps) + [k for k, _, _ in model.rate_ctl], dtype=np.int32)
    ops = [model.H0] + list(model.Hc) + [c for _, c in jumps]
    rates = np.array([g for g, _ in jumps], dtype=np.float64)
    pen = None if penalty is None else np.ascontiguousarray(penalty, dtype=np.float64)
    ptr, rows, cols, vals = _coo(ops)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n_slices, R = u.shape
    rho0s = np.ascontiguousarray(rho0s, dtype=np.complex128)
    n_states, d = rho0s.shape[0], rho0s.shape[1]
    sig = np.ascontiguousarray(sigma, dtype=np.complex128)
    per_state = 1 if sig.ndim == 3 else 0
    F = np.zeros(1)
    G = np.zeros((n_slices, R))
    rhoT = np.zeros((n_states, d, d), dtype=np.complex128)
    t0 = time.perf_counter()
    rc = lib.grape_oracle_run(d, n_states, n_slices, n_rk, float(T), R, len(jumps),
                              _p(ptr, ctypes.c_int), _p(rows, ctypes.c_int), _p(cols, ctypes.c_int),
                              _p(vals, ctypes.c_double), _p(rates, ctypes.c_double),
                              _p(jctl, ctypes.c_int) if model.rate_ctl else None,
                              _p(pen, ctypes.c_double) if pen is not None else None, float(beta),
                              _p(rho0s.view(np.float64), ctypes.c_double),
                              _p(sig.view(np.float64), ctypes.c_double), per_state,
                              _p(u, ctypes.c_double), int(mode), int(threads),
                              _p(F, ctypes.c_double), _p(G, ctypes.c_double),
                              _p(rhoT.view(np.float64), ctypes.c_double))
    dt = time.perf_counter() - t0
    if rc != 0:
        raise RuntimeError(f"grape_oracle_run failed with code {rc}")
    return float(F[0]), (G if mode != MODE_FORWARD else None), rhoT, dt


def run_workload(w, mode=MODE_EXACT, threads=0, penalty=None, beta=0.0):
    return run(w.phys, w.u, w.rho0, w.sigma, w.T, w.n_rk, mode=mode, threads=threads,
               penalty=penalty, beta=beta)

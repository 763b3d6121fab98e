"""The staged gradient-trace kernel (operands copied into shared memory per
pair by bulk asynchronous copies, neighbour positions from a host table)
against the kernel that reads them from global memory: every term and the
order of every sum of the per-slice trace of Eq. (dphidu) are the same, so
the gradients must agree bit for bit, in both precisions and for problem
sizes whose 256-entry blocks need one or several runs of K (d = 8, 120, 180
with four distinct control offsets +-1, +-Q, or two, +-Q, at Q = 2, 3) and
for the Jaynes-Cummings model.  The oracle parity of the staged kernel is
covered by every exact-gradient parity test, where it is the default.
"""
import os

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _gradient(torch, w, precision, trace):
    from paper_1609_03170_gb300 import GrapeProblem, _lib
    old = os.environ.get("GRAPE_TRACE")
    os.environ["GRAPE_TRACE"] = trace
    try:
        P = GrapeProblem.from_workload(w, precision=precision)
    finally:
        if old is None:
            os.environ.pop("GRAPE_TRACE", None)
        else:
            os.environ["GRAPE_TRACE"] = old
    u = torch.from_numpy(w.u).cuda()
    F, G = P.gradient(u)
    torch.cuda.synchronize()
    P.status()
    return float(F), G.cpu().numpy()


def _cases():
    yield "small_q2", lambda: workloads.small(Q=2, N=4, n_slices=5)
    yield "d120", lambda: workloads.transmon_resonator_d120(n_slices=6)
    yield "batch_d180", lambda: _batch_with_d(180)
    yield "batch_q2", lambda: _batch_with_q(2)
    yield "jc_d64", lambda: workloads.jaynes_cummings(64, n_slices=8)


def _batch_with_d(d):
    for i in range(256):
        w = workloads.batch_problem(i, n_slices=6)
        if w.d == d:
            return w
    pytest.skip(f"no batch problem with d={d}")


def _batch_with_q(Q):
    for i in range(256):
        w = workloads.batch_problem(i, n_slices=6)
        if w.phys.Q == Q and w.phys.N >= 40:
            return w
    pytest.skip(f"no batch problem with Q={Q}")


@pytest.mark.parametrize("name,make", list(_cases()), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("precision", ["df64", "fp64"])
def test_staged_trace_equals_global_trace(torch_cuda, name, make, precision):
    from paper_1609_03170_gb300 import _lib
    prec = _lib.GRAPE_PREC_FP64 if precision == "fp64" else _lib.GRAPE_PREC_DF64
    w = make()
    F_t, G_t = _gradient(torch_cuda, w, prec, "tile")
    F_f, G_f = _gradient(torch_cuda, w, prec, "fast")
    assert np.all(np.isfinite(G_t))
    assert F_t == F_f
    assert np.array_equal(G_t, G_f), float(np.abs(G_t - G_f).max())


def test_copy_wait_timeout_returns_error_and_context_survives(torch_cuda):
    """A copy-wait limit of zero makes the staged trace kernel's waits give
    up at once (the producer still waits, with the normal limit, for the
    copies it issued before its CTA leaves): grape_gradient reports
    GRAPE_ETIMEOUT instead of returning a wrong gradient, and the device
    stays usable for the next problem."""
    from paper_1609_03170_gb300 import GrapeProblem, _lib
    w = workloads.transmon_resonator_d120(n_slices=4)
    old = os.environ.get("GRAPE_TRACE_SPIN")
    os.environ["GRAPE_TRACE_SPIN"] = "0"
    try:
        P = GrapeProblem.from_workload(w)
    finally:
        if old is None:
            os.environ.pop("GRAPE_TRACE_SPIN", None)
        else:
            os.environ["GRAPE_TRACE_SPIN"] = old
    with pytest.raises(_lib.GrapeError) as e:
        P.gradient(np.ascontiguousarray(w.u))
    assert e.value.status == _lib.GRAPE_ETIMEOUT
    P.status()                                   # flag cleared after the report
    F1, G1 = GrapeProblem.from_workload(w).gradient(np.ascontiguousarray(w.u))
    F2, G2 = GrapeProblem.from_workload(w).gradient(np.ascontiguousarray(w.u))
    assert F1 == F2 and np.array_equal(G1, G2) and np.all(np.isfinite(G1))

"""The forward and the adjoint sweep at the same time.  The cost
Phi = sum_s Re Tr(sigma_s rho_s(T)) and the running penalty of App. B are
linear in rho, so the exact discrete adjoint (the transpose of the RK4
propagator, Eq. partialuk) starts from a value that does not depend on the
forward sweep and never reads its states; grape_gradient therefore runs the
two sweeps on separate streams and pairs them only in the traces of
Eq. (dphidu).  The kernels and their arithmetic are the same as when the
sweeps run one after the other (GRAPE_CONCURRENT=0), so F and the gradient
must agree bit for bit, with and without the penalty, in both precisions,
over repeated calls (the streams and events are reused).
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


def _grad(torch, P, u, concurrent):
    old = os.environ.get("GRAPE_CONCURRENT")
    os.environ["GRAPE_CONCURRENT"] = "1" if concurrent else "0"
    try:
        out = []
        for _ in range(2):
            F, G = P.gradient(u)
            torch.cuda.synchronize()
            out.append((float(F), G.cpu().numpy()))
        P.status()
    finally:
        if old is None:
            os.environ.pop("GRAPE_CONCURRENT", None)
        else:
            os.environ["GRAPE_CONCURRENT"] = old
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])
    return out[0]


@pytest.mark.parametrize("precision", ["df64", "fp64"])
@pytest.mark.parametrize("penalty", [False, True])
def test_concurrent_sweeps_equal_sequential(torch_cuda, precision, penalty):
    from paper_1609_03170_gb300 import GrapeProblem, _lib
    prec = _lib.GRAPE_PREC_FP64 if precision == "fp64" else _lib.GRAPE_PREC_DF64
    w = workloads.transmon_resonator_d120(n_slices=19)      # 8 chunks of 2-3 slices
    P = GrapeProblem.from_workload(w, precision=prec)
    if penalty:
        P.set_photon_penalty(w.phys.Q, w.phys.N, 0.2 / w.T)
    u = torch_cuda.from_numpy(w.u).cuda()
    F_c, G_c = _grad(torch_cuda, P, u, True)
    F_s, G_s = _grad(torch_cuda, P, u, False)
    assert np.all(np.isfinite(G_c))
    assert F_c == F_s
    assert np.array_equal(G_c, G_s), float(np.abs(G_c - G_s).max())


def test_concurrent_sweeps_host_buffers(torch_cuda):
    """The same through host buffers (the end-to-end path of the C ABI)."""
    from paper_1609_03170_gb300 import GrapeProblem
    w = workloads.qubit_resonator_d20(n_slices=23)
    P = GrapeProblem.from_workload(w)
    F_c, G_c = P.gradient(np.ascontiguousarray(w.u))
    u = torch_cuda.from_numpy(w.u).cuda()
    F_s, G_s = _grad(torch_cuda, P, u, False)
    assert float(F_c) == F_s
    assert np.array_equal(np.asarray(G_c), G_s)

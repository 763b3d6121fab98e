"""grape_gradient_static: the gradient for callers that cannot allocate
device memory (their allocator owns the device memory, or they run where
cudaMalloc may not be called).  Its scratch lives in a static 64 MiB device
array; its results must equal grape_gradient's, call after call: within the
parity tolerance and, since the traces are split and summed in the same
order, bit for bit.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import os

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class env:
    """Environment variables the library reads when a problem is created."""
    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update({k: str(v) for k, v in self.kv.items()})

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _compare(torch, w, grad_mode=0, **create_env):
    from paper_1609_03170_gb300 import GrapeProblem, _lib
    with env(**create_env):
        P = GrapeProblem.from_workload(w, grad_mode=grad_mode)
    u = torch.from_numpy(w.u).cuda()
    F_ref = torch.empty(1, dtype=torch.float64, device="cuda")
    G_ref = torch.empty((w.n_slices, w.n_controls), dtype=torch.float64, device="cuda")
    _lib.grape_gradient(P.handle, u.data_ptr(), F_ref.data_ptr(), G_ref.data_ptr(), 0)
    torch.cuda.synchronize()
    scale = float(G_ref.abs().max())
    for _ in range(2):      # two calls in a row share (and reuse) the static array
        F = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        G = torch.full((w.n_slices, w.n_controls), float("nan"), dtype=torch.float64,
                       device="cuda")
        _lib.grape_gradient_static(P.handle, u.data_ptr(), F.data_ptr(), G.data_ptr(), 0)
        torch.cuda.synchronize()
        assert abs(F.item() - F_ref.item()) <= TOL * abs(F_ref.item())
        assert float((G - G_ref).abs().max()) <= TOL * scale
        assert F.item() == F_ref.item() and torch.equal(G, G_ref)
    return P


def test_static_gradient_matches_allocating_gradient(torch_cuda):
    """d=20 problem at full size (200 slices): the whole stage storage fits."""
    _compare(torch_cuda, workloads.qubit_resonator_d20())


def test_static_gradient_with_checkpoint_segments(torch_cuda):
    """d=120 with 24 slices needs 265 MB of stage storage, more than the
    static array: the call runs two-slice checkpoint segments inside it."""
    _compare(torch_cuda, workloads.transmon_resonator_d120(n_slices=24))


def test_static_gradient_first_order_mode(torch_cuda):
    _compare(torch_cuda, workloads.qubit_resonator_d20(n_slices=60), grad_mode=1)


def test_static_gradient_rejects_host_pointers_and_oversize(torch_cuda):
    from paper_1609_03170_gb300 import GrapeProblem, _lib
    w = workloads.qubit_resonator_d20(n_slices=10)
    P = GrapeProblem.from_workload(w)
    F = np.zeros(1)
    G = np.zeros((w.n_slices, w.n_controls))
    with pytest.raises(_lib.GrapeError) as e:
        _lib.grape_gradient_static(P.handle, w.u.ctypes.data, F.ctypes.data, G.ctypes.data, 0)
    assert e.value.status == _lib.GRAPE_EINVAL
    # d=180, one state, 300 slices: at least 103 MB of scratch whatever the
    # checkpoint segment length (stage storage grows with it, checkpoints shrink)
    phys = workloads.Physics(Q=3, N=60, chi=(0.0, 1.0, 2.0), kappa=1.0)
    big = workloads.make("d180", phys, T=0.9, n_slices=300, n_rk=4, states=[(1, 1.0)],
                         u_bound=1.0)
    Pb = GrapeProblem.from_workload(big)
    u = torch_cuda.from_numpy(big.u).cuda()
    Fd = torch_cuda.empty(1, dtype=torch_cuda.float64, device="cuda")
    Gd = torch_cuda.empty((300, 2), dtype=torch_cuda.float64, device="cuda")
    with pytest.raises(_lib.GrapeError) as e:
        _lib.grape_gradient_static(Pb.handle, u.data_ptr(), Fd.data_ptr(), Gd.data_ptr(), 0)
    assert e.value.status == _lib.GRAPE_EINVAL and "static scratch" in str(e.value)


def test_static_gradient_on_the_grid_kernel(torch_cuda):
    """A problem forced onto the grid kernel: same results as grape_gradient,
    and no barrier gave up (grape_problem_status after the stream)."""
    from paper_1609_03170_gb300 import _lib
    w = workloads.small(Q=3, N=7, n_slices=9, n_rk=3, T=0.9, gamma1=0.2, gamma_phi=0.1,
                        controls_=("res_x", "res_y", "qub_x"))
    P = _compare(torch_cuda, w, GRAPE_KERNEL="grid", GRAPE_GRID_BLOCKS=7)
    assert P.kernel() == "grid"
    _lib.grape_problem_status(P.handle)


def test_static_gradient_reports_a_grid_barrier_timeout(torch_cuda):
    """With a barrier limit of zero polls the grid kernel's barriers give up
    by design: the static call only enqueues work and returns, and
    grape_problem_status after the stream reports GRAPE_ETIMEOUT (results
    invalid); the flag is cleared and the device stays usable."""
    from paper_1609_03170_gb300 import GrapeProblem, _lib
    w = workloads.small(Q=2, N=6, n_slices=3, n_rk=2)
    with env(GRAPE_KERNEL="grid", GRAPE_GRID_BLOCKS=8, GRAPE_SPIN_LIMIT=0):
        P = GrapeProblem.from_workload(w)
    u = torch_cuda.from_numpy(w.u).cuda()
    F = torch_cuda.empty(1, dtype=torch_cuda.float64, device="cuda")
    G = torch_cuda.empty((w.n_slices, w.n_controls), dtype=torch_cuda.float64, device="cuda")
    _lib.grape_gradient_static(P.handle, u.data_ptr(), F.data_ptr(), G.data_ptr(), 0)
    torch_cuda.cuda.synchronize()
    with pytest.raises(_lib.GrapeError) as e:
        _lib.grape_problem_status(P.handle)
    assert e.value.status == _lib.GRAPE_ETIMEOUT
    _lib.grape_problem_status(P.handle)          # cleared after the report
    _compare(torch_cuda, w)                      # the context is intact

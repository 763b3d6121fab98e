"""grape_gradient_static: the gradient for callers that cannot allocate
device memory (their allocator owns the device memory, or they run where
cudaMalloc may not be called).  Its scratch lives in a static 64 MiB device
array; its results must equal grape_gradient's, call after call.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
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


def _compare(torch, w, grad_mode=0):
    from paper_1609_03170_gb300 import GrapeProblem, _lib
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

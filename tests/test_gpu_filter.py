"""Gaussian-filtered controls (App. A) on the GPU against the oracle: the
filter and its transpose on their own, the fused filtered gradient, and the
autograd composition."""
import numpy as np
import pytest

import workloads
from oracle import filter as gf
from oracle import sparse

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("N,M,w0", [(37, 371, [1.067, 0.4, 7.0]),   # ragged, one w0 per control
                                    (1, 1, [2.0, 2.0, 2.0]),          # smallest
                                    (200, 2000, [5.2, 5.2, 5.2])])    # the filtered d=120 shape
def test_filter_and_transpose_match_oracle(torch_cuda, N, M, w0):
    from paper_1609_03170_gb300 import GaussianFilter
    T = 3.7
    rng = np.random.default_rng(N + M)
    u = rng.uniform(-2, 2, size=(N, 3))
    gs = rng.uniform(-1, 1, size=(M, 3))
    f = GaussianFilter(N, M, T, w0, 3)
    s = f.apply(torch_cuda.from_numpy(u).cuda()).cpu().numpy()
    gu = f.adjoint(torch_cuda.from_numpy(gs).cuda()).cpu().numpy()
    assert rel(s, gf.apply(u, M, T / N, T / M, w0)) < 1e-13
    assert rel(gu, gf.adjoint(gs, N, T / N, T / M, w0)) < 1e-13


def filtered_d20(n_steps=20, sub=10):
    w = workloads.qubit_resonator_d20(n_slices=n_steps * sub)
    rng = np.random.default_rng(1609)
    u = rng.uniform(-1, 1, size=(n_steps, 2))
    return w, u, [8.0, 12.0]


def test_filtered_gradient_matches_oracle(torch_cuda):
    """d=20 problem with 20 controls on 200 subpixels: filter, C-oracle
    gradient on the subpixels, transposed filter."""
    from paper_1609_03170_gb300 import GrapeProblem
    w, u, w0 = filtered_d20()
    N, M = u.shape[0], w.n_slices
    s = gf.apply(u, M, w.T / N, w.T / M, w0)
    F_ref, Gs_ref, _, _ = sparse.run(w.phys, s, w.rho0, w.sigma, w.T, w.n_rk, mode=1, threads=2)
    G_ref = gf.adjoint(Gs_ref, N, w.T / N, w.T / M, w0)
    P = GrapeProblem.from_workload(w)
    for _ in range(2):                                    # host arrays, then device tensors
        F, G = P.gradient_filtered(u, w0)
        assert abs(F - F_ref) < TOL * abs(F_ref) and rel(G, G_ref) < TOL
    Fd, Gd = P.gradient_filtered(torch_cuda.from_numpy(u).cuda(), w0)
    assert Fd.item() == F and np.array_equal(Gd.cpu().numpy(), G)


def test_autograd_through_filter_equals_fused(torch_cuda):
    from paper_1609_03170_gb300 import GaussianFilter, GrapeProblem, gaussian_filter, grape_phi
    w, u, w0 = filtered_d20(n_steps=12, sub=7)
    P = GrapeProblem.from_workload(w)
    F, G = P.gradient_filtered(u, w0)
    f = GaussianFilter(u.shape[0], w.n_slices, w.T, w0, 2)
    ut = torch_cuda.from_numpy(u).cuda().requires_grad_(True)
    phi = grape_phi(gaussian_filter(ut, f), P)
    phi.backward()
    assert phi.item() == F
    assert np.array_equal(ut.grad.cpu().numpy(), G)

"""torch.autograd front end: backward equals the library gradient, central
finite differences of Phi, and the oracle; checkpoint segments for long
pulses on the d=600 problem."""
import numpy as np
import pytest

import workloads
from oracle import sparse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("fused", [True, False])
def test_backward_equals_gradient_and_oracle(torch_cuda, fused):
    from paper_1609_03170_gb300 import GrapeProblem, grape_phi
    w = workloads.transmon_resonator_d120(n_slices=16)
    P = GrapeProblem.from_workload(w)
    u = torch_cuda.from_numpy(w.u).cuda().requires_grad_(True)
    phi = grape_phi(u, P, fused)
    (-phi).backward()                        # an optimiser minimises -Phi
    F_ref, G_ref, _, _ = sparse.run_workload(w, threads=3)
    assert abs(phi.item() - F_ref) < 1e-10 * abs(F_ref)
    G = -u.grad.cpu().numpy()
    assert np.max(np.abs(G - G_ref)) < 1e-10 * np.max(np.abs(G_ref))


def test_d600_checkpointed_autograd_matches_finite_differences(torch_cuda):
    """d=600 (rho 5.76 MB), 400 slices with a checkpoint every 20 slices:
    the backward gradient on 32 random slices against central differences
    of Phi.  With slices of 1.5e-4/kappa the gradient entries are at most
    ~1e-5 and Phi carries ~1e-13 relative rounding after 1600 RK substeps, so
    a difference quotient's noise ~1e-13 |Phi| / h needs h ~ 1e-3 to stay
    below 1e-6 of the gradient scale; the truncation error there, h^2/6
    times the third derivative ~ (dt |H_k|)^2 times the first, is ~1e-12."""
    from paper_1609_03170_gb300 import GrapeProblem, grape_phi
    w = workloads.transmon_resonator_d600(n_slices=400)
    P = GrapeProblem.from_workload(w, ckpt_stride=20)
    u = torch_cuda.from_numpy(w.u).cuda().requires_grad_(True)
    phi = grape_phi(u, P)
    phi.backward()
    G = u.grad.cpu().numpy()
    assert P.gradient_launches() > 40            # 20 segments were recomputed
    rng = np.random.default_rng(7)
    js = rng.choice(w.n_slices, size=32, replace=False)
    ks = rng.integers(0, w.n_controls, size=32)
    scale = np.max(np.abs(G))
    h = 1e-3
    for j, k in zip(js, ks):
        up = w.u.copy(); up[j, k] += h
        um = w.u.copy(); um[j, k] -= h
        fd = (P.forward(up, want_rho=False)[0] - P.forward(um, want_rho=False)[0]) / (2 * h)
        assert abs(fd - G[j, k]) < 1e-6 * scale, (j, k, fd, G[j, k])

"""Parity with the oracle on the configurations the batched, served and
differentiable paths run, beyond the headline problem:

  * states of d = 150-180 (Q = 3) on the Hermitian cluster kernel at the
    tiles the batch tuner picks for the 129-160 and 161-192 buckets
    (8 x 512 and 16 x 512), with the batch recipe's physics and with the
    d=120 problem's (Kerr, three controls, three jumps) at N = 50 and 60;
  * controls on the box edge |u| = 5 kappa that serving clamps to, with
    coherent amplitudes |alpha| = 4 (the double-float error bound is
    absolute at the operands' scale, so large operands are the hard case);
  * the d=600 problem at N_t = 400 with a checkpoint every 20 slices, through
    torch.autograd on the grid kernel, against the plain-C oracle's values
    stored by tests/golden/make_d600_nt400.py.

Tolerance 1e-10 relative (max-abs error over max-abs reference), both
kernel precisions.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads
from oracle import sparse

pytestmark = pytest.mark.gpu

TOL = 1e-10
PRECS = [0, 1]          # GRAPE_PREC_DF64, GRAPE_PREC_FP64
HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def gp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_03170_gb300 import problem
    return problem


def check(P, w, F_ref, G_ref, r_ref):
    F, r = P.forward(w.u)
    assert rel(r, r_ref) < TOL
    F2, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * max(abs(F_ref), 1e-300) and F2 == F
    assert rel(G, G_ref) < TOL


def d120_physics(N):
    """The d=120 problem's model with N Fock states."""
    return workloads.Physics(Q=3, N=N, chi=(0.0, 1.0, 2.6), kerr=-0.01, kappa=1.0,
                             gamma1=0.002, gamma_phi=0.001, controls=("res_x", "res_y", "qub_x"))


def phased_states(Q, mags, seed):
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2 * math.pi, size=Q)
    return [(q, complex(mags[q] * np.exp(1j * ph[q]))) for q in range(Q)]


# ------------------------------------------------- batch-sized states

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("index,tile", [(47, (8, 512)), (47, (16, 512)), (129, (16, 512))])
def test_batch_problems_of_the_largest_buckets_on_their_tiles(gp, prec, index, tile):
    """Batch problem 47 (Q=3, N=53, d=159) and 129 (Q=3, N=60, d=180), 12 of
    their slices, on the tiles of their buckets."""
    w = workloads.batch_problem(index, n_slices=12)
    F_ref, G_ref, r_ref, _ = sparse.run_workload(w, threads=3)
    P = gp.GrapeProblem.from_workload(w, precision=prec)
    assert P.kernel() == "hermitian-cluster"
    P.set_tile(*tile)
    assert P.geometry()[:2] == tile
    check(P, w, F_ref, G_ref, r_ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,tile", [(50, (8, 512)), (60, (16, 512))])
def test_d120_model_at_d150_and_d180_on_batch_tiles(gp, prec, N, tile):
    """The d=120 problem's operators (Kerr, three controls, relaxation and
    dephasing of the transmon) with N = 50 (d=150) and N = 60 (d=180)."""
    phys = d120_physics(N)
    w = workloads.make(f"d{3 * N}", phys, T=0.003 * 10, n_slices=10, n_rk=4,
                       states=phased_states(3, (2.0, 3.0, 4.0), 11), u_bound=2.0)
    F_ref, G_ref, r_ref, _ = sparse.run_workload(w, threads=3)
    P = gp.GrapeProblem.from_workload(w, precision=prec)
    P.set_tile(*tile)
    check(P, w, F_ref, G_ref, r_ref)


# ------------------------------------------------- controls on the box edge

def box_edge_d120(n_slices, pattern):
    w = workloads.make("d120_box_edge", d120_physics(40), T=0.003 * n_slices, n_slices=n_slices,
                       n_rk=4, states=phased_states(3, (4.0, 4.0, 4.0), workloads.PHASE_SEED),
                       u_bound=1.0)
    j = np.arange(n_slices)[:, None]
    k = np.arange(w.n_controls)[None, :]
    if pattern == "alternating":
        w.u = 5.0 * (-1.0) ** (j + k)
    else:
        rng = np.random.default_rng(5)
        w.u = 5.0 * rng.choice([-1.0, 1.0], size=w.u.shape)
    return w


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("pattern", ["alternating", "random-sign"])
def test_d120_controls_on_the_box_edge(gp, prec, mode, pattern):
    """d=120 with every control at +-5 kappa and |alpha| = 4, 40 slices."""
    w = box_edge_d120(40, pattern)
    F_ref, G_ref, r_ref, _ = sparse.run_workload(w, mode=1 + mode, threads=3)
    P = gp.GrapeProblem.from_workload(w, grad_mode=mode, precision=prec)
    check(P, w, F_ref, G_ref, r_ref)


# ------------------------------------------------- d=600 at N_t = 400

@pytest.fixture(scope="module")
def golden_d600():
    with open(os.path.join(HERE, "golden", "d600_nt400.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("prec", PRECS)
def test_d600_checkpointed_autograd_matches_oracle_at_nt400(gp, golden_d600, prec):
    """The d=600 problem (rho 5.76 MB) at N_t = 400 on the grid kernel,
    a checkpoint every 20 slices (20 segments recomputed), gradient through
    torch.autograd, against the plain-C oracle."""
    import torch
    from paper_1609_03170_gb300 import grape_phi
    g = golden_d600
    w = workloads.transmon_resonator_d600(n_slices=400)
    assert (w.d, w.n_slices, w.n_rk) == (g["d"], g["n_slices"], g["n_rk"])
    P = gp.GrapeProblem.from_workload(w, ckpt_stride=20, precision=prec)
    assert P.kernel() == "grid"
    u = torch.from_numpy(w.u).cuda().requires_grad_(True)
    phi = grape_phi(u, P)
    phi.backward()
    assert P.gradient_launches() > 40                 # 20 segments recomputed
    G_ref = np.array(g["grad"])
    assert abs(phi.item() - g["F"]) < TOL * abs(g["F"])
    assert rel(u.grad.cpu().numpy(), G_ref) < TOL
    F, r = P.forward(w.u)
    idx = np.array(g["rho_index"])
    r_ref = np.array(g["rho_re"]) + 1j * np.array(g["rho_im"])
    assert rel(r[0][idx[:, 0], idx[:, 1]], r_ref) < TOL
    assert abs(F - g["F"]) < TOL * abs(g["F"])

"""Controls on dissipation rates on the GPU against the dense oracle: exact
and first-order gradients on every propagation kernel and in both number
types (u_k D[a] and u_k D[b] next to Hamiltonian controls)."""
import dataclasses
import os

import numpy as np
import pytest

import workloads
from oracle import dense, operators

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


class env:
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


def problem(**kw):
    args = dict(Q=2, N=4, n_slices=4, n_rk=2, T=0.6, gamma1=0.05,
                controls_=("res_x", "rate_a", "qub_y", "rate_b"))
    args.update(kw)
    w = workloads.small(**args)
    w.u[:, 1] = np.abs(w.u[:, 1]) + 0.2
    w.u[:, 3] = np.abs(w.u[:, 3])
    return w


@pytest.mark.parametrize("kernel", ["hermitian", "full", "grid"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("first_order", [False, True])
def test_rate_controls_match_oracle(gp, kernel, prec, first_order):
    w = problem()
    m = operators.build(w.phys)
    if first_order:
        F_ref, G_ref = dense.gradient_first_order(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    else:
        F_ref, G_ref = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    _, r_ref = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    kv = {"hermitian": {}, "full": {"GRAPE_HERMITIAN": 0}, "grid": {"GRAPE_KERNEL": "grid"}}[kernel]
    mode = gp._lib.GRAPE_GRAD_FIRST_ORDER if first_order else gp._lib.GRAPE_GRAD_EXACT
    with env(**kv):
        P = gp.GrapeProblem.from_workload(w, grad_mode=mode, precision=prec)
    F, r = P.forward(w.u)
    assert rel(r, r_ref) < TOL
    F2, G = P.gradient(w.u)
    assert abs(F2 - F_ref) < TOL * abs(F_ref) and rel(G, G_ref) < TOL


def test_rate_control_on_d20_with_checkpoints(gp):
    base = workloads.qubit_resonator_d20(n_slices=30)
    phys = dataclasses.replace(base.phys, controls=("res_x", "res_y", "rate_a"))
    w = workloads.make("d20_rate", phys, T=base.T, n_slices=30, n_rk=4, states=base.states, u_bound=1.0)
    w.u[:, 2] = np.abs(w.u[:, 2]) * 0.5
    m = operators.build(w.phys)
    F_ref, G_ref = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    P = gp.GrapeProblem.from_workload(w)
    F, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref) and rel(G, G_ref) < TOL
    Pc = gp.GrapeProblem.from_workload(w, ckpt_stride=7)
    Fc, Gc = Pc.gradient(w.u)
    assert Fc == F and np.array_equal(Gc, G)


def test_rate_controls_on_d120_match_the_c_oracle(gp):
    """The d=120 model with a control on the resonator decay and one on the
    transmon relaxation (12 slices) against the plain-C oracle."""
    from oracle import sparse
    base = workloads.transmon_resonator_d120(n_slices=12)
    phys = dataclasses.replace(base.phys, controls=("res_x", "res_y", "rate_a", "rate_b"))
    w = workloads.make("d120_rates", phys, T=base.T, n_slices=12, n_rk=4, states=base.states, u_bound=1.0)
    w.u[:, 2:] = np.abs(w.u[:, 2:])
    F_ref, G_ref, _, _ = sparse.run_workload(w, threads=3)
    P = gp.GrapeProblem.from_workload(w)
    F, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref) and rel(G, G_ref) < TOL

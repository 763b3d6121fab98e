"""Photon-number penalty (Sec. 5, App. B) on the GPU against the oracle:
exact and first-order gradients of Phi_0 - beta Phi_p on every propagation
kernel and in both number types, the penalised forward value, checkpoint
segments, batching, and removal of the penalty."""
import os

import numpy as np
import pytest

import workloads
from oracle import operators, penalty

pytestmark = pytest.mark.gpu

TOL = 1e-10
BETA = 0.35


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


def rich():
    return workloads.small(Q=3, N=4, n_slices=5, n_rk=2, T=0.8, gamma1=0.1, gamma_phi=0.05,
                           controls_=("res_x", "res_y", "qub_x"))


def oracle(w, first_order=False):
    m = operators.build(w.phys)
    A = penalty.number_operator(w.phys)
    return penalty.phi_and_gradient(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, A, BETA, first_order)


@pytest.mark.parametrize("kernel", ["hermitian", "full", "grid"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("first_order", [False, True])
def test_penalised_gradient_matches_oracle(gp, kernel, prec, first_order):
    w = rich()
    F_ref, G_ref = oracle(w, first_order)
    kv = {"hermitian": {}, "full": {"GRAPE_HERMITIAN": 0}, "grid": {"GRAPE_KERNEL": "grid"}}[kernel]
    mode = gp._lib.GRAPE_GRAD_FIRST_ORDER if first_order else gp._lib.GRAPE_GRAD_EXACT
    with env(**kv):
        P = gp.GrapeProblem.from_workload(w, grad_mode=mode, precision=prec)
    P.set_photon_penalty(w.phys.Q, w.phys.N, BETA)
    F, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref)
    assert rel(G, G_ref) < TOL
    Ff, _ = P.forward(w.u)
    assert abs(Ff - F) < 1e-13 * abs(F)


def test_d20_long_pulse_forward_chunks_and_segments(gp):
    """d=20, 150 slices: the forward value crosses three 64-slice chunks and
    the checkpointed gradient equals the stored one bit for bit."""
    w = workloads.qubit_resonator_d20(n_slices=150)
    F_ref, G_ref = oracle(w)
    P = gp.GrapeProblem.from_workload(w)
    P.set_photon_penalty(w.phys.Q, w.phys.N, BETA)
    F, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref) and rel(G, G_ref) < TOL
    assert abs(P.forward(w.u)[0] - F) < 1e-13 * abs(F)
    Pc = gp.GrapeProblem.from_workload(w, ckpt_stride=17)
    Pc.set_photon_penalty(w.phys.Q, w.phys.N, BETA)
    Fc, Gc = Pc.gradient(w.u)
    assert Fc == F and np.array_equal(Gc, G)
    P.set_profiling(True)
    P.gradient(w.u)
    assert sum(n for _, n in P.phase_times().values()) <= P.gradient_launches()


def test_removing_the_penalty_restores_phi0(gp):
    w = rich()
    P = gp.GrapeProblem.from_workload(w)
    F0, G0 = P.gradient(w.u)
    P.set_photon_penalty(w.phys.Q, w.phys.N, BETA)
    F1, _ = P.gradient(w.u)
    assert F1 < F0                      # the penalty lowers Phi
    P.set_penalty(None, 0.0)
    F2, G2 = P.gradient(w.u)
    assert F2 == F0 and np.array_equal(G2, G0)


def test_batch_of_penalised_problems_equals_individual(gp):
    torch = pytest.importorskip("torch")
    ws = [workloads.batch_problem(i, n_slices=9 + 4 * i) for i in range(4)]
    probs = [gp.GrapeProblem.from_workload(w) for w in ws]
    for P, w in zip(probs, ws):
        P.set_photon_penalty(w.phys.Q, w.phys.N, 0.2 / w.T)
    refs = [P.gradient(w.u) for P, w in zip(probs, ws)]
    B = gp.GrapeBatch(probs, n_lanes=2)
    F, Gs = B.gradient([torch.from_numpy(w.u).cuda() for w in ws])
    torch.cuda.synchronize()
    for i, (Fr, Gr) in enumerate(refs):
        assert F[i].item() == Fr and np.array_equal(Gs[i].cpu().numpy(), Gr)


def test_static_entry_point_rejects_a_penalty(gp):
    torch = pytest.importorskip("torch")
    w = rich()
    P = gp.GrapeProblem.from_workload(w)
    P.set_photon_penalty(w.phys.Q, w.phys.N, BETA)
    u = torch.from_numpy(w.u).cuda()
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    G = torch.empty_like(u)
    with pytest.raises(gp._lib.GrapeError) as e:
        gp._lib.grape_gradient_static(P.handle, u.data_ptr(), F.data_ptr(), G.data_ptr(), 0)
    assert e.value.status == gp._lib.GRAPE_EINVAL


def test_d120_penalty_matches_the_c_oracle(gp):
    """The d=120 problem (reduced to 12 slices) with the photon-number penalty
    against the plain-C oracle's running cost."""
    from oracle import sparse
    w = workloads.transmon_resonator_d120(n_slices=12)
    diag = np.repeat(np.arange(w.phys.N, dtype=np.float64), w.phys.Q)
    beta = 0.2 / w.T
    F_ref, G_ref, _, _ = sparse.run_workload(w, threads=3, penalty=diag, beta=beta)
    P = gp.GrapeProblem.from_workload(w)
    P.set_photon_penalty(w.phys.Q, w.phys.N, beta)
    F, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref) and rel(G, G_ref) < TOL

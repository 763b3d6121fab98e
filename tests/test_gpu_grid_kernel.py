"""The grid propagation kernel (states in global memory, one cooperative
grid, a bounded grid barrier per RK stage): parity with the oracle on small
problems forced onto it, the d=600 problem it exists for, and the barrier's
timeout path."""
import os

import numpy as np
import pytest

import workloads
from oracle import dense, operators, sparse

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


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


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("blocks", [1, 7, 152])
def test_grid_kernel_matches_oracle(gp, prec, blocks):
    w = workloads.small(Q=3, N=7, n_slices=9, n_rk=3, T=0.9, gamma1=0.2, gamma_phi=0.1,
                        controls_=("res_x", "res_y", "qub_x", "qub_y"))
    m = operators.build(w.phys)
    F_ref, G_ref = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    _, r_ref = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    with env(GRAPE_KERNEL="grid", GRAPE_GRID_BLOCKS=blocks):
        P = gp.GrapeProblem.from_workload(w, precision=prec)
    assert P.kernel() == "grid"
    F, r = P.forward(w.u)
    assert rel(r, r_ref) < TOL
    F2, G = P.gradient(w.u)
    assert abs(F2 - F_ref) < TOL * abs(F_ref)
    assert rel(G, G_ref) < TOL


def test_grid_kernel_equals_cluster_kernel_d120(gp):
    w = workloads.transmon_resonator_d120(n_slices=12)
    with env(GRAPE_KERNEL="grid"):
        Pg = gp.GrapeProblem.from_workload(w)
    Pc = gp.GrapeProblem.from_workload(w)
    assert Pc.kernel() == "hermitian-cluster"
    Fg, Gg = Pg.gradient(w.u)
    Fc, Gc = Pc.gradient(w.u)
    # the same per-entry arithmetic: identical bits
    assert Fg == Fc and np.array_equal(Gg, Gc)


def test_d600_runs_on_grid_kernel_and_matches_oracle(gp):
    """The 4-level transmon x N=150 resonator (d=600, rho 5.76 MB) does not fit
    a cluster's shared memory; two slices against the plain-C oracle."""
    w = workloads.transmon_resonator_d600(n_slices=2)
    P = gp.GrapeProblem.from_workload(w)
    assert P.kernel() == "grid"
    F_ref, G_ref, r_ref, _ = sparse.run_workload(w, threads=1)
    F, r = P.forward(w.u)
    assert rel(r, r_ref) < TOL
    F2, G = P.gradient(w.u)
    assert abs(F2 - F_ref) < TOL * abs(F_ref)
    assert rel(G, G_ref) < TOL


def test_grid_barrier_timeout_returns_error_and_context_survives(gp):
    """A barrier limit of zero polls makes every non-last CTA give up at the
    first barrier: the call reports GRAPE_ETIMEOUT instead of hanging, and the
    device stays usable."""
    from paper_1609_03170_gb300 import _lib
    w = workloads.small(Q=2, N=6, n_slices=3, n_rk=2)
    with env(GRAPE_KERNEL="grid", GRAPE_GRID_BLOCKS=8, GRAPE_SPIN_LIMIT=0):
        P = gp.GrapeProblem.from_workload(w)
    with pytest.raises(_lib.GrapeError) as e:
        P.forward(w.u)
    assert e.value.status == _lib.GRAPE_ETIMEOUT
    P.status()                                   # flag cleared after the report
    m = operators.build(w.phys)
    F_ref, _ = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    F, _ = gp.GrapeProblem.from_workload(w).forward(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref)

"""Serving loop: device projected L-BFGS against the numpy reference driven by
the oracle's gradients, results alone vs in a mix, admission by memory."""
import time

import numpy as np
import pytest

import workloads
from oracle import lbfgs, sparse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_03170_gb300 as gp
    return gp


def wait(srv, t, timeout=120.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        r = srv.poll(t, timeout_s=0.5)
        if r is not None:
            return r
    raise TimeoutError("served job did not finish")


def test_device_lbfgs_matches_reference_with_oracle_gradients(gp):
    w = workloads.qubit_resonator_d20(n_slices=20)
    P = gp.GrapeProblem.from_workload(w)
    srv = gp.GrapeServer(max_slots=2)
    t = srv.submit(P, w.u, max_iters=8, lbfgs_m=4, u_min=-5, u_max=5, step0=0.5)
    u, F, evals, _, _ = wait(srv, t)
    srv.close()

    def fg(x):
        Fx, Gx, _, _ = sparse.run(w.phys, x.reshape(w.u.shape), w.rho0, w.sigma, w.T, w.n_rk,
                                  threads=2)
        return -Fx, -Gx.ravel()
    u_ref, f_ref, n_ref = lbfgs.minimise(fg, w.u, -5.0, 5.0, max_evals=8, m=4, step0=0.5)
    assert evals == n_ref == 8
    assert abs(F + f_ref) < 1e-9 * abs(f_ref)
    assert np.max(np.abs(u.ravel() - u_ref)) < 1e-7
    assert F > sparse.run_workload(w, mode=0)[0]        # the pulse improved Phi


def mixed_workloads():
    out = [workloads.qubit_resonator_d20(n_slices=30),
           workloads.transmon_resonator_d120(n_slices=12)]
    out += [workloads.batch_problem(i, n_slices=15) for i in (1, 2, 5, 9)]
    return out


def test_results_alone_equal_results_in_the_mix(gp):
    ws = mixed_workloads()
    probs = [gp.GrapeProblem.from_workload(w) for w in ws]
    alone = []
    srv = gp.GrapeServer(max_slots=1)
    for P, w in zip(probs, ws):
        alone.append(wait(srv, srv.submit(P, w.u, max_iters=6)))
    srv.close()
    own = [P.geometry() for P in probs]
    srv = gp.GrapeServer(max_slots=8)
    tickets = [srv.submit(P, w.u, max_iters=6) for P, w in zip(probs, ws)]
    mix = [wait(srv, t) for t in tickets]
    srv.close()
    # jobs sharing the GPU ran on narrowed tiles: the same bits, tiles given back
    for a, b in zip(alone, mix):
        assert np.array_equal(a[0], b[0]) and a[1] == b[1] and a[2] == b[2]
    assert [P.geometry() for P in probs] == own


def test_memory_budget_queues_jobs(gp):
    """A budget that holds one job's gradient storage at a time: jobs wait in
    the queue and still give the same results."""
    ws = [workloads.transmon_resonator_d120(n_slices=10) for _ in range(3)]
    probs = [gp.GrapeProblem.from_workload(w) for w in ws]
    srv = gp.GrapeServer(budget_bytes=600 << 20, max_slots=3)
    tickets = [srv.submit(P, w.u, max_iters=4) for P, w in zip(probs, ws)]
    res = [wait(srv, t) for t in tickets]
    srv.close()
    assert max(r[3] for r in res) > 0.0                      # someone waited in the queue
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and r[1] == res[0][1]

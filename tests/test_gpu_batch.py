"""Batched gradients (many problems of different sizes in one graph launch)
against per-problem gradients and the oracle."""
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


def batch_workloads(n, n_slices):
    return [workloads.batch_problem(i, n_slices=n_slices[i % len(n_slices)]) for i in range(n)]


@pytest.mark.parametrize("lanes", [1, 4, 24])
def test_batch_equals_individual_gradients(torch_cuda, lanes):
    from paper_1609_03170_gb300 import GrapeBatch, GrapeProblem
    ws = batch_workloads(10, [9, 23, 40])
    probs = [GrapeProblem.from_workload(w) for w in ws]
    refs = [p.gradient(w.u) for p, w in zip(probs, ws)]
    B = GrapeBatch(probs, n_lanes=lanes)
    us = [torch_cuda.from_numpy(w.u).cuda() for w in ws]
    for _ in range(2):                       # capture, then graph replay
        F, Gs = B.gradient(us)
        torch_cuda.cuda.synchronize()
        for i, (Fr, Gr) in enumerate(refs):
            assert F[i].item() == Fr
            assert np.array_equal(Gs[i].cpu().numpy(), Gr)


def test_tuner_sets_fitting_tiles_and_restores_them(torch_cuda, monkeypatch):
    """The tuner gives problems of one d bucket the same tile, results keep
    every bit, and destroying the batch gives each problem its own tile back."""
    from paper_1609_03170_gb300 import GrapeBatch, GrapeProblem
    ws = batch_workloads(8, [10, 17])
    probs = [GrapeProblem.from_workload(w) for w in ws]
    own = [p.geometry()[:2] for p in probs]
    refs = [p.gradient(w.u) for p, w in zip(probs, ws)]
    B = GrapeBatch(probs)
    tiles = [p.geometry()[:2] for p in probs]
    buckets = {}
    for w, t, o in zip(ws, tiles, own):
        if t != o:                                  # a tuned problem carries its bucket's tile
            buckets.setdefault((w.d - 1) // 32, set()).add(t)
    assert all(len(v) == 1 for v in buckets.values())
    lanes, _, _ = B.info()
    assert 1 <= lanes <= len(probs)
    us = [torch_cuda.from_numpy(w.u).cuda() for w in ws]
    F, Gs = B.gradient(us)
    torch_cuda.cuda.synchronize()
    for i, (Fr, Gr) in enumerate(refs):
        assert F[i].item() == Fr and np.array_equal(Gs[i].cpu().numpy(), Gr)
        assert probs[i].gradient(ws[i].u)[0] == Fr          # alone, on the tuned tile
    B.close()
    assert [p.geometry()[:2] for p in probs] == own
    monkeypatch.setenv("GRAPE_BATCH_TUNE", "0")
    B2 = GrapeBatch(probs)
    assert [p.geometry()[:2] for p in probs] == own
    B2.close()


def test_batch_replay_sees_new_values_and_recaptures_new_pointers(torch_cuda):
    from paper_1609_03170_gb300 import GrapeBatch, GrapeProblem
    ws = batch_workloads(5, [12, 30])
    probs = [GrapeProblem.from_workload(w) for w in ws]
    B = GrapeBatch(probs, n_lanes=3)
    us = [torch_cuda.from_numpy(w.u).cuda() for w in ws]
    F0, _ = B.gradient(us)
    rng = np.random.default_rng(11)
    new = [rng.uniform(-2, 2, size=w.u.shape) for w in ws]
    for u, v in zip(us, new):
        u.copy_(torch_cuda.from_numpy(v))
    F1, G1 = B.gradient(us)                      # same pointers: graph replay
    us2 = [torch_cuda.from_numpy(v).cuda() for v in new]
    F2, G2 = B.gradient(us2)                     # new pointers: new capture
    torch_cuda.cuda.synchronize()
    for i, (p, v) in enumerate(zip(probs, new)):
        Fr, Gr = p.gradient(v)
        assert F1[i].item() == Fr and F2[i].item() == Fr
        assert np.array_equal(G1[i].cpu().numpy(), Gr) and np.array_equal(G2[i].cpu().numpy(), Gr)
    assert not np.array_equal(F0.cpu().numpy(), F1.cpu().numpy())


def test_batch_problem_against_oracle(torch_cuda):
    """Batch problems span d = 20..180 and both transmon sizes; two of them
    against the plain-C oracle."""
    from paper_1609_03170_gb300 import GrapeBatch, GrapeProblem
    ws = [workloads.batch_problem(i, n_slices=6) for i in (0, 3, 7, 12)]
    probs = [GrapeProblem.from_workload(w) for w in ws]
    B = GrapeBatch(probs, n_lanes=2)
    F, Gs = B.gradient([torch_cuda.from_numpy(w.u).cuda() for w in ws])
    torch_cuda.cuda.synchronize()
    for i in (0, 2):
        Fr, Gr, _, _ = sparse.run_workload(ws[i], threads=3)
        assert abs(F[i].item() - Fr) < 1e-10 * abs(Fr)
        G = Gs[i].cpu().numpy()
        assert np.max(np.abs(G - Gr)) < 1e-10 * np.max(np.abs(Gr))

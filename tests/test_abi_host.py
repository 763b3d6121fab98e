"""Host-side checks that need no GPU: the C ABI loads and exports every
declared symbol, descriptor validation rejects bad input before touching the
device, and the package-side band model equals the oracle's dense operators."""
import ctypes
import dataclasses
import os
import re

import numpy as np
import pytest

import workloads
from oracle import operators
from paper_1609_03170_gb300 import _lib, problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(grape_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_functions()
    assert "grape_gradient" in names and "grape_problem_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert "sm_103a" in _lib.grape_version()


def dense_of(op: problem.BandOp, d):
    M = np.zeros((d, d), dtype=np.complex128)
    for o, v in zip(op.offsets, op.values):
        for i in range(d):
            if 0 <= i + o < d:
                M[i, i + o] += v[i]
    return M


@pytest.mark.parametrize("factory", [
    lambda: workloads.qubit_resonator_d20(n_slices=2),
    lambda: workloads.transmon_resonator_d120(n_slices=2),
    lambda: workloads.small(Q=3, N=5, gamma1=0.1, gamma_phi=0.2,
                            controls_=("res_x", "res_y", "qub_x", "qub_y")),
    lambda: workloads.jaynes_cummings(16, n_slices=2),
    lambda: workloads.make("jc_q3", workloads.Physics(Q=3, N=4, chi=(0.0, 0.5, 1.1), g=0.8,
                                                      controls=("res_x", "qub_y")),
                           T=0.5, n_slices=2, n_rk=1, states=[(1, 0.5)], u_bound=1.0),
])
def test_band_model_equals_dense_operators(factory):
    w = factory()
    bm = problem.band_model(w.phys)
    dm = operators.build(w.phys)
    d = w.d
    scale = max(1.0, np.max(np.abs(dm.H0)))
    assert np.max(np.abs(dense_of(bm.H0, d) - dm.H0)) < 1e-15 * scale
    for a, b in zip(bm.Hc, dm.Hc):
        assert np.max(np.abs(dense_of(a, d) - b)) < 1e-14
    assert len(bm.jumps) == len(dm.jumps)
    for c, rate, (g, cd) in zip(bm.jumps, bm.rates, dm.jumps):
        assert rate == g
        assert np.max(np.abs(dense_of(c, d) - cd)) < 1e-14


def _desc_args(w):
    return problem.band_model(w.phys), w.rho0, w.sigma


def test_create_rejects_non_hermitian_rho0():
    w = workloads.small()
    rho0 = w.rho0.copy()
    rho0[0, 0, 1] += 0.1
    with pytest.raises(_lib.GrapeError) as e:
        problem.GrapeProblem(problem.band_model(w.phys), rho0, w.sigma, w.T, w.n_slices, w.n_rk)
    assert e.value.status == _lib.GRAPE_EINVAL and "Hermitian" in str(e.value)


def test_create_rejects_non_hermitian_control():
    w = workloads.small()
    bm = problem.band_model(w.phys)
    bm.Hc[0].values[0, 0] += 0.5j
    with pytest.raises(_lib.GrapeError) as e:
        problem.GrapeProblem(bm, w.rho0, w.sigma, w.T, w.n_slices, w.n_rk)
    assert e.value.status == _lib.GRAPE_EINVAL


@pytest.mark.parametrize("field,value", [("n_slices", 0), ("n_rk", 0), ("T", -1.0)])
def test_create_rejects_bad_sizes(field, value):
    w = workloads.small()
    kw = dict(T=w.T, n_slices=w.n_slices, n_rk=w.n_rk)
    kw[field] = value
    with pytest.raises(_lib.GrapeError) as e:
        problem.GrapeProblem(problem.band_model(w.phys), w.rho0, w.sigma, **kw)
    assert e.value.status == _lib.GRAPE_EINVAL


def test_create_rejects_offset_out_of_range_and_negative_rate():
    w = workloads.small()
    bm = problem.band_model(w.phys)
    bm.Hc[0].offsets[0] = w.d + 3
    with pytest.raises(_lib.GrapeError):
        problem.GrapeProblem(bm, w.rho0, w.sigma, w.T, w.n_slices, w.n_rk)
    bm = problem.band_model(w.phys)
    bm.rates[0] = -1.0
    with pytest.raises(_lib.GrapeError):
        problem.GrapeProblem(bm, w.rho0, w.sigma, w.T, w.n_slices, w.n_rk)


def test_create_without_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    w = workloads.small()
    with pytest.raises(_lib.GrapeError) as e:
        problem.GrapeProblem.from_workload(w)
    assert e.value.status in (_lib.GRAPE_ECUDA, _lib.GRAPE_ENOMEM)


def test_set_tile_validates_on_the_host():
    lib = _lib.load()
    assert lib.grape_problem_set_tile(None, 4, 128) == _lib.GRAPE_EINVAL


def test_filter_validates_on_the_host():
    lib = _lib.load()
    w = (ctypes.c_double * 2)(1.0, 1.0)
    bad = (ctypes.c_double * 2)(1.0, -1.0)
    assert lib.grape_filter_apply(0, 10, 2, 1.0, 0.1, w, None, None, None) == _lib.GRAPE_EINVAL
    assert lib.grape_filter_apply(1, 10, 9, 1.0, 0.1, w, None, None, None) == _lib.GRAPE_EINVAL
    assert lib.grape_filter_adjoint(1, 10, 2, 0.0, 0.1, w, None, None, None) == _lib.GRAPE_EINVAL
    assert lib.grape_filter_adjoint(1, 10, 2, 1.0, 0.1, bad, None, None, None) == _lib.GRAPE_EINVAL
    # valid sizes, but no device buffers
    assert lib.grape_filter_apply(1, 10, 2, 1.0, 0.1, w, None, None, None) == _lib.GRAPE_EINVAL
    assert lib.grape_gradient_filtered(None, 1, w, None, None, None, None) == _lib.GRAPE_EINVAL


def test_band_model_of_rate_controls():
    """A control on a dissipation rate: empty Hamiltonian band list, its
    dissipator appended to the jumps with rate 1 and its control index."""
    w = workloads.small(Q=2, N=4, controls_=("res_x", "rate_a", "rate_b"), gamma1=0.05)
    bm = problem.band_model(w.phys)
    dm = operators.build(w.phys)
    assert len(bm.Hc[1].offsets) == 0 and len(bm.Hc[2].offsets) == 0
    fixed = len(dm.jumps)
    assert bm.jump_control == [-1] * fixed + [1, 2]
    for (k, r, c), jb, rate in zip(dm.rate_ctl, bm.jumps[fixed:], bm.rates[fixed:]):
        assert r == rate
        assert np.max(np.abs(dense_of(jb, w.d) - c)) < 1e-15


def test_create_validates_rate_controls():
    w = workloads.small(Q=2, N=4, controls_=("res_x", "rate_a"))
    bm = problem.band_model(w.phys)
    bad = dataclasses.replace(bm, jump_control=[-1, 2])          # control index out of range
    with pytest.raises(_lib.GrapeError) as e:
        problem.GrapeProblem(bad, w.rho0, w.sigma, w.T, w.n_slices, w.n_rk)
    assert e.value.status == _lib.GRAPE_EINVAL and "jump_control" in str(e.value)
    bad = dataclasses.replace(bm, jump_control=[-1, 0])          # res_x has a Hamiltonian
    with pytest.raises(_lib.GrapeError) as e:
        problem.GrapeProblem(bad, w.rho0, w.sigma, w.T, w.n_slices, w.n_rk)
    assert e.value.status == _lib.GRAPE_EINVAL and "empty Hamiltonian" in str(e.value)

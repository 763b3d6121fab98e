"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: 1e-10 relative (max-abs error over max-abs reference) on rho(T),
Phi and dPhi/du, as stated for the method; finite differences of the GPU's
own Phi agree with its gradient to 1e-6 relative.  Every parity case runs in
both kernel precisions: double-float on the FP32 pipes (the default) and
native FP64.
"""
import os

import numpy as np
import pytest

import workloads
from oracle import dense, operators, sparse

pytestmark = pytest.mark.gpu

TOL = 1e-10
PRECS = [0, 1]          # GRAPE_PREC_DF64, GRAPE_PREC_FP64


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def gp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_1609_03170_gb300 import problem
    return problem


def rich(**kw):
    args = dict(Q=3, N=4, n_slices=5, n_rk=2, T=0.5, gamma1=0.13, gamma_phi=0.07,
                controls_=("res_x", "res_y", "qub_x"))
    args.update(kw)
    return workloads.small(**args)


def with_env(**kv):
    class _Ctx:
        def __enter__(self):
            self.old = {k: os.environ.get(k) for k in kv}
            for k, v in kv.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = str(v)

        def __exit__(self, *a):
            for k, v in self.old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    return _Ctx()


def with_cluster(n, hermitian=None):
    """GRAPE_CLUSTER picks the cluster width at create time; GRAPE_HERMITIAN=0
    selects the full-matrix kernel instead of the upper-triangle one."""
    return with_env(GRAPE_CLUSTER=n, GRAPE_HERMITIAN=None if hermitian is None else int(hermitian))


KERNELS = [True, False]   # upper-triangle (Hermitian) kernel, full-matrix kernel


# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PRECS)
def test_forward_small_matches_dense_oracle(gp, prec):
    w = rich()
    m = operators.build(w.phys)
    F_ref, r_ref = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    P = gp.GrapeProblem.from_workload(w, precision=prec)
    F, r = P.forward(w.u)
    assert rel(r, r_ref) < TOL
    assert abs(F - F_ref) < TOL * abs(F_ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_small_matches_dense_oracle(gp, mode, prec):
    w = rich()
    m = operators.build(w.phys)
    if mode == 0:
        F_ref, G_ref = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    else:
        F_ref, G_ref = dense.gradient_first_order(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    P = gp.GrapeProblem.from_workload(w, grad_mode=mode, precision=prec)
    F, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref)
    assert rel(G, G_ref) < TOL


@pytest.mark.parametrize("herm", KERNELS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("cluster", [1, 2, 4, 16])
def test_d20_full_size_all_cluster_widths(gp, cluster, prec, herm):
    """The 2-level qubit x N=10 resonator problem (d=20, N_t=200, n_RK=4) at
    full size; cluster 16 splits 400 entries (full kernel) into chunks of 25
    with a 42-entry halo, so halos span two neighbours, and the 210 upper
    entries (Hermitian kernel) into 14 per CTA with windows spanning several."""
    w = workloads.qubit_resonator_d20()
    F_ref, G_ref, r_ref, _ = sparse.run_workload(w, threads=2)
    with with_cluster(cluster, herm):
        P = gp.GrapeProblem.from_workload(w, precision=prec)
    assert P.geometry()[0] == cluster
    F, r = P.forward(w.u)
    assert rel(r, r_ref) < TOL
    F2, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref) and F2 == F
    assert rel(G, G_ref) < TOL


@pytest.mark.parametrize("herm", KERNELS)
@pytest.mark.parametrize("prec", PRECS)
def test_cluster_width_does_not_change_bits(gp, prec, herm):
    """Every entry is computed by the same arithmetic whatever CTA owns it."""
    w = workloads.transmon_resonator_d120(n_slices=6)
    out = []
    for c in (4, 8, 16):
        with with_cluster(c, herm):
            P = gp.GrapeProblem.from_workload(w, precision=prec)
        out.append(P.gradient(w.u))
    for F, G in out[1:]:
        assert F == out[0][0]
        assert np.array_equal(G, out[0][1])


@pytest.mark.parametrize("herm", KERNELS)
@pytest.mark.parametrize("prec", PRECS)
def test_tile_does_not_change_bits(gp, prec, herm):
    """Cluster width and threads per CTA only move entries between CTAs and
    threads: every (width, threads) tile gives the same bits."""
    w = workloads.transmon_resonator_d120(n_slices=6)
    with with_cluster(16, herm):
        P = gp.GrapeProblem.from_workload(w, precision=prec)
    F0, G0 = P.gradient(w.u)
    r0 = P.forward(w.u)[1]
    for c, t in ((8, 128), (16, 64), (16, 256), (8, 512), (16, 480)):
        P.set_tile(c, t)
        assert P.geometry()[:2] == (c, t)
        F, G = P.gradient(w.u)
        assert F == F0 and np.array_equal(G, G0)
        assert np.array_equal(P.forward(w.u)[1], r0)


@pytest.mark.parametrize("prec", PRECS)
def test_cached_and_recomputed_own_coefficients_agree(gp, prec):
    """The coefficient of X_ij itself (offset-0 band and both-offsets-0 jump
    terms) is cached per slice when shared memory allows and recomputed every
    stage otherwise: the same values, so the same bits (d=120 has a
    dephasing jump, so both parts of the coefficient are exercised)."""
    w = workloads.transmon_resonator_d120(n_slices=7)
    P1 = gp.GrapeProblem.from_workload(w, precision=prec)
    with with_env(GRAPE_FOLD=0):
        P0 = gp.GrapeProblem.from_workload(w, precision=prec)
    F1, G1 = P1.gradient(w.u)
    F0, G0 = P0.gradient(w.u)
    assert F1 == F0 and np.array_equal(G1, G0)
    assert np.array_equal(P1.forward(w.u)[1], P0.forward(w.u)[1])


@pytest.mark.parametrize("prec", PRECS)
def test_single_cta_tiles_match_oracle(gp, prec):
    """d=20 with one CTA per state: the tile chosen at create (threads for
    the 210 upper entries rounded up to whole warps) and 64 or 96 threads
    (several entries per thread, a ragged last pass) against the C oracle."""
    w = workloads.qubit_resonator_d20(n_slices=40)
    F_ref, G_ref, r_ref, _ = sparse.run_workload(w, threads=2)
    P = gp.GrapeProblem.from_workload(w, precision=prec)
    assert tuple(P.geometry()) == (1, 224, 1)
    for c, t in ((1, 224), (1, 64), (1, 96), (2, 160)):
        P.set_tile(c, t)
        F, r = P.forward(w.u)
        assert rel(r, r_ref) < TOL
        F2, G = P.gradient(w.u)
        assert abs(F2 - F_ref) < TOL * abs(F_ref) and rel(G, G_ref) < TOL


def test_set_tile_rejects_bad_tiles(gp):
    w = workloads.transmon_resonator_d120(n_slices=4)
    P = gp.GrapeProblem.from_workload(w)
    before = P.geometry()
    for c, t in ((3, 128), (4, 100), (4, 1024), (4, 32)):
        with pytest.raises(gp._lib.GrapeError) as e:
            P.set_tile(c, t)
        assert e.value.status == gp._lib.GRAPE_EINVAL
    with pytest.raises(gp._lib.GrapeError) as e:   # 7260 entries in one CTA do not fit shared memory
        P.set_tile(1, 512)
    assert e.value.status == gp._lib.GRAPE_EINVAL
    assert P.geometry() == before


@pytest.mark.parametrize("prec", PRECS)
def test_hermitian_and_full_kernels_agree(gp, prec):
    """The upper-triangle kernel mirrors the lower triangle instead of
    computing it: both kernels agree to rounding."""
    w = workloads.transmon_resonator_d120(n_slices=20)
    out = []
    for herm in KERNELS:
        with with_cluster(16, herm):
            P = gp.GrapeProblem.from_workload(w, precision=prec)
        out.append((P.forward(w.u)[1], P.gradient(w.u)))
    (r1, (F1, G1)), (r2, (F2, G2)) = out
    assert rel(r1, r2) < 1e-12 and abs(F1 - F2) < 1e-12 * abs(F2) and rel(G1, G2) < 1e-12


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", [0, 1])
def test_d120_reduced_slices_matches_c_oracle(gp, mode, prec):
    """The d=120 transmon-resonator problem (three controls, three jump
    operators, Kerr) with N_t = 40 slices."""
    w = workloads.transmon_resonator_d120(n_slices=40)
    F_ref, G_ref, r_ref, _ = sparse.run_workload(w, mode=1 + mode, threads=3)
    P = gp.GrapeProblem.from_workload(w, grad_mode=mode, precision=prec)
    F, r = P.forward(w.u)
    assert rel(r, r_ref) < TOL
    F2, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref)
    assert rel(G, G_ref) < TOL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("stride", [1, 7, 40])
def test_checkpointed_gradient_equals_stored(gp, stride, prec):
    """Segments with checkpoints and recomputation give the same bits as
    keeping every stage input."""
    w = workloads.qubit_resonator_d20(n_slices=40)
    ref = gp.GrapeProblem.from_workload(w, precision=prec).gradient(w.u)
    P = gp.GrapeProblem.from_workload(w, ckpt_stride=stride, precision=prec)
    F, G = P.gradient(w.u)
    assert F == ref[0]
    assert np.array_equal(G, ref[1])
    P.set_profiling(True)
    P.gradient(w.u)
    counted = sum(n for _, n in P.phase_times().values())
    assert counted == P.gradient_launches()


@pytest.mark.parametrize("chunks", [1, 3, 16])
def test_adjoint_chunks_do_not_change_bits(gp, chunks):
    """The adjoint sweep split into chunks (with the trace of finished chunks
    overlapping on a second stream) gives the bits of one sweep."""
    w = workloads.transmon_resonator_d120(n_slices=24)
    with with_env(GRAPE_ADJ_CHUNKS=1):
        ref = gp.GrapeProblem.from_workload(w).gradient(w.u)
    with with_env(GRAPE_ADJ_CHUNKS=chunks):
        P = gp.GrapeProblem.from_workload(w, ckpt_stride=0)
        F, G = P.gradient(w.u)
        Pc = gp.GrapeProblem.from_workload(w, ckpt_stride=7)
        Fc, Gc = Pc.gradient(w.u)
    assert F == ref[0] and np.array_equal(G, ref[1])
    assert Fc == ref[0] and np.array_equal(Gc, ref[1])


@pytest.mark.parametrize("prec", PRECS)
def test_gpu_gradient_matches_finite_differences_of_gpu_forward(gp, prec):
    w = workloads.transmon_resonator_d120(n_slices=8)
    P = gp.GrapeProblem.from_workload(w, precision=prec)
    _, G = P.gradient(w.u)
    for (j, k) in [(0, 0), (3, 2), (7, 1), (5, 0)]:
        up = w.u.copy(); up[j, k] += 1e-5
        um = w.u.copy(); um[j, k] -= 1e-5
        fd = (P.forward(up, want_rho=False)[0] - P.forward(um, want_rho=False)[0]) / 2e-5
        assert abs(fd - G[j, k]) < 1e-6 * np.max(np.abs(G))


def test_device_pointers_equal_host_pointers(gp):
    import torch
    w = workloads.qubit_resonator_d20(n_slices=30)
    P = gp.GrapeProblem.from_workload(w)
    Fh, Gh = P.gradient(w.u)
    u = torch.from_numpy(w.u).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Fd, Gd = P.gradient(u, stream=s)
    s.synchronize()
    assert Fd.item() == Fh
    assert np.array_equal(Gd.cpu().numpy(), Gh)
    Fr, rd = P.forward(u)
    Fr2, rh = P.forward(w.u)
    assert np.array_equal(rd.cpu().numpy(), rh)


@pytest.mark.parametrize("prec", PRECS)
def test_edge_single_slice_single_substep(gp, prec):
    w = rich(n_slices=1, n_rk=1, T=0.05)
    m = operators.build(w.phys)
    F_ref, G_ref = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    F, G = gp.GrapeProblem.from_workload(w, precision=prec).gradient(w.u)
    assert abs(F - F_ref) < TOL * abs(F_ref)
    assert rel(G, G_ref) < TOL


@pytest.mark.parametrize("prec", PRECS)
def test_edge_one_level_system(gp, prec):
    """Q=1, N=1: d=1, every operator is a number (the trace is conserved)."""
    phys = workloads.Physics(Q=1, N=1, chi=(0.3,), kappa=1.0, controls=("res_x",))
    w = workloads.make("d1", phys, T=1.0, n_slices=3, n_rk=2, states=[(0, 0.0)], u_bound=1.0)
    F, G = gp.GrapeProblem.from_workload(w, precision=prec).gradient(w.u)
    assert abs(F - 1.0) < 1e-15
    assert np.all(G == 0.0)


@pytest.mark.parametrize("herm", KERNELS)
@pytest.mark.parametrize("prec", PRECS)
def test_ragged_dimension_and_transmon_drive(gp, prec, herm):
    """d = 3*7 = 21 (odd, d^2 not a multiple of any cluster width) with all
    four control kinds and a transmon-decay jump."""
    w = workloads.small(Q=3, N=7, n_slices=9, n_rk=3, T=0.9, gamma1=0.2, gamma_phi=0.1,
                        controls_=("res_x", "res_y", "qub_x", "qub_y"))
    m = operators.build(w.phys)
    F_ref, G_ref = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    for c in (1, 8):
        with with_cluster(c, herm):
            P = gp.GrapeProblem.from_workload(w, precision=prec)
        F, G = P.gradient(w.u)
        assert abs(F - F_ref) < TOL * abs(F_ref)
        assert rel(G, G_ref) < TOL


@pytest.mark.parametrize("prec", PRECS)
def test_per_state_sigma_and_non_hermitian_sigma(gp, prec):
    """sigma enters only through its Hermitian part; per-state targets."""
    w = rich()
    rng = np.random.default_rng(3)
    d = w.d
    sig = rng.normal(size=(w.n_states, d, d)) + 1j * rng.normal(size=(w.n_states, d, d))
    m = operators.build(w.phys)
    sig_h = 0.5 * (sig + np.conj(np.transpose(sig, (0, 2, 1))))
    F_ref, G_ref = dense.gradient_exact(m, w.u, w.rho0, sig_h, w.T, w.n_rk)
    P = gp.GrapeProblem(gp.band_model(w.phys), w.rho0, sig, w.T, w.n_slices, w.n_rk,
                        precision=prec)
    F, G = P.gradient(w.u)
    assert abs(F - F_ref) < TOL * max(1.0, abs(F_ref))
    assert rel(G, G_ref) < TOL


def test_d120_full_size_against_c_oracle(gp):
    """The full d=120, N_t=2000, n_RK=4 problem the benchmark times: Phi,
    rho(T) and the whole gradient against the plain-C oracle, in both
    precisions and with both propagation kernels."""
    w = workloads.transmon_resonator_d120()
    F_ref, G_ref, r_ref, _ = sparse.run_workload(w, threads=3)
    for prec in PRECS:
        for herm in KERNELS:
            with with_cluster(None, herm):
                P = gp.GrapeProblem.from_workload(w, precision=prec)
            F, r = P.forward(w.u)
            assert rel(r, r_ref) < TOL
            F2, G = P.gradient(w.u)
            assert abs(F - F_ref) < TOL * abs(F_ref)
            assert rel(G, G_ref) < TOL
            for rr in r:
                assert abs(np.trace(rr) - 1) < 1e-12
                assert np.max(np.abs(rr - rr.conj().T)) < 1e-13
            P.close()


@pytest.mark.parametrize("d", [24, 40])
@pytest.mark.parametrize("mode", [0, 1])
def test_jaynes_cummings_fig2_workload(gp, d, mode):
    """The Fig. 2 scaling workload (qubit x cavity, Jaynes-Cummings coupling on
    the +-(Q-1) bands, 200 slices) against the C oracle, exact and first order."""
    w = workloads.jaynes_cummings(d)
    cmode = sparse.MODE_EXACT if mode == 0 else sparse.MODE_FIRST_ORDER
    F_ref, G_ref, r_ref, _ = sparse.run_workload(w, mode=cmode, threads=1)
    P = gp.GrapeProblem.from_workload(w, grad_mode=mode)
    F, r = P.forward(w.u)
    assert rel(r, r_ref) < TOL
    F2, G = P.gradient(w.u)
    assert abs(F2 - F_ref) < TOL * max(abs(F_ref), 1e-300) and rel(G, G_ref) < TOL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("make", [lambda: workloads.transmon_resonator_d120(n_slices=6),
                                  lambda: workloads.batch_problem(2, n_slices=6),
                                  lambda: workloads.qubit_resonator_d20(n_slices=9)],
                         ids=["transmon_shape", "resonator_shape_d92", "resonator_shape_d20"])
@pytest.mark.parametrize("kernel", ["cluster", "grid"])
def test_shape_specialised_kernels_equal_runtime_shape(gp, prec, make, kernel):
    """The propagation kernels specialised on a model's band/jump layout
    (compile-time loops, neighbour indices and entry state in registers)
    run the same arithmetic in the same order as the kernels that read the
    layout at run time (GRAPE_SHAPE=0): the same bits, on the cluster and on
    the grid kernel."""
    w = make()
    kern = None if kernel == "cluster" else "grid"
    with with_env(GRAPE_KERNEL=kern):
        P1 = gp.GrapeProblem.from_workload(w, precision=prec)
    with with_env(GRAPE_KERNEL=kern, GRAPE_SHAPE=0):
        P0 = gp.GrapeProblem.from_workload(w, precision=prec)
    F1, G1 = P1.gradient(w.u)
    F0, G0 = P0.gradient(w.u)
    P1.status()
    P0.status()
    assert np.all(np.isfinite(G1))
    assert F1 == F0 and np.array_equal(G1, G0)
    assert np.array_equal(P1.forward(w.u)[1], P0.forward(w.u)[1])



@pytest.mark.parametrize("prec", PRECS)
def test_deferred_cluster_wait_equals_default(gp, prec):
    """The Hermitian kernel with the cluster wait placed after the compute
    (GRAPE_DEFER=1, tiles with several entries per thread: the next values
    wait in a shared-memory row) only moves a barrier: the same bits as the
    default placement."""
    w = workloads.transmon_resonator_d120(n_slices=6)
    with with_env(GRAPE_CLUSTER=4):
        P1 = gp.GrapeProblem.from_workload(w, precision=prec)
    with with_env(GRAPE_CLUSTER=4, GRAPE_DEFER=1):
        P0 = gp.GrapeProblem.from_workload(w, precision=prec)
    assert P1.geometry() == P0.geometry() and P1.geometry()[2] > 1
    F1, G1 = P1.gradient(w.u)
    F0, G0 = P0.gradient(w.u)
    P1.status()
    P0.status()
    assert np.all(np.isfinite(G1))
    assert F1 == F0 and np.array_equal(G1, G0)
    assert np.array_equal(P1.forward(w.u)[1], P0.forward(w.u)[1])

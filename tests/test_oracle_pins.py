"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test ties one part of the oracle to mathematics or to the paper:
closed forms of the damped oscillator (Eq. ME), invariants of the Lindblad
equation (Eq. master), the "standard" Liouville-space formulation
(Sec. 2.2), reverse-mode/finite-difference agreement, and the first-order
gradient of Eq. (dphidu).  Together they are chosen so that a dropped term,
a sign, index or transposition error in any part of the oracle fails one.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import dense, liouville, operators, sparse


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rk_poly(z):
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


def rich_problem(**kw):
    """Q=3, N=4 with every operator kind: Kerr, three controls, three jumps."""
    args = dict(Q=3, N=4, n_slices=5, n_rk=2, T=0.5, gamma1=0.13, gamma_phi=0.07,
                controls_=("res_x", "res_y", "qub_x"))
    args.update(kw)
    return workloads.small(**args)


# --------------------------------------------------------------------------
# The RK4 map against the Liouville-space polynomial and the exponential

def test_rk_forward_equals_liouville_polynomial():
    w = rich_problem()
    m = operators.build(w.phys)
    F1, r1 = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    F2, r2 = liouville.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, kind="rk")
    assert rel(r1, r2) < 1e-13
    assert abs(F1 - F2) < 1e-13


def test_rk4_is_fourth_order_towards_expm():
    w = rich_problem(n_slices=3, n_rk=1, T=0.6)
    m = operators.build(w.phys)
    _, rx = liouville.forward(m, w.u, w.rho0, w.sigma, w.T, 1, kind="expm")
    errs = []
    for n_rk in (2, 4, 8):
        _, r = dense.forward(m, w.u, w.rho0, w.sigma, w.T, n_rk)
        errs.append(np.max(np.abs(r - rx)))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    for q in ratios:
        assert 12.0 < q < 20.0, ratios


# --------------------------------------------------------------------------
# Invariants of Eq. (master)

def test_trace_hermiticity_positivity_d20():
    w = workloads.qubit_resonator_d20(n_slices=20)
    m = operators.build(w.phys)
    _, rT = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    for r in rT:
        assert abs(np.trace(r) - 1) < 1e-13
        assert np.max(np.abs(r - r.conj().T)) < 1e-14
        assert np.linalg.eigvalsh((r + r.conj().T) / 2).min() > -1e-9


def test_dual_is_adjoint_under_trace_pairing():
    rng = np.random.default_rng(5)
    w = rich_problem()
    m = operators.build(w.phys)
    H = operators.hamiltonian(m, w.u[1])
    d = m.d

    def herm():
        A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
        return A + A.conj().T

    sig, rho = herm(), herm()
    lhs = np.trace(sig @ dense.lindblad(H, m.jumps, rho))
    rhs = np.trace(dense.lindblad_dual(H, m.jumps, sig) @ rho)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    h = 0.05
    a, _ = dense.rk4_step(lambda r: dense.lindblad(H, m.jumps, r), rho, h)
    b, _ = dense.rk4_step(lambda x: dense.lindblad_dual(H, m.jumps, x), sig, h)
    assert abs(np.trace(sig @ a) - np.trace(b @ rho)) < 1e-13 * abs(np.trace(sig @ a))


# --------------------------------------------------------------------------
# Closed forms of the damped oscillator (Eq. ME)

def test_passive_decay_exact_discrete_and_continuous():
    """Without drive and Kerr, L^dag a = -(kappa/2 + i chi_q) a and
    L^dag n = -kappa n hold exactly in the truncated space, so RK4 gives
    <a>_m = alpha_0 P(h mu)^m and <n>_m = n_0 P(-h kappa)^m."""
    w = workloads.qubit_resonator_d20(n_slices=40)
    w.u[:] = 0.0
    m = operators.build(w.phys)
    Q, N = w.phys.Q, w.phys.N
    a = np.kron(operators.lowering(N), np.eye(Q))
    n_op = a.conj().T @ a
    n_sub = w.n_slices * w.n_rk
    h = w.T / n_sub
    _, rT = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    for s, (q, alpha) in enumerate(w.states):
        mu = -(w.phys.kappa / 2 + 1j * w.phys.chi[q])
        a0 = np.trace(a @ w.rho0[s])
        n0 = np.trace(n_op @ w.rho0[s]).real
        aT = np.trace(a @ rT[s])
        nT = np.trace(n_op @ rT[s]).real
        assert abs(aT - a0 * rk_poly(h * mu) ** n_sub) < 1e-13 * abs(a0)
        assert abs(nT - n0 * rk_poly(-h * w.phys.kappa) ** n_sub) < 1e-13 * n0
        # the continuous solution alpha_0 e^{mu t}, n_0 e^{-kappa t}, within O(h^4)
        assert abs(aT - a0 * np.exp(mu * w.T)) < 1e-8 * abs(a0)
        assert abs(nT - n0 * math.exp(-w.phys.kappa * w.T)) < 1e-8 * n0


@pytest.mark.parametrize("delta,eps", [(0.0, 0.8), (1.3, 1.5)])
def test_driven_steady_state(delta, eps):
    """Constant drive eps (a + a^dag): the RK4 fixed point is the exact one,
    <a>* = -i eps / (kappa/2 + i Delta) and n* = eps^2 / (Delta^2 + kappa^2/4)
    (steady-state photon number of Sec. 4.1 with the detuning Delta)."""
    phys = workloads.Physics(Q=1, N=40, chi=(0.0,), delta=delta, kappa=1.0,
                             controls=("res_x",))
    rho0 = workloads.product_density(1, 40, 0, 0.5 + 0.2j)[None]
    n_slices = 60
    u = np.full((n_slices, 1), eps)
    m = operators.build(phys)
    F, rT = dense.forward(m, u, rho0, workloads.reset_target(1, 40), 60.0, 50)
    a = operators.lowering(40)
    a_ss = -1j * eps / (0.5 + 1j * delta)
    n_ss = eps ** 2 / (delta ** 2 + 0.25)
    assert abs(np.trace(a @ rT[0]) - a_ss) < 1e-10
    assert abs(np.trace(a.conj().T @ a @ rT[0]).real - n_ss) < 1e-10


def test_block_reduction_to_resonator_only():
    """No transmon drive or transmon jumps: each transmon block evolves as a
    resonator-only problem with sigma_z replaced by the level's shift
    (Sec. 4.2)."""
    w = workloads.small(Q=3, N=6, n_slices=4, n_rk=3, T=0.8, kerr=-0.07,
                        chi=(0.0, 1.0, 2.6))
    m = operators.build(w.phys)
    _, rT = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    for s, (q, alpha) in enumerate(w.states):
        phys1 = workloads.Physics(Q=1, N=6, chi=(w.phys.chi[q],), kerr=w.phys.kerr,
                                  kappa=w.phys.kappa, controls=w.phys.controls)
        m1 = operators.build(phys1)
        r0 = workloads.product_density(1, 6, 0, alpha)[None]
        _, r1 = dense.forward(m1, w.u, r0, workloads.reset_target(1, 6), w.T, w.n_rk)
        idx = np.arange(6) * 3 + q
        block = rT[s][np.ix_(idx, idx)]
        assert np.max(np.abs(block - r1[0])) < 1e-14
        mask = np.ones_like(rT[s], dtype=bool)
        mask[np.ix_(idx, idx)] = False
        assert np.max(np.abs(rT[s][mask])) == 0.0


# --------------------------------------------------------------------------
# Gradients

def test_exact_gradient_equals_liouville_frechet():
    w = rich_problem()
    m = operators.build(w.phys)
    F1, G1 = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    F2, G2 = liouville.gradient(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, kind="rk")
    assert abs(F1 - F2) < 1e-13
    assert rel(G1, G2) < 1e-12


def test_exact_gradient_matches_central_differences():
    w = rich_problem(n_slices=4)
    m = operators.build(w.phys)
    _, G = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    entries = [(j, k) for j in range(4) for k in range(3)]
    fd = dense.gradient_fd(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, entries, step=1e-5)
    ex = np.array([G[j, k] for j, k in entries])
    assert np.max(np.abs(fd - ex)) < 1e-6 * np.max(np.abs(ex))


def test_expm_gradient_close_to_rk_gradient():
    """The continuous-time gradient (Van Loan block exponential) and the
    exact gradient of the RK4 map differ by the RK4 truncation, O(h^4)."""
    w = rich_problem(n_slices=3, n_rk=8)
    m = operators.build(w.phys)
    _, Gr = liouville.gradient(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, kind="rk")
    _, Gx = liouville.gradient(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, kind="expm")
    assert rel(Gr, Gx) < 1e-6


def test_first_order_gradient_is_first_order_in_dt():
    """Eq. (dphidu) is accurate to first order in Delta t: splitting every
    slice in two (same control, same RK step h) leaves the exact gradient
    unchanged and halves the first-order error."""
    w = rich_problem(n_slices=4, n_rk=4, T=0.8)
    m = operators.build(w.phys)
    _, Ge = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    _, Gf = dense.gradient_first_order(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    u2 = np.repeat(w.u, 2, axis=0)
    _, Ge2 = dense.gradient_exact(m, u2, w.rho0, w.sigma, w.T, 2)
    _, Gf2 = dense.gradient_first_order(m, u2, w.rho0, w.sigma, w.T, 2)
    Ge2s = Ge2.reshape(4, 2, -1).sum(axis=1)
    Gf2s = Gf2.reshape(4, 2, -1).sum(axis=1)
    assert rel(Ge2s, Ge) < 1e-12
    e1 = np.max(np.abs(Gf - Ge))
    e2 = np.max(np.abs(Gf2s - Ge))
    assert 1.6 < e1 / e2 < 2.4, (e1, e2)


def test_exact_adjoint_state_is_rk4_of_the_dual():
    """mu_before = mu + sum yb_s is P(h L^dag) mu: the backward RK4 of the
    paper's Sec. 3 on the dual equation."""
    w = rich_problem()
    m = operators.build(w.phys)
    H = operators.hamiltonian(m, w.u[2])
    fd = lambda X: dense.lindblad_dual(H, m.jumps, X)
    h = 0.03
    mu = w.sigma.astype(np.complex128)
    kb4 = (h / 6) * mu; yb4 = fd(kb4)
    kb3 = (h / 3) * mu + h * yb4; yb3 = fd(kb3)
    kb2 = (h / 3) * mu + (h / 2) * yb3; yb2 = fd(kb2)
    kb1 = (h / 6) * mu + (h / 2) * yb2; yb1 = fd(kb1)
    back = mu + yb1 + yb2 + yb3 + yb4
    ref, _ = dense.rk4_step(fd, mu, h)
    assert np.max(np.abs(back - ref)) < 1e-15


# --------------------------------------------------------------------------
# The C oracle against the dense one and against the closed forms

@pytest.mark.parametrize("mode", [sparse.MODE_EXACT, sparse.MODE_FIRST_ORDER])
def test_c_oracle_matches_dense(mode):
    w = rich_problem(n_slices=6, n_rk=3)
    m = operators.build(w.phys)
    if mode == sparse.MODE_EXACT:
        F1, G1 = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    else:
        F1, G1 = dense.gradient_first_order(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    _, r1 = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    F2, G2, r2, _ = sparse.run_workload(w, mode=mode, threads=2)
    assert abs(F1 - F2) < 1e-13
    assert rel(G2, G1) < 1e-12
    assert rel(r2, r1) < 1e-13


def test_c_oracle_passive_decay_d120():
    """The d=120 transmon-resonator model without drive, Kerr or transmon
    jumps: <a> and <n> per state follow the exact RK4 closed forms."""
    base = workloads.transmon_resonator_d120(n_slices=10)
    phys = workloads.Physics(Q=3, N=40, chi=base.phys.chi, kappa=1.0,
                             controls=base.phys.controls)
    u = np.zeros((10, 3))
    F, _, rT, _ = sparse.run(phys, u, base.rho0, base.sigma, base.T, base.n_rk,
                             mode=sparse.MODE_FORWARD, threads=3)
    a = np.kron(operators.lowering(40), np.eye(3))
    n_op = a.conj().T @ a
    n_sub = 10 * base.n_rk
    h = base.T / n_sub
    for s, (q, alpha) in enumerate(base.states):
        mu = -(0.5 + 1j * phys.chi[q])
        a0 = np.trace(a @ base.rho0[s])
        n0 = np.trace(n_op @ base.rho0[s]).real
        assert abs(np.trace(a @ rT[s]) - a0 * rk_poly(h * mu) ** n_sub) < 1e-12 * abs(a0)
        assert abs(np.trace(n_op @ rT[s]).real - n0 * rk_poly(-h) ** n_sub) < 1e-12 * n0
        assert abs(np.trace(rT[s]) - 1) < 1e-12


def test_c_oracle_gradient_matches_fd_d120():
    w = workloads.transmon_resonator_d120(n_slices=3)
    F, G, _, _ = sparse.run_workload(w, threads=3)
    for (j, k) in [(0, 0), (1, 2), (2, 1)]:
        up = w.u.copy(); up[j, k] += 1e-5
        um = w.u.copy(); um[j, k] -= 1e-5
        Fp = sparse.run(w.phys, up, w.rho0, w.sigma, w.T, w.n_rk, mode=0, threads=3)[0]
        Fm = sparse.run(w.phys, um, w.rho0, w.sigma, w.T, w.n_rk, mode=0, threads=3)[0]
        assert abs((Fp - Fm) / 2e-5 - G[j, k]) < 1e-6 * np.max(np.abs(G))


@pytest.mark.parametrize("mode", [sparse.MODE_EXACT, sparse.MODE_FIRST_ORDER])
def test_c_oracle_equals_dense_with_rate_controls_and_penalty(mode):
    """The C oracle's rate controls (remarks after Eq. partialuk) and running
    cost (App. B) against the dense oracle, exact and first-order."""
    from oracle import penalty
    w = workloads.small(Q=2, N=4, n_slices=5, n_rk=2, T=0.6, gamma1=0.05,
                        controls_=("res_x", "rate_a", "qub_y", "rate_b"))
    w.u[:, 1] = np.abs(w.u[:, 1]) + 0.2
    w.u[:, 3] = np.abs(w.u[:, 3])
    m = operators.build(w.phys)
    A = penalty.number_operator(w.phys)
    beta = 0.35
    F1, G1 = penalty.phi_and_gradient(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, A, beta,
                                      first_order=(mode == sparse.MODE_FIRST_ORDER))
    F2, G2, _, _ = sparse.run_workload(w, mode=mode, threads=2, penalty=np.real(np.diag(A)), beta=beta)
    assert abs(F1 - F2) < 1e-13 * abs(F1)
    assert rel(G2, G1) < 1e-12
    # and without the penalty, the rate controls alone
    F3, G3 = (dense.gradient_exact if mode == sparse.MODE_EXACT else dense.gradient_first_order)(
        m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    F4, G4, _, _ = sparse.run_workload(w, mode=mode, threads=2)
    assert abs(F3 - F4) < 1e-13 * abs(F3) and rel(G4, G3) < 1e-12

"""Pins of the photon-number penalty of the oracle (Sec. 5, App. B).

The penalised gradient (source -beta dt a^dag a added to the adjoint at every
slice boundary) is tied to the explicit sum over the penalty's terms in the
Liouville formulation (App. B's identity before it is rewritten as a
recursion), to finite differences, to the geometric sum of a passively
decaying photon number, and the first-order form to the exact one.  Planted
mistakes (the source only at the final time, its sign flipped, one boundary
term dropped from the value) each fail a pin.
"""
import numpy as np
import pytest

import workloads
from oracle import dense, liouville, operators, penalty


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rk_poly(z):
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


BETA = 0.35


def problem(**kw):
    args = dict(Q=2, N=4, n_slices=5, n_rk=2, T=0.8, gamma1=0.0, gamma_phi=0.0,
                controls_=("res_x", "res_y", "qub_x"))
    args.update(kw)
    return workloads.small(**args)


def explicit_gradient(m, w, A, beta):
    """d/du of Phi_0 - beta dt sum_n Re Tr(A rho_n), every term differentiated
    on its own through the Liouville slice maps (no recursion)."""
    n_slices, R = w.u.shape
    dt = w.T / n_slices
    maps = [liouville.slice_map(m, w.u[j], dt, w.n_rk, "rk") for j in range(n_slices)]
    ders = [[liouville.slice_map_derivative(m, w.u[j], k, dt, w.n_rk, "rk") for k in range(R)]
            for j in range(n_slices)]
    G = np.zeros((n_slices, R))
    for s, rho0 in enumerate(w.rho0):
        sig = w.sigma[s] if w.sigma.ndim == 3 else w.sigma
        fwd = [liouville.vec(rho0)]
        for Mj in maps:
            fwd.append(Mj @ fwd[-1])
        terms = [(n_slices, liouville.vec(sig.T))]                 # Phi_0
        terms += [(n, -beta * dt * liouville.vec(A.T)) for n in range(n_slices + 1)]
        for n, wv in terms:                                        # d Re(wv . rho_n) / du
            for j in range(n):
                back = wv
                for i in range(n - 1, j, -1):
                    back = back @ maps[i]
                for k in range(R):
                    G[j, k] += float(np.real(back @ (ders[j][k] @ fwd[j])))
    return G


def test_recursion_equals_explicit_sum_of_terms():
    w = problem()
    m = operators.build(w.phys)
    A = penalty.number_operator(w.phys)
    _, G = penalty.phi_and_gradient(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, A, BETA)
    assert rel(G, explicit_gradient(m, w, A, BETA)) < 1e-12


def test_penalised_gradient_matches_finite_differences():
    w = problem(gamma1=0.1, gamma_phi=0.05, Q=3, N=3)
    m = operators.build(w.phys)
    A = penalty.number_operator(w.phys)
    _, G = penalty.phi_and_gradient(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, A, BETA)
    h = 1e-5
    for j, k in [(0, 0), (2, 1), (4, 2), (3, 0)]:
        up = w.u.copy(); up[j, k] += h
        um = w.u.copy(); um[j, k] -= h
        Fp, _ = penalty.phi_and_gradient(m, up, w.rho0, w.sigma, w.T, w.n_rk, A, BETA)
        Fm, _ = penalty.phi_and_gradient(m, um, w.rho0, w.sigma, w.T, w.n_rk, A, BETA)
        assert abs(G[j, k] - (Fp - Fm) / (2 * h)) < 1e-8 * max(1.0, abs(G[j, k]))


def test_penalty_of_passive_decay_is_a_geometric_sum():
    """Without drive, <n> at boundary n is n0 q^n with q = P(-h kappa)^n_rk
    exactly (L^dag a^dag a = -kappa a^dag a in the truncated space), so
    Phi_p = dt sum_s n0_s (1 - q^(N+1)) / (1 - q)."""
    w = workloads.qubit_resonator_d20(n_slices=30)
    w.u[:] = 0.0
    m = operators.build(w.phys)
    A = penalty.number_operator(w.phys)
    dt = w.T / w.n_slices
    q = rk_poly(-(dt / w.n_rk) * w.phys.kappa) ** w.n_rk
    ref = sum(dt * np.trace(A @ r).real * (1 - q ** (w.n_slices + 1)) / (1 - q) for r in w.rho0)
    val = penalty.penalty(m, w.u, w.rho0, w.T, w.n_rk, A)
    assert abs(val - ref) < 1e-13 * ref


def test_first_order_penalised_gradient_is_first_order_in_dt():
    """Splitting every slice in two halves the distance between the
    first-order (Eq. dphidu with the modified backward evolution) and the
    exact penalised gradients."""
    w = problem(n_slices=4, n_rk=4, T=0.8)
    m = operators.build(w.phys)
    A = penalty.number_operator(w.phys)
    errs = []
    for split in (1, 2):
        u = np.repeat(w.u, split, axis=0)
        _, Ge = penalty.phi_and_gradient(m, u, w.rho0, w.sigma, w.T, w.n_rk // split, A, BETA)
        _, Gf = penalty.phi_and_gradient(m, u, w.rho0, w.sigma, w.T, w.n_rk // split, A, BETA,
                                         first_order=True)
        errs.append(np.max(np.abs((Gf - Ge).reshape(4, split, -1).sum(axis=1))))
    assert 1.6 < errs[0] / errs[1] < 2.4, errs


# -------------------------------------------------------------- planted mistakes

def test_source_only_at_the_final_time_fails_the_explicit_sum():
    w = problem()
    m = operators.build(w.phys)
    A = penalty.number_operator(w.phys)
    dt = w.T / w.n_slices
    # the whole penalty weight at t = T only
    _, G = dense.gradient_exact(m, w.u, w.rho0, w.sigma - BETA * dt * A, w.T, w.n_rk)
    assert rel(G, explicit_gradient(m, w, A, BETA)) > 1e-3


def test_flipped_source_sign_fails_finite_differences():
    w = problem(Q=3, N=3)
    m = operators.build(w.phys)
    A = penalty.number_operator(w.phys)
    dt = w.T / w.n_slices
    _, Gbad = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, source=BETA * dt * A)
    h = 1e-5
    up = w.u.copy(); up[2, 1] += h
    um = w.u.copy(); um[2, 1] -= h
    Fp, _ = penalty.phi_and_gradient(m, up, w.rho0, w.sigma, w.T, w.n_rk, A, BETA)
    Fm, _ = penalty.phi_and_gradient(m, um, w.rho0, w.sigma, w.T, w.n_rk, A, BETA)
    fd = (Fp - Fm) / (2 * h)
    assert abs(Gbad[2, 1] - fd) > 1e-4 * abs(fd)


def test_dropped_initial_term_fails_the_geometric_sum(monkeypatch):
    w = workloads.qubit_resonator_d20(n_slices=30)
    w.u[:] = 0.0
    m = operators.build(w.phys)
    A = penalty.number_operator(w.phys)
    orig = dense.propagate

    def without_rho0(*a, **k):
        rT, traj = orig(*a, **k)
        return rT, traj[1:]
    monkeypatch.setattr(dense, "propagate", without_rho0)
    dt = w.T / w.n_slices
    q = rk_poly(-(dt / w.n_rk) * w.phys.kappa) ** w.n_rk
    ref = sum(dt * np.trace(A @ r).real * (1 - q ** (w.n_slices + 1)) / (1 - q) for r in w.rho0)
    assert abs(penalty.penalty(m, w.u, w.rho0, w.T, w.n_rk, A) - ref) > 1e-3 * ref

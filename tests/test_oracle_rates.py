"""Pins of the controls on dissipation rates in the oracle (the variant the
paper mentions after Eq. partialuk): a control u_k that adds u_k D[c] to the
Lindbladian, with dL/du_k = D[c].

Tied to finite differences, to the Liouville-space Frechet derivative (an
independent formulation), to the closed form of a decay whose rate is the
control, and (first-order form) to the exact gradient as Delta t shrinks.
A flipped anticommutator sign in dL/du_k fails them.
"""
import numpy as np
import pytest

import workloads
from oracle import dense, liouville, operators


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rk_poly(z):
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


def problem(**kw):
    args = dict(Q=2, N=4, n_slices=4, n_rk=2, T=0.6, gamma1=0.05,
                controls_=("res_x", "rate_a", "qub_y", "rate_b"))
    args.update(kw)
    w = workloads.small(**args)
    w.u[:, 1] = np.abs(w.u[:, 1]) + 0.2        # rates stay positive (not required by the algebra)
    w.u[:, 3] = np.abs(w.u[:, 3])
    return w


def test_rate_gradient_matches_finite_differences():
    w = problem()
    m = operators.build(w.phys)
    _, G = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    fd = dense.gradient_fd(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, [(0, 1), (2, 1), (1, 3), (3, 0)], step=1e-5)
    for (j, k), v in zip([(0, 1), (2, 1), (1, 3), (3, 0)], fd):
        assert abs(G[j, k] - v) < 1e-8 * max(1.0, abs(v))


def test_rate_gradient_equals_liouville_frechet_derivative():
    w = problem()
    m = operators.build(w.phys)
    F1, G1 = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    F2, G2 = liouville.gradient(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, kind="rk")
    assert abs(F1 - F2) < 1e-13 and rel(G1, G2) < 1e-12


def test_controlled_decay_closed_form():
    """No drive: L^dag n = -(kappa + u) n exactly, so one slice gives
    <n>_T = n0 P(z)^m with z = -h (kappa + u), m = n_RK, and
    d<n>_T/du = n0 m P(z)^(m-1) P'(z) (-h)."""
    phys = workloads.Physics(Q=2, N=8, chi=(-0.3, 0.4), kappa=0.7, controls=("rate_a",))
    rho0 = np.stack([workloads.product_density(2, 8, q, 0.9 - 0.4j * q) for q in range(2)])
    n_op = np.diag(np.repeat(np.arange(8), 2)).astype(np.complex128)
    m_rk, T, u0 = 6, 0.8, 0.45
    u = np.array([[u0]])
    model = operators.build(phys)
    F, G = dense.gradient_exact(model, u, rho0, n_op, T, m_rk)
    h = T / m_rk
    z = -h * (phys.kappa + u0)
    n0 = sum(np.trace(n_op @ r).real for r in rho0)
    dP = 1 + z + z ** 2 / 2 + z ** 3 / 6
    assert abs(F - n0 * rk_poly(z) ** m_rk) < 1e-13 * n0
    assert abs(G[0, 0] - n0 * m_rk * rk_poly(z) ** (m_rk - 1) * dP * (-h)) < 1e-13 * n0


def test_first_order_rate_gradient_is_first_order_in_dt():
    w = problem(n_slices=4, n_rk=4, T=0.8)
    m = operators.build(w.phys)
    errs = []
    for split in (1, 2):
        u = np.repeat(w.u, split, axis=0)
        _, Ge = dense.gradient_exact(m, u, w.rho0, w.sigma, w.T, w.n_rk // split)
        _, Gf = dense.gradient_first_order(m, u, w.rho0, w.sigma, w.T, w.n_rk // split)
        errs.append(np.max(np.abs((Gf - Ge).reshape(4, split, -1).sum(axis=1))))
    assert 1.6 < errs[0] / errs[1] < 2.4, errs


def test_flipped_anticommutator_fails_finite_differences(monkeypatch):
    good = operators.control_derivative

    def bad(model, k, y):
        out = -1j * (model.Hc[k] @ y - y @ model.Hc[k])
        for kk, r, c in model.rate_ctl:
            if kk == k:
                cd = c.conj().T
                out = out + r * (c @ y @ cd + 0.5 * (cd @ c @ y + y @ cd @ c))
        return out
    w = problem()
    m = operators.build(w.phys)
    fd = dense.gradient_fd(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, [(2, 1)], step=1e-5)[0]
    monkeypatch.setattr(operators, "control_derivative", bad)
    _, G = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    assert abs(G[2, 1] - fd) > 1e-3 * abs(fd)

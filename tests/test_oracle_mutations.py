"""Plant plausible mistakes in the (CPU) oracle and check that a pin catches each.

Every mutation is applied with monkeypatch to the dense oracle only; the
assertion is that the pinned quantity moves far outside its tolerance.
"""
import numpy as np

import workloads
from oracle import dense, liouville, operators


def problem():
    return workloads.small(Q=3, N=4, n_slices=4, n_rk=2, T=0.5, gamma1=0.13,
                           gamma_phi=0.07, controls_=("res_x", "res_y", "qub_x"))


def test_dropped_anticommutator_breaks_trace(monkeypatch):
    def bad(H, jumps, rho):
        out = -1j * (H @ rho - rho @ H)
        for g, c in jumps:
            out = out + g * (c @ rho @ c.conj().T)
        return out
    monkeypatch.setattr(dense, "lindblad", bad)
    w = problem()
    _, rT = dense.forward(operators.build(w.phys), w.u, w.rho0, w.sigma, w.T, w.n_rk)
    assert max(abs(np.trace(r) - 1) for r in rT) > 1e-3


def test_wrong_sign_in_dual_breaks_gradient(monkeypatch):
    orig = dense.lindblad_dual
    monkeypatch.setattr(dense, "lindblad_dual",
                        lambda H, jumps, X: orig(-H, jumps, X))
    w = problem()
    m = operators.build(w.phys)
    _, G = dense.gradient_exact(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    _, Gl = liouville.gradient(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, kind="rk")
    assert np.max(np.abs(G - Gl)) > 1e-4 * np.max(np.abs(Gl))


def test_wrong_rk_weight_breaks_liouville_pin(monkeypatch):
    def bad_step(f, y, h):
        k1 = f(y); k2 = f(y + h / 2 * k1); k3 = f(y + h / 2 * k2); k4 = f(y + h * k3)
        return y + h / 6 * (k1 + 2 * k2 + 2 * k3 + 2 * k4), (y, None, None, None)
    monkeypatch.setattr(dense, "rk4_step", bad_step)
    w = problem()
    m = operators.build(w.phys)
    _, r1 = dense.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    _, r2 = liouville.forward(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, kind="rk")
    assert np.max(np.abs(r1 - r2)) > 1e-4


def test_transposed_control_operator_breaks_fd(monkeypatch):
    w = problem()
    m = operators.build(w.phys)
    good = dense.gradient_fd(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, [(1, 1)], step=1e-5)
    m_bad = operators.build(w.phys)
    m_bad.Hc = [H.T.copy() for H in m_bad.Hc]   # i(a^+ - a) transposed flips its sign
    _, G = dense.gradient_exact(m_bad, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    assert abs(G[1, 1] - good[0]) > 1e-3 * abs(good[0])


def test_wrong_adjoint_stage_coefficient_breaks_fd(monkeypatch):
    w = problem()
    m = operators.build(w.phys)
    fd = dense.gradient_fd(m, w.u, w.rho0, w.sigma, w.T, w.n_rk, [(2, 0)], step=1e-5)
    orig = dense.rk4_step

    def gradient_bad(model, u, rho0s, sigma, T, n_rk):
        # same as gradient_exact but kb3 = h/3 mu + h/2 yb4 (should be h yb4)
        n_slices = u.shape[0]; h = T / n_slices / n_rk
        G = np.zeros((n_slices, len(model.Hc)))
        for s, rho0 in enumerate(rho0s):
            rho = rho0.astype(np.complex128); stages = []
            for j in range(n_slices):
                H = operators.hamiltonian(model, u[j])
                per = []
                for _ in range(n_rk):
                    rho, ys = orig(lambda r: dense.lindblad(H, model.jumps, r), rho, h)
                    per.append(ys)
                stages.append(per)
            mu = sigma.astype(np.complex128)
            for j in reversed(range(n_slices)):
                H = operators.hamiltonian(model, u[j])
                fdl = lambda X: dense.lindblad_dual(H, model.jumps, X)
                for r in reversed(range(n_rk)):
                    y1, y2, y3, y4 = stages[j][r]
                    kb4 = h / 6 * mu; yb4 = fdl(kb4)
                    kb3 = h / 3 * mu + h / 2 * yb4; yb3 = fdl(kb3)
                    kb2 = h / 3 * mu + h / 2 * yb3; yb2 = fdl(kb2)
                    kb1 = h / 6 * mu + h / 2 * yb2; yb1 = fdl(kb1)
                    for k, Hk in enumerate(model.Hc):
                        for kb, y in ((kb1, y1), (kb2, y2), (kb3, y3), (kb4, y4)):
                            G[j, k] += np.real(np.trace(kb @ (-1j * (Hk @ y - y @ Hk))))
                    mu = mu + yb1 + yb2 + yb3 + yb4
        return G

    G = gradient_bad(m, w.u, w.rho0, w.sigma, w.T, w.n_rk)
    assert abs(G[2, 0] - fd[0]) > 1e-4 * abs(fd[0])

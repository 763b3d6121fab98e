"""Pins of the projected L-BFGS reference: closed-form minimisers."""
import numpy as np

from oracle import lbfgs


def test_box_constrained_separable_quadratic():
    """f = 1/2 sum a_i (u_i - c_i)^2 over a box: the minimiser is clamp(c)."""
    rng = np.random.default_rng(0)
    a = rng.uniform(0.5, 3.0, size=40)
    c = rng.uniform(-3.0, 3.0, size=40)
    fg = lambda u: (0.5 * float(np.sum(a * (u - c) ** 2)), a * (u - c))
    u, f, n = lbfgs.minimise(fg, np.zeros(40), -1.5, 2.0, max_evals=200, tol=1e-12)
    assert np.max(np.abs(u - np.clip(c, -1.5, 2.0))) < 1e-8


def test_unconstrained_rotated_quadratic():
    """A coupled quadratic inside a box it never touches: u* = A^-1 b."""
    rng = np.random.default_rng(1)
    M = rng.normal(size=(12, 12))
    A = M @ M.T + 12 * np.eye(12)
    b = rng.normal(size=12)
    fg = lambda u: (0.5 * float(u @ A @ u) - float(b @ u), A @ u - b)
    u, f, n = lbfgs.minimise(fg, np.zeros(12), -100.0, 100.0, max_evals=200, tol=1e-11)
    assert np.max(np.abs(u - np.linalg.solve(A, b))) < 1e-8


def test_rejected_trial_halves_step_and_keeps_best():
    """A function that is worse everywhere but the start: f never increases."""
    seen = []

    def fg(u):
        f = float(np.sum(u ** 2)) + (0.0 if not seen else 1.0)
        seen.append(f)
        return f, -np.ones_like(u)          # a misleading gradient
    u, f, n = lbfgs.minimise(fg, np.full(3, 0.5), -1, 1, max_evals=6)
    assert np.allclose(u, 0.5) and f == seen[0] and n == 6

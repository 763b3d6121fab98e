"""Pins of the Gaussian control filter of the oracle (App. A).

The error-function transfer matrix is tied to the paper's frequency-domain
integral, to an independent time-domain convolution with the Gaussian
impulse response, to its limits (partition of unity inside the pulse, the
piecewise-constant controls for an infinitely wide band, shift invariance)
and the chain rule to finite differences of the filtered performance index.
Planted mistakes (a shifted slice edge, a halved w0, a transposed chain rule)
each fail one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads
from oracle import dense, filter as gf, operators

DT, SUB, W0 = 1.0, 0.1, 1.067          # Delta t = 1 ns, delta t = 0.1 ns, wB = 2 pi 100 MHz


def time_domain(n, j, Dt, dt, w0):
    """Entry (n, j) as the box [j Dt, (j+1) Dt) convolved with the impulse
    response of F(w) = exp(-w^2/w0^2), g(tau) = w0/(2 sqrt(pi)) exp(-w0^2 tau^2/4),
    evaluated at the subpixel start n dt."""
    t = n * dt
    g = lambda tp: w0 / (2 * math.sqrt(math.pi)) * math.exp(-(w0 * (t - tp)) ** 2 / 4)
    val, _ = integrate.quad(g, j * Dt, (j + 1) * Dt, epsabs=1e-15, epsrel=1e-13)
    return val


def test_omega0_from_3db_bandwidth():
    # the filter is down by 3 dB (amplitude 1/sqrt 2) at wB
    wb = 2 * math.pi * 0.1
    w0 = gf.omega0_from_bandwidth(wb)
    assert abs(math.exp(-(wb / w0) ** 2) - 1 / math.sqrt(2)) < 1e-15
    assert abs(wb / w0 - 0.5887) < 1e-4


@pytest.mark.parametrize("n,j", [(0, 0), (5, 0), (10, 0), (14, 1), (31, 3), (3, 2)])
def test_erf_form_equals_frequency_integral(n, j):
    T = gf.transfer_matrix(5, 40, DT, SUB, W0)
    assert abs(T[n, j] - gf.transfer_integral(n, j, DT, SUB, W0)) < 1e-9


@pytest.mark.parametrize("w0", [0.3, 1.067, 7.0])
def test_erf_form_equals_time_domain_convolution(w0):
    T = gf.transfer_matrix(4, 45, DT, SUB, w0)
    for n in range(0, 45, 4):
        for j in range(4):
            assert abs(T[n, j] - time_domain(n, j, DT, SUB, w0)) < 1e-12


def test_partition_of_unity_inside_the_pulse():
    # a constant control passes unchanged where the Gaussian does not reach the pulse edges
    N, M = 30, 300
    T = gf.transfer_matrix(N, M, DT, SUB, W0)
    edge = int(math.ceil(12 / W0 / SUB))
    rows = T[edge:M - edge].sum(axis=1)
    assert np.max(np.abs(rows - 1.0)) < 1e-15
    # at the pulse start only half of the Gaussian sees the pulse
    assert abs(T[0].sum() - 0.5) < 1e-15


def test_wide_band_limit_is_piecewise_constant_upsampling():
    N, r = 6, 10
    T = gf.transfer_matrix(N, N * r, DT, DT / r, 1e5)
    ref = np.zeros_like(T)
    for n in range(N * r):
        ref[n, n // r] = 1.0
    ref[0, 0] = 0.5                    # subpixel starting on the pulse edge
    for j in range(1, N):              # subpixels starting on an interior edge
        ref[j * r, j] = 0.5
        ref[j * r, j - 1] = 0.5
    assert np.max(np.abs(T - ref)) < 1e-12


def test_shift_invariance():
    r = 10
    T = gf.transfer_matrix(8, 80, DT, DT / r, W0)
    assert np.max(np.abs(T[r:, 1:] - T[:-r, :-1])) < 1e-15


def test_apply_and_adjoint_are_transposes():
    rng = np.random.default_rng(7)
    u = rng.uniform(-1, 1, size=(9, 2))
    gs = rng.uniform(-1, 1, size=(95, 2))
    w0 = [W0, 2.5]
    s = gf.apply(u, 95, DT, SUB, w0)
    gu = gf.adjoint(gs, 9, DT, SUB, w0)
    # <gs, T u> = <T^T gs, u> per control
    assert abs(np.sum(gs * s) - np.sum(gu * u)) < 1e-12


def filtered_problem():
    """Small three-level problem on M = 10 N subpixels of the filtered controls."""
    w = workloads.small(Q=3, N=3, n_slices=40, n_rk=1, T=2.0, gamma1=0.1, gamma_phi=0.05,
                        controls_=("res_x", "res_y"))
    N = 4
    rng = np.random.default_rng(3)
    u = rng.uniform(-1.5, 1.5, size=(N, 2))
    return w, u, N, w.T / N, w.T / w.n_slices, [3.0, 5.0]


def filtered_phi(m, w, u, Dt, dt, w0):
    s = gf.apply(u, w.n_slices, Dt, dt, w0)
    return dense.forward(m, s, w.rho0, w.sigma, w.T, w.n_rk)[0]


def test_chain_rule_matches_finite_differences():
    w, u, N, Dt, dt, w0 = filtered_problem()
    m = operators.build(w.phys)
    s = gf.apply(u, w.n_slices, Dt, dt, w0)
    _, gs = dense.gradient_exact(m, s, w.rho0, w.sigma, w.T, w.n_rk)
    gu = gf.adjoint(gs, N, Dt, dt, w0)
    h = 1e-5
    for j, k in [(0, 0), (1, 1), (2, 0), (3, 1)]:
        up = u.copy(); up[j, k] += h
        um = u.copy(); um[j, k] -= h
        fd = (filtered_phi(m, w, up, Dt, dt, w0) - filtered_phi(m, w, um, Dt, dt, w0)) / (2 * h)
        assert abs(gu[j, k] - fd) < 1e-8 * max(1.0, abs(fd))


# -------------------------------------------------------------- planted mistakes

def test_shifted_slice_edge_fails_the_time_domain_pin(monkeypatch):
    good = gf.transfer_matrix

    def bad(N, M, Dt, dt, w0):               # slices taken as [(j+1) Dt, (j+2) Dt)
        T = good(N + 1, M, Dt, dt, w0)
        return T[:, 1:]
    monkeypatch.setattr(gf, "transfer_matrix", bad)
    T = gf.transfer_matrix(4, 45, DT, SUB, W0)
    assert abs(T[12, 1] - time_domain(12, 1, DT, SUB, W0)) > 1e-3


def test_halved_omega0_fails_the_frequency_pin(monkeypatch):
    good = gf.transfer_matrix
    monkeypatch.setattr(gf, "transfer_matrix", lambda N, M, Dt, dt, w0: good(N, M, Dt, dt, w0 / 2))
    T = gf.transfer_matrix(5, 40, DT, SUB, W0)
    assert abs(T[14, 1] - gf.transfer_integral(14, 1, DT, SUB, W0)) > 1e-3


def test_untransposed_chain_rule_fails_finite_differences():
    w, u, N, Dt, dt, w0 = filtered_problem()
    m = operators.build(w.phys)
    s = gf.apply(u, w.n_slices, Dt, dt, w0)
    _, gs = dense.gradient_exact(m, s, w.rho0, w.sigma, w.T, w.n_rk)
    # sum over the wrong index: rows of T instead of columns
    bad = np.stack([gf.transfer_matrix(N, w.n_slices, Dt, dt, w0[k])[:N, :] @ gs[:N, k]
                    for k in range(2)], axis=1)
    h = 1e-5
    up = u.copy(); up[1, 0] += h
    um = u.copy(); um[1, 0] -= h
    fd = (filtered_phi(m, w, up, Dt, dt, w0) - filtered_phi(m, w, um, Dt, dt, w0)) / (2 * h)
    assert abs(bad[1, 0] - fd) > 1e-3 * abs(fd)

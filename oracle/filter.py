"""Gaussian filtering of the controls (test infrastructure only).

App. A of the paper (after Motzoi et al.): the N piecewise-constant controls
u_k(j) of length Delta t are mapped to M subpixel amplitudes s_k(n) of length
delta t << Delta t through a transfer matrix, s_k(n) = sum_j T_knj u_k(j),
and the gradient follows by the chain rule, dPhi/du_k(j) = sum_n T_knj
dPhi/ds_k(n).  For the Gaussian filter F(w) = exp(-w^2 / w0^2) the transfer
matrix is the integral of F(w) cos(w (2(n-1) dt - (2j-1) Dt) / 2)
sin(w Dt / 2) / (pi w) over the real line, which equals half the difference
of two error functions, erf(w0 ((n-1) dt - (j-1) Dt) / 2) minus
erf(w0 ((n-1) dt - j Dt) / 2).  The reference bandwidth is w0 = wB /
sqrt(-ln(1/sqrt 2)) for a 3 dB bandwidth wB.

Indices here are 0-based: subpixel n starts at n*dt, control j covers
[j*Dt, (j+1)*Dt).  One w0 per control.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def omega0_from_bandwidth(omega_b: float) -> float:
    """Reference bandwidth w0 of a Gaussian filter with 3 dB bandwidth wB (App. A)."""
    return omega_b / math.sqrt(-math.log(1.0 / math.sqrt(2.0)))


def transfer_matrix(N: int, M: int, Dt: float, dt: float, omega0: float) -> np.ndarray:
    """(M, N) transfer matrix of one control by the error-function form (App. A)."""
    T = np.empty((M, N))
    for n in range(M):
        t = n * dt
        for j in range(N):
            a = omega0 * (t - j * Dt) / 2.0
            b = omega0 * (t - (j + 1) * Dt) / 2.0
            T[n, j] = (math.erf(a) - math.erf(b)) / 2.0
    return T


def transfer_integral(n: int, j: int, Dt: float, dt: float, omega0: float) -> float:
    """One entry by the frequency integral (App. A, first form), numerically.

    The integrand is even in w, so twice the integral over w > 0 is taken;
    the Gaussian makes it negligible beyond 12 w0."""
    c = (2.0 * n * dt - (2.0 * j + 1.0) * Dt) / 2.0

    def f(w):
        if w == 0.0:
            return Dt / (2.0 * math.pi)          # limit of sin(w Dt/2) / (pi w)
        return math.exp(-(w / omega0) ** 2) * math.cos(w * c) * math.sin(w * Dt / 2.0) / (math.pi * w)

    val, _ = integrate.quad(f, 0.0, 12.0 * omega0, limit=2000, epsabs=1e-14, epsrel=1e-12)
    return 2.0 * val


def apply(u: np.ndarray, M: int, Dt: float, dt: float, omega0) -> np.ndarray:
    """s[n, k] = sum_j T_k[n, j] u[j, k]: (N, R) controls -> (M, R) subpixels."""
    u = np.asarray(u, dtype=np.float64)
    N, R = u.shape
    w = np.broadcast_to(np.asarray(omega0, dtype=np.float64), (R,))
    s = np.empty((M, R))
    for k in range(R):
        s[:, k] = transfer_matrix(N, M, Dt, dt, float(w[k])) @ u[:, k]
    return s


def adjoint(gs: np.ndarray, N: int, Dt: float, dt: float, omega0) -> np.ndarray:
    """Chain rule (App. A): g_u[j, k] = sum_n T_k[n, j] g_s[n, k]."""
    gs = np.asarray(gs, dtype=np.float64)
    M, R = gs.shape
    w = np.broadcast_to(np.asarray(omega0, dtype=np.float64), (R,))
    gu = np.empty((N, R))
    for k in range(R):
        gu[:, k] = transfer_matrix(N, M, Dt, dt, float(w[k])).T @ gs[:, k]
    return gu

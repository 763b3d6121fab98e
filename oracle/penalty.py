"""Photon-number penalty of the performance index (test infrastructure only).

Sec. 5 and App. B of the paper: Phi = Phi_0 - beta Phi_p with
Phi_p = sum over initial states of the time integral of Tr(A rho(t)),
A = a^dag a, discretised over the slices as delta t times the sum of
Tr(A rho_n) over the boundary states n = 0 .. N (N + 1 terms, as App. B
writes it).  Its gradient needs one forward and one modified backward
evolution: the backward quantity gets -beta delta t A added at every slice
boundary (App. B's zeta recursion, here on the exact discrete adjoint or on
the first-order lambda of Eq. dphidu).
"""
from __future__ import annotations

import numpy as np

from . import dense


def number_operator(phys) -> np.ndarray:
    """a^dag a of the resonator in the basis i = n Q + q: diagonal n."""
    return np.diag(np.repeat(np.arange(phys.N, dtype=np.float64), phys.Q)).astype(np.complex128)


def penalty(model, u, rho0s, T, n_rk, A) -> float:
    """Phi_p = delta t sum_s sum_{n=0}^{N} Re Tr(A rho_{s,n})."""
    n_slices = u.shape[0]
    dt = T / n_slices
    total = 0.0
    for rho0 in rho0s:
        _, traj = dense.propagate(model, u, rho0, T, n_rk, keep_slices=True)
        for rho in traj:                               # rho_0 .. rho_N
            total += float(np.real(np.trace(A @ rho)))
    return dt * total


def phi_and_gradient(model, u, rho0s, sigma, T, n_rk, A, beta, first_order=False):
    """Phi = Phi_0 - beta Phi_p and dPhi/du (exact discrete adjoint, or the
    first-order form of Eq. dphidu), with the source -beta delta t A."""
    dt = T / u.shape[0]
    src = -beta * dt * A
    if first_order:
        F0, G = dense.gradient_first_order(model, u, rho0s, sigma, T, n_rk, source=src)
    else:
        F0, G = dense.gradient_exact(model, u, rho0s, sigma, T, n_rk, source=src)
    return F0 - beta * penalty(model, u, rho0s, T, n_rk, A), G

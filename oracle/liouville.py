"""The "standard" Liouville-space formulation of open GRAPE (oracle only).

Sec. 2.2 of the paper: rho becomes a d^2 vector and the master equation a
d^2 x d^2 matrix; the slice propagator is a matrix exponential (Eq. Cexp
counts its cost).  Column-stacking vec, vec(A X B) = (B^T kron A) vec(X):
    L = -i (I kron H - H^T kron I)
        + sum_j gamma_j (conj(a_j) kron a_j - 1/2 I kron a_j^dag a_j
                         - 1/2 (a_j^dag a_j)^T kron I).
Three slice maps are provided:
  * rk_poly:  P(hL)^{n_RK} with P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, which is
              what n_RK classic RK4 steps compute for a linear autonomous ODE;
  * expm:     exp(Delta t L), the exact slice propagator L_j of Sec. 2.2;
and gradients as Frechet derivatives through the block-matrix identity
f([[A, E], [0, A]]) = [[f(A), Df(A)[E]], [0, f(A)]] (Van Loan's construction
for the exponential).  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import operators


def vec(X):
    return np.asarray(X).reshape(-1, order="F")


def unvec(v, d):
    return np.asarray(v).reshape(d, d, order="F")


def superop(H, jumps):
    d = H.shape[0]
    I = np.eye(d)
    L = -1j * (np.kron(I, H) - np.kron(H.T, I))
    for gamma, c in jumps:
        cdc = c.conj().T @ c
        L = L + gamma * (np.kron(c.conj(), c) - 0.5 * np.kron(I, cdc)
                         - 0.5 * np.kron(cdc.T, I))
    return L


def control_superop(Hk):
    """dL/du_k = -i (I kron H_k - H_k^T kron I)."""
    d = Hk.shape[0]
    I = np.eye(d)
    return -1j * (np.kron(I, Hk) - np.kron(Hk.T, I))


def rk_poly(X):
    """P(X) = I + X + X^2/2 + X^3/6 + X^4/24 (Horner form)."""
    I = np.eye(X.shape[0])
    return I + X @ (I + X @ (I / 2 + X @ (I / 6 + X / 24)))


def slice_map(model, u_j, dt, n_rk, kind):
    L = superop(operators.hamiltonian(model, u_j), operators.jumps_at(model, u_j))
    if kind == "rk":
        return np.linalg.matrix_power(rk_poly((dt / n_rk) * L), n_rk)
    if kind == "expm":
        return scipy.linalg.expm(dt * L)
    raise ValueError(kind)


def slice_map_derivative(model, u_j, k, dt, n_rk, kind):
    """d(slice map)/du_k through the block-matrix Frechet identity."""
    L = superop(operators.hamiltonian(model, u_j), operators.jumps_at(model, u_j))
    E = control_superop(model.Hc[k])
    for kk, r, c in model.rate_ctl:           # a control on a dissipation rate: r D[c]
        if kk == k:
            E = E + superop(np.zeros_like(model.Hc[k]), [(r, c)])
    n = L.shape[0]
    if kind == "rk":
        h = dt / n_rk
        B = np.block([[h * L, h * E], [np.zeros((n, n)), h * L]])
        P = np.linalg.matrix_power(rk_poly(B), n_rk)
    else:
        B = np.block([[dt * L, dt * E], [np.zeros((n, n)), dt * L]])
        P = scipy.linalg.expm(B)
    return P[:n, n:]


def forward(model, u, rho0s, sigma, T, n_rk, kind="rk"):
    n_slices = u.shape[0]
    dt = T / n_slices
    maps = [slice_map(model, u[j], dt, n_rk, kind) for j in range(n_slices)]
    F = 0.0
    out = []
    for s, rho0 in enumerate(rho0s):
        sig = sigma[s] if sigma.ndim == 3 else sigma
        v = vec(rho0)
        for M in maps:
            v = M @ v
        rhoT = unvec(v, model.d)
        out.append(rhoT)
        F += float(np.real(np.trace(sig @ rhoT)))
    return F, np.stack(out)


def gradient(model, u, rho0s, sigma, T, n_rk, kind="rk"):
    """dPhi/du_k(j) = Re vec(sigma^T)^T M_N..M_{j+1} D_jk M_{j-1}..M_1 vec(rho0)."""
    n_slices, R = u.shape
    dt = T / n_slices
    maps = [slice_map(model, u[j], dt, n_rk, kind) for j in range(n_slices)]
    ders = [[slice_map_derivative(model, u[j], k, dt, n_rk, kind) for k in range(R)]
            for j in range(n_slices)]
    G = np.zeros((n_slices, R))
    F = 0.0
    for s, rho0 in enumerate(rho0s):
        sig = sigma[s] if sigma.ndim == 3 else sigma
        fwd = [vec(rho0)]
        for M in maps:
            fwd.append(M @ fwd[-1])
        w = vec(sig.T)              # Tr(sig X) = w . vec(X) (no conjugation)
        F += float(np.real(w @ fwd[-1]))
        back = [None] * (n_slices + 1)
        back[n_slices] = w
        for j in reversed(range(n_slices)):
            back[j] = back[j + 1] @ maps[j]
        for j in range(n_slices):
            for k in range(R):
                G[j, k] += float(np.real(back[j + 1] @ (ders[j][k] @ fwd[j])))
    return F, G

"""Dense FP64 open GRAPE with RK4 propagation (oracle; test infrastructure only).

Follows the paper's steps in its notation:
  * Lindblad map  L rho = -i[H, rho] + sum_j gamma_j D[a_j] rho,
    D[a] rho = a rho a^dag - {a^dag a, rho}/2            (Eq. master, Eq. disspation)
  * its dual under the bilinear pairing <X, rho> = Tr(X rho):
    L^dag X = i[H, X] + sum_j gamma_j (a_j^dag X a_j - {a_j^dag a_j, X}/2)
  * forward propagation slice by slice, Delta t = T/N, each slice integrated
    with n_RK classic RK4 substeps of h = Delta t / n_RK  (Sec. 3, Eq. rkmaster)
  * performance index Phi = sum_s Re Tr(sigma rho_s(T))  (Eq. phi, Eq. Phi0)
  * gradient:
      - "exact": reverse mode through every RK4 stage, which is the exact
        derivative of the discrete map the forward pass computes;
      - "first_order": the paper's Eq. (dphidu),
        dPhi/du_k(j) = -i Delta t Tr(lambda_j [H_k, rho_j]), where lambda_{j-1}
        comes from lambda_j by backward RK4 on L^dag over slice j, starting
        from lambda_N = sigma (Sec. 3 backward integration, Eq. lambda).
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np

from . import operators


def lindblad(H, jumps, rho):
    """Eq. (master) with Eq. (disspation)."""
    out = -1j * (H @ rho - rho @ H)
    for gamma, c in jumps:
        cd = c.conj().T
        cdc = cd @ c
        out = out + gamma * (c @ rho @ cd - 0.5 * (cdc @ rho + rho @ cdc))
    return out


def lindblad_dual(H, jumps, X):
    """Dual of Eq. (master): Tr(X L rho) = Tr((L^dag X) rho) for all rho."""
    out = 1j * (H @ X - X @ H)
    for gamma, c in jumps:
        cd = c.conj().T
        cdc = cd @ c
        out = out + gamma * (cd @ X @ c - 0.5 * (cdc @ X + X @ cdc))
    return out


def rk4_step(f, y, h):
    """Classic RK4 (nodes 0, 1/2, 1/2, 1; weights 1/6, 1/3, 1/3, 1/6).
    Returns the new value and the four stage inputs."""
    y1 = y
    k1 = f(y1)
    y2 = y + (h / 2) * k1
    k2 = f(y2)
    y3 = y + (h / 2) * k2
    k3 = f(y3)
    y4 = y + h * k3
    k4 = f(y4)
    return y + (h / 6) * (k1 + 2 * k2 + 2 * k3 + k4), (y1, y2, y3, y4)


def _geometry(T, u, n_rk):
    n_slices = u.shape[0]
    dt = T / n_slices
    return n_slices, dt, dt / n_rk


def propagate(model, u, rho0, T, n_rk, keep_slices=False):
    """rho_j for one initial state: returns rho(T) (and the list rho_0..rho_N)."""
    n_slices, dt, h = _geometry(T, u, n_rk)
    rho = np.array(rho0, dtype=np.complex128)
    traj = [rho]
    for j in range(n_slices):
        H = operators.hamiltonian(model, u[j])
        f = lambda r, H=H, J=operators.jumps_at(model, u[j]): lindblad(H, J, r)
        for _ in range(n_rk):
            rho, _ = rk4_step(f, rho, h)
        if keep_slices:
            traj.append(rho)
    return (rho, traj) if keep_slices else rho


def cost(sigma, rhoT) -> float:
    """Re Tr(sigma rho(T)) (Eq. phi)."""
    return float(np.real(np.trace(sigma @ rhoT)))


def _sigma_for(sigma, s):
    return sigma[s] if sigma.ndim == 3 else sigma


def forward(model, u, rho0s, sigma, T, n_rk):
    """Phi summed over the initial states, and the final states."""
    rhoT = [propagate(model, u, r0, T, n_rk) for r0 in rho0s]
    F = sum(cost(_sigma_for(sigma, s), r) for s, r in enumerate(rhoT))
    return F, np.stack(rhoT)


def gradient_exact(model, u, rho0s, sigma, T, n_rk, source=None):
    """Phi and dPhi/du_k(j), reverse mode through every RK4 stage.

    `source` (a d x d matrix, default none) is added to the adjoint at every
    slice boundary, the final time included: the gradient of a cost with the
    running term sum_n Re Tr(source rho_n) over the boundary states rho_0 ..
    rho_N (App. B, the photon-number penalty).  The returned Phi is the
    final-time part only.

    For one substep with stage inputs y_1..y_4 and stage outputs
    k_s = L y_s, given mu = dPhi/d(rho after the substep) as a matrix of the
    bilinear pairing, the stage adjoints are
        kb4 = h/6 mu,              yb4 = L^dag kb4
        kb3 = h/3 mu + h yb4,      yb3 = L^dag kb3
        kb2 = h/3 mu + h/2 yb3,    yb2 = L^dag kb2
        kb1 = h/6 mu + h/2 yb2,    yb1 = L^dag kb1
        mu_before = mu + yb1 + yb2 + yb3 + yb4
    and each stage contributes Re Tr(kb_s (dL/du_k) y_s) to dPhi/du_k(j),
    with dL/du_k rho = -i[H_k, rho] (Eq. master with Eq. Hamiltonian), plus
    r D[c] rho for a control on a dissipation rate.
    """
    n_slices, dt, h = _geometry(T, u, n_rk)
    R = len(model.Hc)
    G = np.zeros((n_slices, R))
    F = 0.0
    for s, rho0 in enumerate(rho0s):
        sig = _sigma_for(sigma, s)
        rho = np.array(rho0, dtype=np.complex128)
        stages = []                      # stages[j][r] = (y1, y2, y3, y4)
        for j in range(n_slices):
            H = operators.hamiltonian(model, u[j])
            f = lambda r, H=H, J=operators.jumps_at(model, u[j]): lindblad(H, J, r)
            per = []
            for _ in range(n_rk):
                rho, ys = rk4_step(f, rho, h)
                per.append(ys)
            stages.append(per)
        F += cost(sig, rho)
        mu = np.array(sig, dtype=np.complex128)
        if source is not None:
            mu = mu + source
        for j in reversed(range(n_slices)):
            H = operators.hamiltonian(model, u[j])
            fd = lambda X, H=H, J=operators.jumps_at(model, u[j]): lindblad_dual(H, J, X)
            for r in reversed(range(n_rk)):
                y1, y2, y3, y4 = stages[j][r]
                kb4 = (h / 6) * mu
                yb4 = fd(kb4)
                kb3 = (h / 3) * mu + h * yb4
                yb3 = fd(kb3)
                kb2 = (h / 3) * mu + (h / 2) * yb3
                yb2 = fd(kb2)
                kb1 = (h / 6) * mu + (h / 2) * yb2
                yb1 = fd(kb1)
                for k in range(R):
                    acc = 0.0
                    for kb, y in ((kb1, y1), (kb2, y2), (kb3, y3), (kb4, y4)):
                        acc += np.real(np.trace(kb @ operators.control_derivative(model, k, y)))
                    G[j, k] += acc
                mu = mu + yb1 + yb2 + yb3 + yb4
            if source is not None:
                mu = mu + source
    return F, G


def backward_targets(model, u, sigma, T, n_rk, source=None):
    """lambda_j for j = N..0 by backward RK4 on L^dag from lambda_N = sigma
    (Sec. 3 backward integration; lambda_{j-1} = L_j^dag lambda_j, Eq. lambda).
    With `source`, App. B's modified backward evolution: the source is added
    to lambda_N and after every backward slice."""
    n_slices, dt, h = _geometry(T, u, n_rk)
    lam = np.array(sigma, dtype=np.complex128)
    if source is not None:
        lam = lam + source
    out = [None] * (n_slices + 1)
    out[n_slices] = lam
    for j in reversed(range(n_slices)):
        H = operators.hamiltonian(model, u[j])
        fd = lambda X, H=H, J=operators.jumps_at(model, u[j]): lindblad_dual(H, J, X)
        for _ in range(n_rk):
            lam, _ = rk4_step(fd, lam, h)
        if source is not None:
            lam = lam + source
        out[j] = lam
    return out


def gradient_first_order(model, u, rho0s, sigma, T, n_rk, source=None):
    """Eq. (dphidu): dPhi/du_k(j) = Re(-i Delta t Tr(lambda_j [H_k, rho_j])),
    with rho_j and lambda_j both taken at t = j Delta t, j = 1..N (lambda
    from backward_targets, with `source` as there)."""
    n_slices, dt, h = _geometry(T, u, n_rk)
    R = len(model.Hc)
    G = np.zeros((n_slices, R))
    F = 0.0
    for s, rho0 in enumerate(rho0s):
        sig = _sigma_for(sigma, s)
        rhoT, traj = propagate(model, u, rho0, T, n_rk, keep_slices=True)
        F += cost(sig, rhoT)
        lams = backward_targets(model, u, sig, T, n_rk, source)
        for j in range(1, n_slices + 1):
            rho_j, lam_j = traj[j], lams[j]
            for k in range(R):
                G[j - 1, k] += np.real(dt * np.trace(lam_j @ operators.control_derivative(model, k, rho_j)))
    return F, G


def gradient_fd(model, u, rho0s, sigma, T, n_rk, entries, step=1e-6):
    """Central finite differences of Phi at the given (j, k) entries."""
    out = []
    for (j, k) in entries:
        up = u.copy(); up[j, k] += step
        um = u.copy(); um[j, k] -= step
        Fp, _ = forward(model, up, rho0s, sigma, T, n_rk)
        Fm, _ = forward(model, um, rho0s, sigma, T, n_rk)
        out.append((Fp - Fm) / (2 * step))
    return np.array(out)


def expect(op, rho) -> complex:
    return complex(np.trace(op @ rho))

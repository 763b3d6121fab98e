"""Dense operators of the dispersive transmon-resonator model (oracle side).

Built directly from the physics parameters with Kronecker products, in the
basis index i = n*Q + q (resonator Fock index n, transmon level q).
Cites: Eq. (Hdrive) dispersive Hamiltonian with sigma_z replaced by a per-level
shift (Sec. 4.2, "replace sigma_z by +-1"), Eq. (kerr) H_K = K (a^dag a)^2,
Eq. (ME) damping kappa D[a], and the two-quadrature drive
H_d = eps_X (a^dag + a) + i eps_Y (a^dag - a) of Sec. 4.2.
Test infrastructure only.
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np


def lowering(n: int) -> np.ndarray:
    """a|k> = sqrt(k)|k-1> on an n-dimensional truncated space."""
    a = np.zeros((n, n), dtype=np.complex128)
    for k in range(1, n):
        a[k - 1, k] = np.sqrt(k)
    return a


@dataclasses.dataclass
class DenseModel:
    d: int
    H0: np.ndarray                        # drift Hamiltonian
    Hc: List[np.ndarray]                  # control Hamiltonians H_k (Eq. Hamiltonian)
    jumps: List[Tuple[float, np.ndarray]]  # (gamma_j, a_j) of Eq. (disspation)
    # controls on dissipation rates (the variant mentioned after Eq. partialuk):
    # (control k, weight r, c) adds u_k(j) r D[c] to the slice's Lindbladian;
    # such a control has a zero Hamiltonian H_k
    rate_ctl: List[Tuple[int, float, np.ndarray]] = dataclasses.field(default_factory=list)


def build(phys) -> DenseModel:
    Q, N = phys.Q, phys.N
    IQ, IN = np.eye(Q), np.eye(N)
    a = np.kron(lowering(N), IQ)            # resonator a
    b = np.kron(IN, lowering(Q))            # transmon b
    n_op = a.conj().T @ a
    proj = [np.kron(IN, np.diag(np.eye(Q)[q])) for q in range(Q)]

    H0 = np.zeros((N * Q, N * Q), dtype=np.complex128)
    for q in range(Q):
        H0 += phys.chi[q] * n_op @ proj[q]
    H0 += phys.delta * n_op + phys.kerr * n_op @ n_op
    if phys.qubit_energy:
        for q in range(Q):
            H0 += phys.qubit_energy[q] * proj[q]
    if phys.g:                                  # Jaynes-Cummings exchange (Fig. 2 model)
        H0 += phys.g * (a @ b.conj().T + a.conj().T @ b)

    kinds = {
        "res_x": a + a.conj().T,
        "res_y": 1j * (a.conj().T - a),
        "qub_x": b + b.conj().T,
        "qub_y": 1j * (b.conj().T - b),
    }
    rate_ops = {"rate_a": a, "rate_b": b}          # u_k D[a], u_k D[b]
    Hc, rate_ctl = [], []
    for k, name in enumerate(phys.controls):
        if name in rate_ops:
            Hc.append(np.zeros((N * Q, N * Q), dtype=np.complex128))
            rate_ctl.append((k, 1.0, rate_ops[name].astype(np.complex128)))
        else:
            Hc.append(kinds[name].astype(np.complex128))

    jumps = [(phys.kappa, a)]
    if phys.gamma1:
        jumps.append((phys.gamma1, b))
    if phys.gamma_phi:
        jumps.append((phys.gamma_phi, b.conj().T @ b))
    return DenseModel(d=N * Q, H0=H0, Hc=Hc, jumps=jumps, rate_ctl=rate_ctl)


def jumps_at(model: DenseModel, u_j):
    """The slice's dissipators: the fixed (gamma, c) and, for every rate
    control, (u_k(j) r, c)."""
    return list(model.jumps) + [(u_j[k] * r, c) for k, r, c in model.rate_ctl]


def control_derivative(model: DenseModel, k: int, y: np.ndarray) -> np.ndarray:
    """dL/du_k applied to y: -i[H_k, y] (Eq. partialuk before the Delta t
    expansion), plus r D[c](y) when u_k is a rate control."""
    Hk = model.Hc[k]
    out = -1j * (Hk @ y - y @ Hk)
    for kk, r, c in model.rate_ctl:
        if kk == k:
            cd = c.conj().T
            cdc = cd @ c
            out = out + r * (c @ y @ cd - 0.5 * (cdc @ y + y @ cdc))
    return out


def hamiltonian(model: DenseModel, u_j) -> np.ndarray:
    """H_j = H0 + sum_k u_k(j) H_k (Eq. Hamiltonian, piecewise constant)."""
    H = model.H0.copy()
    for k, Hk in enumerate(model.Hc):
        H = H + u_j[k] * Hk
    return H

"""Pins of the Jaynes-Cummings model of the oracle (the Fig. 2 workload).

Without drive and decay, |0, e> exchanges its excitation with |1, g> at the
vacuum Rabi frequency: with H = Delta |e><e| + g (a sigma+ + a^dag sigma-) the
excited-state population is 1 - (4 g^2 / W^2) sin^2(W t / 2), W = sqrt(Delta^2
+ 4 g^2) (two-level algebra in the one-excitation subspace).  A dropped
coupling, a wrong factor or the coupling on the wrong band fails it.
"""
import math

import numpy as np

import workloads
from oracle import dense, operators


def test_vacuum_rabi_oscillation():
    g, delta = 1.3, 0.7
    phys = workloads.Physics(Q=2, N=3, chi=(0.0, 0.0), kappa=0.0, qubit_energy=(0.0, delta), g=g,
                             controls=("res_x",))
    m = operators.build(phys)
    rho0 = workloads.product_density(2, 3, 1, 0.0)[None]        # |0> (x) |e>
    W = math.sqrt(delta ** 2 + 4 * g ** 2)
    pe = np.zeros((6, 6), dtype=np.complex128)
    pe[np.arange(3) * 2 + 1, np.arange(3) * 2 + 1] = 1.0         # projector on |e>
    for T in (0.37, 1.1, 2.9):
        n_slices = 40
        u = np.zeros((n_slices, 1))
        _, rT = dense.forward(m, u, rho0, pe, T, 100)   # RK4 error ~ (h W)^4 far below the bound
        p_e = float(np.real(np.trace(pe @ rT[0])))
        assert abs(p_e - (1 - 4 * g ** 2 / W ** 2 * math.sin(W * T / 2) ** 2)) < 1e-11


def test_fig2_workload_shape():
    w = workloads.jaynes_cummings(24)
    assert (w.d, w.n_slices, w.n_states) == (24, 200, 1)
    assert abs(w.T - math.pi / 100) < 1e-15
    # initial photon number |alpha|^2 = d / 8 (truncation leaves it within 1e-6 here)
    n_op = np.diag(np.repeat(np.arange(12), 2)).astype(float)
    assert abs(np.trace(n_op @ w.rho0[0]).real - 3.0) < 1e-3
    assert w.sigma[1, 1] == 1.0 and abs(w.sigma).sum() == 1.0


def test_half_coupling_fails_the_rabi_pin():
    g, delta = 1.3, 0.7
    phys = workloads.Physics(Q=2, N=3, chi=(0.0, 0.0), kappa=0.0, qubit_energy=(0.0, delta), g=g / 2,
                             controls=("res_x",))            # the planted mistake: g halved
    m = operators.build(phys)
    rho0 = workloads.product_density(2, 3, 1, 0.0)[None]
    W = math.sqrt(delta ** 2 + 4 * g ** 2)
    pe = np.zeros((6, 6), dtype=np.complex128)
    pe[np.arange(3) * 2 + 1, np.arange(3) * 2 + 1] = 1.0
    _, rT = dense.forward(m, np.zeros((40, 1)), rho0, pe, 1.1, 100)
    p_e = float(np.real(np.trace(pe @ rT[0])))
    assert abs(p_e - (1 - 4 * g ** 2 / W ** 2 * math.sin(W * 1.1 / 2) ** 2)) > 1e-2

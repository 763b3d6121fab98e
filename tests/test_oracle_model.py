"""Pins of the oracle's model construction (oracle.operators.build) against
closed forms of the exact discrete RK4 map, with a planted mistake for each.

Each pin isolates one term of the model on a space where that term's
Lindbladian (or its dual) maps one observable or one matrix entry onto a
multiple of itself.  Then every RK4 substep multiplies it by the polynomial
P(h lam) = 1 + h lam + (h lam)^2/2 + (h lam)^3/6 + (h lam)^4/24 exactly, and
m substeps by P(h lam)^m, whatever the other entries do.  The rates lam come
from the operators as the paper writes them:

  * Kerr term K (a^dag a)^2 (Eq. kerr): -i[H, .] on the Fock coherence
    |n1><n2| gives lam = -i K (n1^2 - n2^2).  The misreading K a^dag a^dag a a
    = K n (n - 1) gives -i K (n1^2 - n1 - n2^2 + n2) instead.
  * Transmon relaxation sqrt(gamma1) b with b = sum_q sqrt(q) |q-1><q|
    (the transmon ladder of Sec. 4.2): on the top level of a Q-level ladder
    b^dag |Q-1> = 0, so L^dag |Q-1><Q-1| = -(Q-1) gamma1 |Q-1><Q-1| and the
    top population decays by P(-(Q-1) h gamma1)^m.  A ladder without sqrt(q)
    gives the rate gamma1 at every level.
  * Pure dephasing sqrt(gamma_phi) b^dag b: D[n_b] maps |q><q'| to
    -gamma_phi (q - q')^2 / 2 |q><q'|.
  * The second drive quadrature i eps (a^dag - a) of Sec. 4.2: with constant
    eps and no detuning the fixed point of every RK4 step is
    <a>* = eps / (kappa/2 + i Delta), the quadrature rotated by i against the
    a + a^dag drive (whose fixed point -i eps / (kappa/2 + i Delta) is pinned
    in test_oracle_pins.py).

Test infrastructure only.
"""
import numpy as np
import pytest

import workloads
from oracle import dense, operators


def rk_poly(z):
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


def fock_superposition(N, levels, Q=1, q=0):
    """rho = |psi><psi|, psi an equal superposition of the given Fock levels
    (transmon level q), index n Q + q."""
    psi = np.zeros(N * Q, dtype=np.complex128)
    for n in levels:
        psi[n * Q + q] = 1.0
    psi /= np.linalg.norm(psi)
    return np.outer(psi, psi.conj())


def level_superposition(Q, weights):
    psi = np.asarray(weights, dtype=np.complex128)
    psi = psi / np.linalg.norm(psi)
    return np.outer(psi, psi.conj())


def propagate(model, rho0, T, n_slices, n_rk, R):
    u = np.zeros((n_slices, R))
    return dense.propagate(model, u, rho0, T, n_rk)


# ------------------------------------------------------------------- Kerr

KERR = -0.7
KERR_T, KERR_SLICES, KERR_RK = 1.2, 3, 4


def kerr_model():
    phys = workloads.Physics(Q=1, N=6, chi=(0.0,), kerr=KERR, kappa=0.0, controls=("res_x",))
    return operators.build(phys)


def kerr_check(model):
    """Largest relative deviation of the coherences rho_{n1 n2} from the
    closed form P(-i h K (n1^2 - n2^2))^m."""
    levels = (0, 1, 3, 5)
    rho0 = fock_superposition(6, levels)
    rT = propagate(model, rho0, KERR_T, KERR_SLICES, KERR_RK, 1)
    m = KERR_SLICES * KERR_RK
    h = KERR_T / m
    worst = 0.0
    for n1 in levels:
        for n2 in levels:
            want = rho0[n1, n2] * rk_poly(-1j * h * KERR * (n1 ** 2 - n2 ** 2)) ** m
            worst = max(worst, abs(rT[n1, n2] - want) / abs(rho0[n1, n2]))
    return worst


def test_kerr_coherence_phases_follow_k_n_squared():
    assert kerr_check(kerr_model()) < 1e-13


def test_kerr_read_as_n_n_minus_1_fails_the_pin():
    m = kerr_model()
    n_op = np.diag(np.arange(6, dtype=np.complex128))
    m.H0 = m.H0 - KERR * n_op @ n_op + KERR * n_op @ (n_op - np.eye(6))
    assert kerr_check(m) > 1e-2


# ------------------------------------------------- transmon relaxation

G1 = 0.31
REL_T, REL_SLICES, REL_RK = 2.0, 4, 3


def relaxation_model(Q):
    phys = workloads.Physics(Q=Q, N=1, chi=(0.0,) * Q, kappa=0.0, gamma1=G1, controls=("qub_x",))
    return operators.build(phys)


def relaxation_check(model, Q):
    """Relative deviation of the top-level population from
    P(-(Q-1) h gamma1)^m, plus the trace drift."""
    rho0 = np.diag(np.linspace(1.0, 2.0, Q)).astype(np.complex128)
    rho0 /= np.trace(rho0)
    rT = propagate(model, rho0, REL_T, REL_SLICES, REL_RK, 1)
    m = REL_SLICES * REL_RK
    h = REL_T / m
    top = Q - 1
    want = rho0[top, top].real * rk_poly(-(Q - 1) * h * G1) ** m
    return abs(rT[top, top].real - want) / want + abs(np.trace(rT) - 1.0)


@pytest.mark.parametrize("Q", [3, 4])
def test_top_transmon_level_decays_at_q_gamma1(Q):
    assert relaxation_check(relaxation_model(Q), Q) < 1e-13


@pytest.mark.parametrize("Q", [3, 4])
def test_ladder_without_sqrt_q_fails_the_pin(monkeypatch, Q):
    def ladder_without_sqrt(n):
        a = np.zeros((n, n), dtype=np.complex128)
        for k in range(1, n):
            a[k - 1, k] = 1.0
        return a
    monkeypatch.setattr(operators, "lowering", ladder_without_sqrt)
    assert relaxation_check(relaxation_model(Q), Q) > 1e-2


# --------------------------------------------------------- dephasing

GPHI = 0.23
DEP_T, DEP_SLICES, DEP_RK = 1.5, 3, 2


def dephasing_model(Q=3):
    phys = workloads.Physics(Q=Q, N=1, chi=(0.0,) * Q, kappa=0.0, gamma_phi=GPHI,
                             controls=("qub_x",))
    return operators.build(phys)


def dephasing_check(model, Q=3):
    """Largest relative deviation of the transmon coherences rho_{q q'} from
    P(-gamma_phi (q - q')^2 h / 2)^m."""
    rho0 = level_superposition(Q, [1.0, 0.8 - 0.3j, 0.6 + 0.5j][:Q])
    rT = propagate(model, rho0, DEP_T, DEP_SLICES, DEP_RK, 1)
    m = DEP_SLICES * DEP_RK
    h = DEP_T / m
    worst = 0.0
    for q in range(Q):
        for p in range(Q):
            want = rho0[q, p] * rk_poly(-GPHI * (q - p) ** 2 * h / 2) ** m
            worst = max(worst, abs(rT[q, p] - want) / abs(rho0[q, p]))
    return worst


def test_dephasing_coherences_decay_at_gamma_phi_q_diff_squared_over_2():
    assert dephasing_check(dephasing_model()) < 1e-13


def test_dephasing_through_b_instead_of_b_dag_b_fails_the_pin():
    m = dephasing_model()
    b = operators.lowering(3)
    m.jumps = [(g, c) for g, c in m.jumps if g != GPHI] + [(GPHI, b)]
    assert dephasing_check(m) > 1e-2


def test_dephasing_through_sigma_z_like_operator_fails_the_pin():
    """b^dag b shifted by a multiple of the identity gives the same D (a
    constant drops out of D); a rescaled operator (2 b^dag b - 1, the sigma_z
    convention of a qubit carried to three levels) does not."""
    m = dephasing_model()
    nb = np.diag(np.arange(3, dtype=np.complex128))
    m.jumps = [(g, c) for g, c in m.jumps if g != GPHI] + [(GPHI, 2 * nb - np.eye(3))]
    assert dephasing_check(m) > 1e-2


# ------------------------------------------ the second drive quadrature

def quadrature_check(model, eps, delta):
    rho0 = workloads.product_density(1, 40, 0, 0.3 - 0.4j)[None]
    u = np.full((60, 1), eps)
    _, rT = dense.forward(model, u, rho0, workloads.reset_target(1, 40), 60.0, 50)
    a = operators.lowering(40)
    return abs(np.trace(a @ rT[0]) - eps / (0.5 + 1j * delta))


@pytest.mark.parametrize("delta,eps", [(0.0, 0.9), (0.7, 1.4)])
def test_res_y_drive_steady_state(delta, eps):
    phys = workloads.Physics(Q=1, N=40, chi=(0.0,), delta=delta, kappa=1.0, controls=("res_y",))
    assert quadrature_check(operators.build(phys), eps, delta) < 1e-10


def test_res_y_drive_with_flipped_sign_fails_the_pin():
    phys = workloads.Physics(Q=1, N=40, chi=(0.0,), delta=0.7, kappa=1.0, controls=("res_y",))
    m = operators.build(phys)
    m.Hc = [-H for H in m.Hc]
    assert quadrature_check(m, 1.4, 0.7) > 1e-2

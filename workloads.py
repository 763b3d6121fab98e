"""Seeded synthetic workloads shaped like the paper's resonator-reset problems.

This module holds input recipes only: physics parameters, piecewise-constant
control amplitudes, initial coherent states and the reset target.  It contains
no propagation and no Lindblad algebra, so the CUDA path and the CPU oracle can
both draw their inputs from it without sharing any of the method's arithmetic.

Basis convention (both sides follow it): a transmon with Q levels times a
resonator truncated at N Fock states, flattened "Fock x transmon" with
index i = n*Q + q (resonator index n is the slow one), d = N*Q.

Physics recipe (Sec. 4 of the paper, Eq. Hdrive, Eq. kerr, Eq. ME, and the
two-quadrature drive of Sec. 4.2), in units of kappa:
  H0   = sum_q chi_q * n * |q><q|  +  delta * n  +  kerr * n^2  +  sum_q E_q |q><q|
  H_k  = one of  res_x: a + a^dag,  res_y: i (a^dag - a),
                 qub_x: b + b^dag,  qub_y: i (b^dag - b)
  jumps sqrt(kappa) a,  sqrt(gamma1) b,  sqrt(gamma_phi) b^dag b
with a the resonator lowering operator and b = sum_q sqrt(q) |q-1><q|.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

CONTROL_SEED = 1609
PHASE_SEED = 3170

CONTROL_KINDS = ("res_x", "res_y", "qub_x", "qub_y", "rate_a", "rate_b")   # rate_*: u D[a], u D[b]


@dataclasses.dataclass(frozen=True)
class Physics:
    """Parameters of the dispersive transmon-resonator model."""
    Q: int
    N: int
    chi: Tuple[float, ...]            # dispersive shift per transmon level
    kerr: float = 0.0                 # K of Eq. (kerr)
    delta: float = 0.0                # resonator-drive detuning
    kappa: float = 1.0                # resonator decay rate
    gamma1: float = 0.0               # transmon relaxation rate
    gamma_phi: float = 0.0            # transmon pure-dephasing rate
    qubit_energy: Tuple[float, ...] = ()   # E_q per level, empty = all zero
    g: float = 0.0                    # Jaynes-Cummings coupling g (a b^dag + a^dag b) (Fig. 2 model)
    controls: Tuple[str, ...] = ("res_x", "res_y")

    @property
    def d(self) -> int:
        return self.N * self.Q

    def __post_init__(self):
        if len(self.chi) != self.Q:
            raise ValueError("chi needs one entry per transmon level")
        if self.qubit_energy and len(self.qubit_energy) != self.Q:
            raise ValueError("qubit_energy needs one entry per transmon level")
        for c in self.controls:
            if c not in CONTROL_KINDS:
                raise ValueError(f"unknown control kind {c!r}")


@dataclasses.dataclass
class Workload:
    """One open-GRAPE gradient problem with its inputs."""
    name: str
    phys: Physics
    T: float
    n_slices: int
    n_rk: int
    states: List[Tuple[int, complex]]    # (transmon level q, coherent amplitude alpha)
    u: np.ndarray                        # (n_slices, R) float64, slice-major
    rho0: np.ndarray                     # (n_states, d, d) complex128
    sigma: np.ndarray                    # (d, d) complex128, broadcast over states

    @property
    def d(self) -> int:
        return self.phys.d

    @property
    def n_states(self) -> int:
        return len(self.states)

    @property
    def n_controls(self) -> int:
        return len(self.phys.controls)

    def with_slices(self, n_slices: int, seed: Optional[int] = None) -> "Workload":
        """Same physics and states with a different number of slices (and T
        scaled so that the slice length stays the same)."""
        dt = self.T / self.n_slices
        lo, hi = float(self.u.min()), float(self.u.max())
        bound = max(abs(lo), abs(hi))
        u = controls(n_slices, self.n_controls, bound,
                     CONTROL_SEED if seed is None else seed)
        return dataclasses.replace(self, name=f"{self.name}/Nt{n_slices}",
                                   T=dt * n_slices, n_slices=n_slices, u=u)


def coherent_ket(N: int, alpha: complex) -> np.ndarray:
    """Truncated coherent state e^{-|a|^2/2} a^n / sqrt(n!), n < N, renormalised."""
    amp = np.zeros(N, dtype=np.complex128)
    amp[0] = 1.0
    for n in range(1, N):
        amp[n] = amp[n - 1] * alpha / math.sqrt(n)
    amp *= math.exp(-abs(alpha) ** 2 / 2)
    return amp / np.linalg.norm(amp)


def product_density(Q: int, N: int, q: int, alpha: complex) -> np.ndarray:
    """rho = |psi><psi| with psi = |alpha> (x) |q>, index n*Q + q."""
    psi = np.zeros(N * Q, dtype=np.complex128)
    psi[np.arange(N) * Q + q] = coherent_ket(N, alpha)
    return np.outer(psi, psi.conj())


def reset_target(Q: int, N: int) -> np.ndarray:
    """sigma = |0><0| (x) I_q: the resonator-vacuum projector of Eq. (Phi0)."""
    s = np.zeros((N * Q, N * Q), dtype=np.complex128)
    s[np.arange(Q), np.arange(Q)] = 1.0
    return s


def controls(n_slices: int, R: int, bound: float, seed: int) -> np.ndarray:
    """Piecewise-constant controls u[j, k] ~ U[-bound, bound]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-bound, bound, size=(n_slices, R)).astype(np.float64)


def make(name: str, phys: Physics, T: float, n_slices: int, n_rk: int,
         states: Sequence[Tuple[int, complex]], u_bound: float,
         control_seed: int = CONTROL_SEED) -> Workload:
    rho0 = np.stack([product_density(phys.Q, phys.N, q, a) for q, a in states])
    return Workload(name=name, phys=phys, T=T, n_slices=n_slices, n_rk=n_rk,
                    states=list(states),
                    u=controls(n_slices, len(phys.controls), u_bound, control_seed),
                    rho0=rho0, sigma=reset_target(phys.Q, phys.N))


# --------------------------------------------------------------------------
# The five problem families (sizes in the docstrings; kappa = 1 units).

def qubit_resonator_d20(n_slices: int = 200) -> Workload:
    """2-level qubit x resonator N=10 (d=20), H0 = chi n sigma_z / 2 with
    chi = kappa = 1, delta = 0, controls res_x/res_y, T = 4, N_t = 200, n_RK = 4,
    states |g>|1.5+0.5i> and |e>|1.5-0.5i>, u ~ U[-1, 1]."""
    phys = Physics(Q=2, N=10, chi=(-0.5, 0.5), kappa=1.0)
    return make("qubit_resonator_d20", phys, T=4.0 * n_slices / 200, n_slices=n_slices,
                n_rk=4, states=[(0, 1.5 + 0.5j), (1, 1.5 - 0.5j)], u_bound=1.0)


def transmon_resonator_d120(n_slices: int = 2000) -> Workload:
    """3-level transmon x resonator N=40 (d=120): chi_q = (0, 1.0, 2.6),
    Kerr -0.01, kappa 1, transmon T1 rate 0.002 and dephasing 0.001, controls
    res_x/res_y/qub_x, T = 6, N_t = 2000, n_RK = 4, one coherent state per
    transmon level with |alpha| ~ U[2, 4] and uniform phase, u ~ U[-1, 1]."""
    phys = Physics(Q=3, N=40, chi=(0.0, 1.0, 2.6), kerr=-0.01, kappa=1.0,
                   gamma1=0.002, gamma_phi=0.001,
                   controls=("res_x", "res_y", "qub_x"))
    rng = np.random.default_rng(PHASE_SEED)
    mags = rng.uniform(2.0, 4.0, size=3)
    phases = rng.uniform(0.0, 2 * math.pi, size=3)
    states = [(q, complex(mags[q] * np.exp(1j * phases[q]))) for q in range(3)]
    return make("transmon_resonator_d120", phys, T=6.0 * n_slices / 2000,
                n_slices=n_slices, n_rk=4, states=states, u_bound=1.0)


BATCH_DT = 0.003   # slice length of the batched problems (same as the d=120 problem)


def batch_problem(i: int, n_slices: Optional[int] = None) -> Workload:
    """Problem i of the 256-problem batch: N ~ U{10..60}, Q ~ U{2, 3},
    N_t ~ U{500..4000}, chi ~ U[0.5, 2] (chi_q = +-chi/2 for Q=2, q*chi for Q=3),
    jump sqrt(kappa) a only, controls res_x/res_y with u ~ U[-2, 2], one state
    per transmon level with |alpha| ~ U[0, 3]; slice length 0.003/kappa."""
    rng = np.random.default_rng(CONTROL_SEED + i)
    N = int(rng.integers(10, 61))
    Q = int(rng.integers(2, 4))
    nt = int(rng.integers(500, 4001))
    chi = float(rng.uniform(0.5, 2.0))
    mags = rng.uniform(0.0, 3.0, size=Q)
    phases = rng.uniform(0.0, 2 * math.pi, size=Q)
    chis = (-chi / 2, chi / 2) if Q == 2 else tuple(q * chi for q in range(Q))
    phys = Physics(Q=Q, N=N, chi=chis, kappa=1.0)
    if n_slices is not None:
        nt = n_slices
    states = [(q, complex(mags[q] * np.exp(1j * phases[q]))) for q in range(Q)]
    return make(f"batch{i}", phys, T=BATCH_DT * nt, n_slices=nt, n_rk=4,
                states=states, u_bound=2.0, control_seed=CONTROL_SEED + i)


def jaynes_cummings(d: int, n_slices: int = 200, n_rk: int = 1) -> Workload:
    """The scaling workload of Fig. 2: a qubit (Q=2) coupled to a cavity of
    N = d/2 levels by a Jaynes-Cummings interaction g = 100 kappa, qubit
    detuning Delta = 10 kappa (drive resonant with the cavity), cavity
    quadrature controls, initial |alpha> (x) |e> with alpha = sqrt(d/8),
    target |0> (x) |e>, T = pi / g over N_t = 200 slices, one state."""
    if d % 2:
        raise ValueError("d must be even (qubit x cavity)")
    g = 100.0
    phys = Physics(Q=2, N=d // 2, chi=(0.0, 0.0), kappa=1.0, qubit_energy=(0.0, 10.0), g=g)
    w = make(f"jaynes_cummings_d{d}", phys, T=math.pi / g, n_slices=n_slices, n_rk=n_rk,
             states=[(1, complex(math.sqrt(d / 8.0)))], u_bound=1.0)
    sigma = np.zeros((d, d), dtype=np.complex128)
    sigma[1, 1] = 1.0                 # |0> (x) |e>: index n Q + q = 1
    w.sigma = sigma
    return w


def transmon_resonator_d600(n_slices: int = 40000) -> Workload:
    """4-level transmon x resonator N=150 (d=600): chi_q = (0, 1, 2.2, 3.6),
    Kerr -0.005, jump sqrt(kappa) a, controls res_x/res_y, N_t = 40000,
    n_RK = 4, one state |1>|alpha=2>, slice length 1.5e-4/kappa (T = 6)."""
    phys = Physics(Q=4, N=150, chi=(0.0, 1.0, 2.2, 3.6), kerr=-0.005, kappa=1.0)
    return make("transmon_resonator_d600", phys, T=6.0 * n_slices / 40000,
                n_slices=n_slices, n_rk=4, states=[(1, 2.0 + 0.0j)], u_bound=1.0)


def small(Q: int = 2, N: int = 4, n_slices: int = 6, n_rk: int = 2, T: float = 0.6,
          controls_=("res_x", "res_y"), kerr: float = -0.05, gamma1: float = 0.0,
          gamma_phi: float = 0.0, chi: Optional[Tuple[float, ...]] = None,
          seed: int = CONTROL_SEED, u_bound: float = 1.0) -> Workload:
    """A tiny problem for brute-force checks (d = N*Q)."""
    if chi is None:
        chi = tuple(0.7 * q - 0.3 for q in range(Q))
    phys = Physics(Q=Q, N=N, chi=chi, kerr=kerr, kappa=1.0, gamma1=gamma1,
                   gamma_phi=gamma_phi, controls=tuple(controls_))
    rng = np.random.default_rng(seed + 7)
    states = [(q, complex(rng.uniform(0.3, 1.0) * np.exp(1j * rng.uniform(0, 6.28))))
              for q in range(Q)]
    return make(f"small_Q{Q}N{N}", phys, T=T, n_slices=n_slices, n_rk=n_rk,
                states=states, u_bound=u_bound, control_seed=seed)

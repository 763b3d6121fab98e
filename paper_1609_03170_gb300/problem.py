"""Open-GRAPE problems as banded operators, and the Python front end of the C ABI.

``band_model(phys)`` writes the dispersive transmon-resonator model (Eq.
Hdrive with sigma_z replaced by a per-level shift, Eq. kerr, Eq. ME, the
two-quadrature drive of Sec. 4.2) directly as DIA bands in the basis
i = n*Q + q: the resonator operators a, a^dag sit on offsets +-Q, the
transmon ladder b, b^dag on +-1 and every number operator on the diagonal.

``GrapeProblem`` owns one ``grape_problem_t`` and marshals arguments for
``grape_forward`` / ``grape_gradient``: numpy inputs are passed as host
pointers, CUDA torch tensors as device pointers (outputs then stay on the
device).  All computation happens in libgrape.so.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import _lib


@dataclasses.dataclass
class BandOp:
    """Op[i][i + offsets[b]] = values[b, i]."""
    offsets: np.ndarray     # int32 [n_diag]
    values: np.ndarray      # complex128 [n_diag, d]

    @staticmethod
    def make(d: int, bands: Sequence[Tuple[int, np.ndarray]]) -> "BandOp":
        bands = [(o, v) for o, v in bands if -d < o < d]     # bands outside the matrix are empty
        offs = np.array([o for o, _ in bands], dtype=np.int32)
        vals = np.zeros((len(bands), d), dtype=np.complex128)
        for b, (_, v) in enumerate(bands):
            vals[b] = v
        return BandOp(offs, vals)


@dataclasses.dataclass
class BandModel:
    d: int
    H0: BandOp
    Hc: List[BandOp]
    jumps: List[BandOp]
    rates: np.ndarray
    # per jump: -1 fixed rate, k: the rate is rates[m] * u_k (a control on a
    # dissipation rate, whose Hc[k] is empty)
    jump_control: Optional[List[int]] = None


def band_model(phys) -> BandModel:
    Q, N = phys.Q, phys.N
    d = Q * N
    i = np.arange(d)
    n = i // Q
    q = i % Q
    up_res = np.where(n + 1 < N, np.sqrt(n + 1.0), 0.0)      # a[i][i+Q]
    dn_res = np.sqrt(n.astype(float))                         # a^dag[i][i-Q]
    up_qub = np.where(q + 1 < Q, np.sqrt(q + 1.0), 0.0)      # b[i][i+1]
    dn_qub = np.sqrt(q.astype(float))                         # b^dag[i][i-1]

    chi = np.asarray(phys.chi, dtype=float)[q]
    diag = chi * n + phys.delta * n + phys.kerr * n.astype(float) ** 2
    if phys.qubit_energy:
        diag = diag + np.asarray(phys.qubit_energy, dtype=float)[q]
    h0 = [(0, diag.astype(np.complex128))]
    if getattr(phys, "g", 0.0):
        # g (a b^dag + a^dag b): row (n, q) <- (n+1, q-1) at offset Q-1 and
        # <- (n-1, q+1) at offset -(Q-1)
        ab = np.where((n + 1 < N) & (q >= 1), np.sqrt(n + 1.0) * np.sqrt(q.astype(float)), 0.0)
        ba = np.where((n >= 1) & (q + 1 < Q), np.sqrt(n.astype(float)) * np.sqrt(q + 1.0), 0.0)
        h0 += [(Q - 1, phys.g * ab + 0j), (-(Q - 1), phys.g * ba + 0j)]
    H0 = BandOp.make(d, h0)

    kinds = {
        "res_x": [(Q, up_res + 0j), (-Q, dn_res + 0j)],
        "res_y": [(Q, -1j * up_res), (-Q, 1j * dn_res)],
        "qub_x": [(1, up_qub + 0j), (-1, dn_qub + 0j)],
        "qub_y": [(1, -1j * up_qub), (-1, 1j * dn_qub)],
    }
    rate_ops = {"rate_a": [(Q, up_res + 0j)], "rate_b": [(1, up_qub + 0j)]}   # u D[a], u D[b]
    Hc = [BandOp.make(d, [] if k in rate_ops else kinds[k]) for k in phys.controls]

    jumps, rates = [BandOp.make(d, [(Q, up_res + 0j)])], [phys.kappa]
    if phys.gamma1:
        jumps.append(BandOp.make(d, [(1, up_qub + 0j)])); rates.append(phys.gamma1)
    if phys.gamma_phi:
        jumps.append(BandOp.make(d, [(0, q.astype(np.complex128))])); rates.append(phys.gamma_phi)
    jc = [-1] * len(jumps)
    for k, name in enumerate(phys.controls):
        if name in rate_ops:
            jumps.append(BandOp.make(d, rate_ops[name])); rates.append(1.0); jc.append(k)
    return BandModel(d=d, H0=H0, Hc=Hc, jumps=jumps, rates=np.array(rates, dtype=np.float64),
                     jump_control=jc if any(c >= 0 for c in jc) else None)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    return int(getattr(stream, "cuda_stream", stream))


class GrapeProblem:
    """One open-GRAPE gradient problem resident on the current CUDA device."""

    def __init__(self, model: BandModel, rho0: np.ndarray, sigma: np.ndarray, T: float,
                 n_slices: int, n_rk: int, grad_mode: int = _lib.GRAPE_GRAD_EXACT,
                 ckpt_stride: int = 0, precision: int = _lib.GRAPE_PREC_DF64):
        _lib.load()
        d = model.d
        rho0 = np.ascontiguousarray(rho0, dtype=np.complex128)
        sigma = np.ascontiguousarray(sigma, dtype=np.complex128)
        if rho0.ndim == 2:
            rho0 = rho0[None]
        self.d, self.n_states = d, rho0.shape[0]
        self.n_slices, self.n_rk, self.T = int(n_slices), int(n_rk), float(T)
        self.R = len(model.Hc)
        keep = []

        def band(op: BandOp) -> _lib.grape_band_op:
            offs = np.ascontiguousarray(op.offsets, dtype=np.int32)
            vals = np.ascontiguousarray(op.values, dtype=np.complex128).view(np.float64)
            keep.extend([offs, vals])
            return _lib.grape_band_op(len(offs), offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      _dptr(vals))

        Hc = (_lib.grape_band_op * max(1, self.R))(*[band(h) for h in model.Hc])
        J = len(model.jumps)
        jumps = (_lib.grape_band_op * max(1, J))(*[band(c) for c in model.jumps])
        rates = np.ascontiguousarray(model.rates, dtype=np.float64)
        rho_f = rho0.view(np.float64)
        sig_f = sigma.view(np.float64)
        jc = None
        if model.jump_control is not None:
            jc_arr = np.ascontiguousarray(model.jump_control, dtype=np.int32)
            keep.append(jc_arr)
            jc = jc_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        desc = _lib.grape_problem_desc(
            d, self.R, J, self.n_states, self.n_slices, self.n_rk, self.T,
            band(model.H0), Hc, jumps, _dptr(rates), _dptr(rho_f), _dptr(sig_f),
            1 if sigma.ndim == 2 else 0, int(grad_mode), int(ckpt_stride), int(precision), jc)
        self.precision = int(precision)
        self._h = _lib.grape_problem_create(desc)
        del keep

    @classmethod
    def from_workload(cls, w, grad_mode: int = _lib.GRAPE_GRAD_EXACT, ckpt_stride: int = 0,
                      precision: int = _lib.GRAPE_PREC_DF64):
        return cls(band_model(w.phys), w.rho0, w.sigma, w.T, w.n_slices, w.n_rk,
                   grad_mode=grad_mode, ckpt_stride=ckpt_stride, precision=precision)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _lib.grape_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- queries ----------------------------------------------------------
    @property
    def handle(self):
        return self._h

    def memory_bytes(self) -> int:
        return _lib.grape_problem_memory(self._h)

    def geometry(self):
        return _lib.grape_problem_geometry(self._h)

    def set_penalty(self, diag, beta: float) -> None:
        """Phi = Phi_0 - beta dt sum_n Re Tr(A rho_n) for A = diag(diag)
        (App. B); diag=None removes it."""
        if diag is not None and len(diag) != self.d:
            raise ValueError(f"diag needs {self.d} values")
        _lib.grape_problem_set_penalty(self._h, diag, beta)

    def set_photon_penalty(self, Q: int, N: int, beta: float) -> None:
        """The paper's photon-number penalty, A = a^dag a in the basis i = n Q + q."""
        self.set_penalty(np.repeat(np.arange(N, dtype=np.float64), Q), beta)

    def set_tile(self, cluster: int, threads: int) -> None:
        """Cluster width and threads per CTA of the propagation kernel
        (results do not change, bit for bit)."""
        _lib.grape_problem_set_tile(self._h, cluster, threads)

    def gradient_launches(self) -> int:
        return _lib.grape_gradient_launches(self._h)

    def kernel(self) -> str:
        """hermitian-cluster, full-cluster or grid."""
        return _lib.grape_problem_kernel(self._h)

    def status(self) -> None:
        """Raise GrapeError(GRAPE_ETIMEOUT) if a grid barrier gave up."""
        _lib.grape_problem_status(self._h)

    def set_profiling(self, on: bool = True) -> None:
        _lib.grape_set_profiling(self._h, on)

    def phase_times(self):
        return _lib.grape_phase_times(self._h)

    # -- compute ----------------------------------------------------------
    def forward(self, u, stream=None, want_rho=True):
        """Phi and rho(T).  numpy u -> numpy results; CUDA tensor u -> CUDA tensors."""
        if _is_cuda(u):
            import torch
            F = torch.empty(1, dtype=torch.float64, device=u.device)
            rho = (torch.empty((self.n_states, self.d, self.d), dtype=torch.complex128,
                               device=u.device) if want_rho else None)
            _lib.grape_forward(self._h, u.data_ptr(), F.data_ptr(),
                               rho.data_ptr() if rho is not None else 0, _stream_ptr(stream))
            return F, rho
        u = np.ascontiguousarray(u, dtype=np.float64)
        F = np.zeros(1)
        rho = np.zeros((self.n_states, self.d, self.d), dtype=np.complex128) if want_rho else None
        _lib.grape_forward(self._h, u.ctypes.data, F.ctypes.data,
                           rho.ctypes.data if rho is not None else 0, _stream_ptr(stream))
        return float(F[0]), rho

    def gradient(self, u, stream=None, out=None):
        """Phi and dPhi/du (n_slices x R)."""
        if _is_cuda(u):
            import torch
            F = torch.empty(1, dtype=torch.float64, device=u.device)
            G = out if out is not None else torch.empty((self.n_slices, self.R),
                                                        dtype=torch.float64, device=u.device)
            _lib.grape_gradient(self._h, u.data_ptr(), F.data_ptr(), G.data_ptr(),
                                _stream_ptr(stream))
            return F, G
        u = np.ascontiguousarray(u, dtype=np.float64)
        F = np.zeros(1)
        G = np.zeros((self.n_slices, self.R))
        _lib.grape_gradient(self._h, u.ctypes.data, F.ctypes.data, G.ctypes.data,
                            _stream_ptr(stream))
        return float(F[0]), G


    def gradient_filtered(self, u, omega0, stream=None):
        """Phi and dPhi/du for n_steps Gaussian-filtered controls u
        (n_steps x R); the problem's slices are the subpixels (App. A)."""
        n_steps = int(u.shape[0])
        if _is_cuda(u):
            import torch
            F = torch.empty(1, dtype=torch.float64, device=u.device)
            G = torch.empty((n_steps, self.R), dtype=torch.float64, device=u.device)
            _lib.grape_gradient_filtered(self._h, n_steps, self.R, omega0, u.data_ptr(),
                                         F.data_ptr(), G.data_ptr(), _stream_ptr(stream))
            return F, G
        u = np.ascontiguousarray(u, dtype=np.float64)
        F = np.zeros(1)
        G = np.zeros((n_steps, self.R))
        _lib.grape_gradient_filtered(self._h, n_steps, self.R, omega0, u.ctypes.data,
                                     F.ctypes.data, G.ctypes.data, _stream_ptr(stream))
        return float(F[0]), G


class GaussianFilter:
    """Gaussian filter of the controls (App. A) on CUDA tensors: n_steps
    controls over [0, T) -> n_sub subpixels, and the transposed map for
    gradients.  omega0: one reference bandwidth per control (or one for all)."""

    def __init__(self, n_steps: int, n_sub: int, T: float, omega0, n_controls: int):
        self.n_steps, self.n_sub, self.R = int(n_steps), int(n_sub), int(n_controls)
        self.Dt, self.dt = T / n_steps, T / n_sub
        self.omega0 = list(omega0) if hasattr(omega0, "__len__") else [float(omega0)] * self.R

    @staticmethod
    def omega0_from_bandwidth(omega_b: float) -> float:
        """w0 = wB / sqrt(-ln(1/sqrt 2)) for a 3 dB bandwidth wB."""
        return omega_b / np.sqrt(-np.log(1.0 / np.sqrt(2.0)))

    def apply(self, u, stream=None):
        import torch
        s = torch.empty((self.n_sub, self.R), dtype=torch.float64, device=u.device)
        _lib.grape_filter_apply(self.n_steps, self.n_sub, self.R, self.Dt, self.dt, self.omega0,
                                u.contiguous().data_ptr(), s.data_ptr(), _stream_ptr(stream))
        return s

    def adjoint(self, g_s, stream=None):
        import torch
        g_u = torch.empty((self.n_steps, self.R), dtype=torch.float64, device=g_s.device)
        _lib.grape_filter_adjoint(self.n_steps, self.n_sub, self.R, self.Dt, self.dt, self.omega0,
                                  g_s.contiguous().data_ptr(), g_u.data_ptr(), _stream_ptr(stream))
        return g_u


class GrapeBatch:
    """Many GrapeProblems evaluated by one batched, graph-captured launch
    (grape_batch_gradient).  Inputs and outputs are CUDA tensors."""

    def __init__(self, problems, n_lanes: int = 0):
        self.problems = list(problems)
        self._h = _lib.grape_batch_create([p.handle for p in self.problems], n_lanes)

    def close(self):
        if getattr(self, "_h", None):
            _lib.grape_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        """(lanes, scratch bytes, kernel launches per call)."""
        return _lib.grape_batch_info(self._h)

    def gradient(self, us, F=None, grads=None, stream=None):
        import torch
        dev = us[0].device
        if F is None:
            F = torch.empty(len(self.problems), dtype=torch.float64, device=dev)
        if grads is None:
            grads = [torch.empty((p.n_slices, p.R), dtype=torch.float64, device=dev)
                     for p in self.problems]
        _lib.grape_batch_gradient(self._h, [u.data_ptr() for u in us], F.data_ptr(),
                                  [g.data_ptr() for g in grads], _stream_ptr(stream))
        return F, grads


class GrapeServer:
    """Pulse-optimisation service (grape_server_*): submit jobs, poll results.

    Each job maximises Phi of one GrapeProblem with projected L-BFGS on the
    device; jobs are admitted by device memory and run with continuous
    batching (see include/grape.h)."""

    def __init__(self, budget_bytes: int = 0, max_slots: int = 16):
        self._h = _lib.grape_server_create(budget_bytes, max_slots)
        self._shapes = {}

    def close(self):
        if getattr(self, "_h", None):
            _lib.grape_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, problem: "GrapeProblem", u0, max_iters=50, lbfgs_m=10, u_min=-5.0,
               u_max=5.0, step0=0.5, tol=0.0) -> int:
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        prm = _lib.grape_opt_params(int(max_iters), int(lbfgs_m), float(u_min), float(u_max),
                                    float(step0), float(tol))
        t = _lib.grape_submit(self._h, problem.handle, u0, prm)
        self._shapes[t] = u0.shape
        return t

    def poll(self, ticket: int, timeout_s: float = 0.0):
        """None while the job runs, else (u_best, Phi, evaluations, queued_s, latency_s)."""
        shape = self._shapes[ticket]
        u = np.zeros(shape)
        F = np.zeros(1)
        info = _lib.grape_job_info()
        if not _lib.grape_poll(self._h, ticket, int(timeout_s * 1e6), u, F, info):
            return None
        del self._shapes[ticket]
        return u, float(F[0]), int(info.evaluations), info.queued_us * 1e-6, info.latency_us * 1e-6

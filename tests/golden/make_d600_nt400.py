"""Writes d600_nt400.json: the plain-C FP64 oracle's Phi, gradient and a
sample of rho(T) for the 4-level transmon x N=150 resonator problem (d=600)
at N_t = 400 slices, n_RK = 4 (the workload transmon_resonator_d600 with 400
slices: chi_q = (0, 1, 2.2, 3.6), Kerr -0.005, jump sqrt(kappa) a, controls
a + a^dag and i(a^dag - a), one state |1>|alpha=2>, slice length
1.5e-4/kappa).  Exact discrete adjoint gradient (Sec. 3, Eq. dphidu).

The oracle needs several minutes on one host core for this size, longer than
a GPU test should wait, so the GPU parity test of the checkpointed d=600
path reads the values from this file.  Everything here comes from oracle/
(no value from the CUDA path).  Run from the repository root:

    python tests/golden/make_d600_nt400.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import sparse  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "d600_nt400.json")


def rho_sample_indices(d):
    """The diagonal and the first two super-diagonals of rho(T) (the entries
    the coherent state and the drive populate most), plus every 37th entry of
    the flat upper triangle."""
    idx = [(i, i) for i in range(d)] + [(i, i + 1) for i in range(d - 1)]
    idx += [(i, i + 2) for i in range(d - 2)]
    up = [(i, j) for i in range(d) for j in range(i, d)]
    idx += up[::37]
    return sorted(set(idx))


def main():
    w = workloads.transmon_resonator_d600(n_slices=400)
    F, G, rT, secs = sparse.run_workload(w, mode=sparse.MODE_EXACT, threads=1)
    idx = rho_sample_indices(w.d)
    r = rT[0]
    out = {
        "what": "oracle (grape_oracle.c, FP64) on transmon_resonator_d600(n_slices=400), exact gradient",
        "d": w.d, "n_slices": w.n_slices, "n_rk": w.n_rk, "T": w.T,
        "oracle_seconds": secs,
        "F": F,
        "grad": G.tolist(),
        "rho_index": idx,
        "rho_re": [float(r[i, j].real) for i, j in idx],
        "rho_im": [float(r[i, j].imag) for i, j in idx],
    }
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(f"wrote {OUT}: Phi = {F!r}, {len(idx)} rho entries, oracle {secs:.0f} s")


if __name__ == "__main__":
    main()

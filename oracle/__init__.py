"""FP64 CPU oracle of open GRAPE with Runge-Kutta propagation (arXiv:1609.03170).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only the tests, the smoke check of
``__graft_entry__`` and the CPU-baseline / reference arm of ``bench.py`` use it.
It shares no code with the CUDA path; the two meet only through the seeded
inputs of ``workloads.py``.

Modules
  operators  dense operators built from the physics parameters (Eq. Hdrive,
             Eq. kerr, Eq. ME, Sec. 4.2 two-quadrature drive)
  dense      Lindblad map (Eq. master, Eq. disspation) and its dual, RK4
             forward propagation (Sec. 3, Eq. rkmaster), cost (Eq. phi), the
             exact discrete adjoint gradient, the paper's first-order gradient
             (Eq. dphidu), central finite differences
  liouville  the "standard" d^2 x d^2 Liouville-space formulation (Sec. 2.2,
             Eq. Cexp): superoperator, RK4 polynomial, matrix exponential and
             block-matrix Frechet derivatives for exact gradients
  sparse     ctypes front end of grape_oracle.c, the same algorithm in plain C
             with sparse operators, for sizes the dense code cannot reach
  filter     Gaussian filtering of the controls and its chain rule (App. A)
  penalty    photon-number penalty Phi_0 - beta Phi_p and its gradient through
             the modified backward evolution (Sec. 5, App. B)
  lbfgs      projected L-BFGS steps of the serving optimiser

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, brute force and independent formulations.
"""

"""Projected L-BFGS reference (test infrastructure only).

The paper updates the controls with BFGS (Sec. 2.1, Eq. update: u <- u + B
grad Phi with B an inverse-Hessian estimate).  This is the plain form of the
projected limited-memory variant the serving loop runs on the device,
written step by step: minimise f = -Phi over lo <= u <= hi; every iteration
evaluates f and its gradient at a trial point; a trial that lowers f is
accepted (and its curvature pair s = u_new - u, y = g_new - g stored when
s.y is positive), otherwise the step multiplier is halved; the next trial
is u + step * d clamped to the box.  The direction comes from the two-loop
recursion d = -H q applied to the projected gradient q (g with the
components zeroed whose variable sits on a bound that the gradient pushes
against), initial scaling s.y / y.y of the newest pair or step0 / max|q|
before any pair; those bound components of d are zeroed, and when d is not a
descent direction (d.q >= 0) the scaled -q is used instead.
"""
from __future__ import annotations

import numpy as np


def minimise(fg, u0, lo, hi, max_evals=50, m=10, step0=0.5, tol=0.0):
    """fg(u) -> (f, g).  Returns (u_best, f_best, evaluations)."""
    u = None
    g = None
    f = None
    ut = np.clip(np.asarray(u0, dtype=np.float64).ravel(), lo, hi)
    S, Y, rho = [], [], []
    gamma = 1.0
    step = 1.0
    evals = 0
    while True:
        ft, gt = fg(ut)
        gt = np.asarray(gt, dtype=np.float64).ravel()
        if evals == 0 or ft < f:
            if evals > 0:
                s = ut - u
                y = gt - g
                sy = float(np.dot(s, y))
                if sy > 1e-12 * np.sqrt(float(np.dot(s, s)) * float(np.dot(y, y))):
                    S.append(s); Y.append(y); rho.append(1.0 / sy)
                    gamma = sy / float(np.dot(y, y))
                    if len(S) > m:
                        S.pop(0); Y.pop(0); rho.pop(0)
            u, f, g = ut.copy(), ft, gt
            step = 1.0
        else:
            step *= 0.5
        evals += 1
        pg = np.max(np.abs(np.clip(u - g, lo, hi) - u)) if u.size else 0.0
        if evals >= max_evals or pg <= tol or step < 1e-10:
            return u, f, evals
        active = ((u <= lo) & (g > 0)) | ((u >= hi) & (g < 0))
        q = np.where(active, 0.0, g)
        q0 = q.copy()
        alpha = [0.0] * len(S)
        for t in reversed(range(len(S))):
            alpha[t] = rho[t] * float(np.dot(S[t], q))
            q -= alpha[t] * Y[t]
        gmax = np.max(np.abs(q0))
        scale = gamma if S else ((step0 / gmax) if gmax > 0 else 0.0)
        q *= scale
        for t in range(len(S)):
            b = rho[t] * float(np.dot(Y[t], q))
            q += (alpha[t] - b) * S[t]
        d = -q
        d[active] = 0.0
        if float(np.dot(d, q0)) >= 0.0:
            d = -scale * q0
        ut = np.clip(u + step * d, lo, hi)

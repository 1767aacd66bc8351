"""Plain FP64 Newton-GMRES for the oracle (numpy).

TEST INFRASTRUCTURE ONLY.  Newton with backtracking line search (the paper solves the
nonlinear system with PETSc's Newton line-search class, appendix "Details of solver
selection"), and the linear steps with restarted, right-preconditioned GMRES(m): Arnoldi
with modified Gram-Schmidt, Givens rotations on the Hessenberg matrix (Saad & Schultz 1986).
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b, x0=None, m=50, rtol=1e-8, atol=0.0, maxiter=1000, precond=None):
    """Solve A x = b.  Returns (x, iterations, residual history)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.astype(np.float64).copy()
    M = precond if precond is not None else (lambda z: z)
    bnorm = np.linalg.norm(b)
    target = max(rtol * bnorm, atol)
    hist = []
    its = 0
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta)
        if beta <= target or its >= maxiter:
            return x, its, hist
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(m):
            Z[k] = M(V[k])
            w = matvec(Z[k])
            for i in range(k + 1):                      # modified Gram-Schmidt
                H[i, k] = np.dot(w, V[i])
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):                          # previous rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / den if den > 0 else 1.0
            sn[k] = H[k + 1, k] / den if den > 0 else 0.0
            H[k, k] = cs[k] * H[k, k] + sn[k] * H[k + 1, k]
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            its += 1
            k_done = k + 1
            hist.append(abs(g[k + 1]))
            if abs(g[k + 1]) <= target or its >= maxiter:
                break
        y = np.zeros(k_done)
        for i in range(k_done - 1, -1, -1):             # back substitution
            y[i] = (g[i] - np.dot(H[i, i + 1:k_done], y[i + 1:k_done])) / H[i, i]
        x = x + Z[:k_done].T @ y


def newton(residual, jvp, u0, rtol=1e-8, atol=0.0, max_newton=20, gmres_m=50, gmres_rtol=1e-3, gmres_maxiter=2000,
           precond_factory=None, line_search=True):
    """Solve residual(u) = 0 to ||R|| <= max(rtol ||R_0||, atol).  jvp(u, v) = J(u) v.
    precond_factory(u) -> callable applying an approximate inverse of J(u), or None.
    Returns (u, stats)."""
    u = u0.astype(np.float64).copy()
    R = residual(u)
    r0 = np.linalg.norm(R)
    hist = [r0]
    gm_its = []
    target = max(rtol * r0, atol)
    for it in range(max_newton):
        if hist[-1] <= target:
            break
        P = precond_factory(u) if precond_factory is not None else None
        du, k, _ = gmres(lambda z: jvp(u, z), -R, m=gmres_m, rtol=gmres_rtol, maxiter=gmres_maxiter, precond=P)
        gm_its.append(k)
        lam, f0 = 1.0, hist[-1]
        while True:                                     # Armijo backtracking, c = 1e-4, halving
            un = u + lam * du
            Rn = residual(un)
            fn = np.linalg.norm(Rn)
            if not line_search or fn <= (1.0 - 1e-4 * lam) * f0 or lam < 2.0 ** -10:
                break
            lam *= 0.5
        u, R = un, Rn
        hist.append(fn)
    return u, {"newton_its": len(hist) - 1, "gmres_its": gm_its, "res_hist": hist,
               "converged": hist[-1] <= target}

"""Restarted GMRES (right preconditioned) and flexible GMRES.

The paper solves each tangent system of Eq. (tangent problem) with GMRES
preconditioned by BDDC (Sections 1-2) and states neither restart nor
orthogonalisation; this oracle uses restart m = 100, modified Gram-Schmidt
and Givens rotations (Saad, Iterative Methods, Alg. 6.9 / 9.5 in words):

* Arnoldi on A M^-1 from v_1 = r_0 / ||r_0||;
* the least-squares residual |g_{j+1}| after j+1 steps is the true residual
  norm of x_0 + M^-1 V y (right preconditioning) or x_0 + Z y (flexible);
* stop when it falls to tol * ||b||, then recompute the true residual.
"""
import numpy as np


def gmres(matvec, b, precond=None, tol=1e-8, restart=100, maxiter=2000,
          x0=None, flexible=False):
    """Returns (x, iterations, history of relative residual estimates)."""
    b = np.asarray(b, dtype=float)
    n = b.size
    M = precond if precond is not None else (lambda v: v)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return np.zeros(n), 0, hist
    its = 0
    while its < maxiter:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm:
            break
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n)) if flexible else None
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            z = M(V[j])
            if flexible:
                Z[j] = z
            w = matvec(z)
            for i in range(j + 1):               # modified Gram-Schmidt
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                   # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or its >= maxiter:
                break
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):      # back substitution
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        if flexible:
            x = x + Z[:j_done].T @ y
        else:
            x = x + M(V[:j_done].T @ y)
        if hist[-1] <= tol:
            break
    return x, its, hist

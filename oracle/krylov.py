"""Restarted flexible GMRES with right preconditioning, FP64 (Sec. 4; FGMRES
is the outer solver and the Krylov accelerator the paper wraps around its
preconditioners).  Saad's flexible variant keeps the preconditioned vectors
z_j so the solution is x0 + Z y.  Arnoldi by modified Gram-Schmidt; the
least-squares problem is updated by Givens rotations.  A cycle ends when the
rotated residual estimate reaches rtol * ||b||; the true residual
||b - K x|| is then recomputed and, if it is still above rtol * ||b||, the
method restarts from the current x.
"""
import numpy as np


def fgmres(K, b, precond, x0=None, rtol=1e-8, restart=30, maxit=1000, history=None):
    """Solve K x = b.  Returns (x, iterations, true relative residual)."""
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), 0, 0.0
    its = 0
    while True:
        r = b - K @ x
        beta = np.linalg.norm(r)
        if history is not None:
            history.append(beta / bnorm)
        if beta <= rtol * bnorm or its >= maxit:
            return x, its, beta / bnorm
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = K @ Z[j]
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] <= 1e-14 * max(abs(H[: j + 1, j]).max(), 1e-300)
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
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
            k = j + 1
            if history is not None:
                history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm or breakdown or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k]) if k else np.zeros(0)
        x = x + Z[:k].T @ y
        if history is not None:
            history.pop()  # the restart records the true residual instead


def gmres_identity(K, b, rtol=1e-14, restart=None):
    """Unpreconditioned GMRES, the special case precond = identity."""
    return fgmres(K, b, lambda v: v.copy(), rtol=rtol, restart=restart or b.size, maxit=10 * b.size)

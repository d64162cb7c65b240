"""Dense LU and a plain restarted GMRES (FP64) for oracle solves (Sec. V: GMRES, rel. residual)."""

import numpy as np


def lu_solve(Z, b):
    return np.linalg.solve(Z, b)


def gmres(matvec, b, tol=1e-6, restart=100, maxiter=2000, precond=None):
    """Right-preconditioned restarted GMRES with modified Gram-Schmidt; returns (x, iters, relres)."""
    n = len(b)
    x = np.zeros(n, dtype=np.complex128)
    bn = np.linalg.norm(b)
    if bn == 0:
        return x, 0, 0.0
    M = precond if precond is not None else (lambda v: v)
    it = 0
    while it < maxiter:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta / bn <= tol:
            return x, it, beta / bn
        V = [r / beta]
        Zs = []
        Hm = np.zeros((restart + 1, restart), dtype=np.complex128)
        j = 0
        for j in range(restart):
            z = M(V[j])
            Zs.append(z)
            w = matvec(z)
            for i in range(j + 1):
                Hm[i, j] = np.vdot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            it += 1
            e1 = np.zeros(j + 2, dtype=np.complex128)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(Hm[:j + 2, :j + 1], e1, rcond=None)
            res = np.linalg.norm(Hm[:j + 2, :j + 1] @ y - e1)
            if res / bn <= tol or Hm[j + 1, j] == 0 or it >= maxiter:
                break
            V.append(w / Hm[j + 1, j])
        x = x + sum(y[i] * Zs[i] for i in range(len(y)))
    r = b - matvec(x)
    return x, it, np.linalg.norm(r) / bn

"""Right-preconditioned restarted GMRES in FP64 (the Section 5 solver).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper states only GMRES with a relative-residual tolerance and a restart
length.  Reading: right preconditioning (A M y = f, u = M y), x0 = 0, Arnoldi
by modified Gram-Schmidt, Givens rotations on the Hessenberg matrix, each
right-hand side solved independently; a cycle stops early when the Arnoldi
residual estimate reaches tol and the run stops when the true relative
residual ||f - A u|| / ||f|| reaches tol (checked after every cycle).
"""
from __future__ import annotations

import numpy as np


def gmres(apply_A, apply_M, f: np.ndarray, tol: float = 1e-6, restart: int = 30,
          maxit: int = 300):
    """Solve A u = f for one right-hand side (any array shape).

    Returns (u, iterations, relres_history) with relres the true residual
    after each cycle.
    """
    f = np.asarray(f, dtype=np.complex128)
    shape = f.shape
    fv = f.ravel()
    fnorm = np.linalg.norm(fv)
    u = np.zeros_like(fv)
    if fnorm == 0.0:
        return u.reshape(shape), 0, [0.0]
    A = lambda x: np.asarray(apply_A(x.reshape(shape))).ravel()   # noqa: E731
    Mp = lambda x: np.asarray(apply_M(x.reshape(shape))).ravel()  # noqa: E731
    r = fv.copy()
    beta = fnorm
    its = 0
    hist = []
    while its < maxit:
        m = min(restart, maxit - its)
        V = np.zeros((m + 1, fv.size), dtype=np.complex128)
        Z = np.zeros((m, fv.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_used = 0
        for j in range(m):
            Z[j] = Mp(V[j])
            w = A(Z[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            if den == 0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j] = a / den
                sn[j] = bb / den
                cs[j], sn[j] = np.conj(cs[j]), np.conj(sn[j])
            H[j, j] = cs[j] * a + sn[j] * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_used = j + 1
            if abs(g[j + 1]) / fnorm <= tol:
                break
        y = np.linalg.solve(np.triu(H[:j_used, :j_used]), g[:j_used])
        u = u + y @ Z[:j_used]
        r = fv - A(u)
        beta = np.linalg.norm(r)
        hist.append(beta / fnorm)
        if beta / fnorm <= tol:
            break
    return u.reshape(shape), its, hist

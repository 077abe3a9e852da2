"""Exact block LDU ("sweeping factorization") of Section 3, dense plane blocks.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A is block tridiagonal along x3 with blocks A_{m,m'} acting on whole planes.
S_1 = A_11, S_m = A_mm - A_{m,m-1} T_{m-1} A_{m-1,m}, T_m = S_m^{-1}, and
u = U_1^{-1}..U_{n-1}^{-1} diag(T) L_{n-1}^{-1}..L_1^{-1} f.  Only for tiny
grids (the blocks are dense N^2 x N^2).
"""
from __future__ import annotations

import numpy as np


def plane_blocks(A, N: int):
    """Dense plane blocks of A (natural order, planes of N*N unknowns)."""
    P = N * N
    Ad = A.toarray()
    diag = [Ad[m * P:(m + 1) * P, m * P:(m + 1) * P] for m in range(N)]
    lower = [None] + [Ad[m * P:(m + 1) * P, (m - 1) * P:m * P] for m in range(1, N)]
    upper = [Ad[m * P:(m + 1) * P, (m + 1) * P:(m + 2) * P] for m in range(N - 1)] + [None]
    return diag, lower, upper


def sweeping_factorization(A, N: int):
    diag, lower, upper = plane_blocks(A, N)
    T = []
    for m in range(N):
        S = diag[m] if m == 0 else diag[m] - lower[m] @ T[m - 1] @ upper[m - 1]
        T.append(np.linalg.inv(S))
    return T, lower, upper


def sweeping_solve(T, lower, upper, f: np.ndarray, N: int) -> np.ndarray:
    """u = A^{-1} f through the factorization (f natural order, length N^3)."""
    P = N * N
    fb = [f[m * P:(m + 1) * P] for m in range(N)]
    # L^{-1}: z_m = f_m - A_{m,m-1} T_{m-1} z_{m-1}
    z = [fb[0]]
    for m in range(1, N):
        z.append(fb[m] - lower[m] @ (T[m - 1] @ z[m - 1]))
    y = [T[m] @ z[m] for m in range(N)]
    # U^{-1}: u_m = y_m - T_m A_{m,m+1} u_{m+1}
    u = [None] * N
    u[N - 1] = y[N - 1]
    for m in range(N - 2, -1, -1):
        u[m] = y[m] - T[m] @ (upper[m] @ u[m + 1])
    return np.concatenate(u)

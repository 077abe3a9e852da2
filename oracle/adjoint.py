"""Adjoint solve and the velocity gradient (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Because s_d depends on x_d only, the operator of Eq. (system) factors as
A = D A_sym with D = diag(s_1 s_2 s_3) (node values) and A_sym complex
symmetric, hence A^T = D^{-1} A D and A^{-T} g = D^{-1} A^{-1} (D g): the
adjoint solve reuses the forward solver.

Loss L(c) = 1/2 sum_r |R u_r - d_r|^2 with A(c) u_r = f_r and A's diagonal
containing kappa = omega^2 / c^2.  With A^T lambda_r = R^T conj(R u_r - d_r),
dL/dc = Re( sum_r lambda_r * (2 omega^2 / c^3) * u_r )   (pointwise),
since d(kappa)/dc = -2 omega^2 / c^3 and dL = Re(-lambda^T dA u).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .operator import Grid, assemble_full, global_profile


def scaling_diagonal(grid: Grid) -> np.ndarray:
    """D = s_1(x) s_2(y) s_3(z) on the padded grid, shape (N, N, N) [z, y, x]."""
    s = global_profile(grid).s_node
    return s[:, None, None] * s[None, :, None] * s[None, None, :]


def adjoint_solve_via_identity(c: np.ndarray, grid: Grid, g: np.ndarray) -> np.ndarray:
    """lambda = A^{-T} g computed as D^{-1} A^{-1} (D g) (sparse LU of A)."""
    D = scaling_diagonal(grid)
    A = assemble_full(c, grid).tocsc()
    mu = spla.spsolve(A, (D * g).ravel()).reshape(g.shape)
    return mu / D


def loss(u: np.ndarray, rec: np.ndarray, d: np.ndarray) -> float:
    """1/2 sum |u[rec] - d|^2 over right-hand sides; rec is a boolean mask (N,N,N)."""
    return 0.5 * float(np.sum(np.abs(u[:, rec] - d) ** 2))


def solve_all(c: np.ndarray, grid: Grid, f: np.ndarray) -> np.ndarray:
    A = assemble_full(c, grid).tocsc()
    lu = spla.splu(A)
    return np.stack([lu.solve(f[r].ravel()).reshape(f[r].shape) for r in range(f.shape[0])])


def velocity_gradient(c: np.ndarray, grid: Grid, f: np.ndarray, rec: np.ndarray, d: np.ndarray):
    """(L, dL/dc) by the adjoint method with direct solves."""
    u = solve_all(c, grid, f)
    A = assemble_full(c, grid).tocsc()
    luT = spla.splu(A.T.tocsc())
    grad = np.zeros(c.shape)
    for r in range(f.shape[0]):
        rhs = np.zeros(c.shape, dtype=np.complex128)
        rhs[rec] = np.conj(u[r][rec] - d[r])
        lam = luT.solve(rhs.ravel()).reshape(c.shape)
        grad += np.real(lam * (2.0 * grid.omega ** 2 / c ** 3) * u[r])
    return loss(u, rec, d), grad

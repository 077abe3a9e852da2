"""PML profile and the discrete Helmholtz operator of Section 2 (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Padded-grid reading: each axis has N = n + 2b nodes g = 0..N-1 at coordinate
(g - b + 1) h, h = 1/(n+1), with zero Dirichlet walls at g = -1 and g = N.
The PML of width eta = b h sits on every face (Section 4 puts PMLs on all six
faces); the physical nodes are g = b..b+n-1.  The PML function of Section 2,
sigma(t) = (C/eta) ((t - eta)/eta)^2 on [0, eta] and 0 beyond, is applied with
t = distance from the nearest Dirichlet wall, so the innermost PML node
(g = b-1, the physical face) has sigma = 0.  Half-integer points use the same
continuous formula.  The stretching is s = 1/(1 + i sigma/omega).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


def pml_sigma(t, eta: float, C: float):
    """sigma(t) of Section 2: (C/eta)((t-eta)/eta)^2 for 0 <= t <= eta, else 0."""
    t = np.asarray(t, dtype=np.float64)
    inside = (t >= 0.0) & (t <= eta)
    return np.where(inside, (C / eta) * ((t - eta) / eta) ** 2, 0.0)


def stretch(sigma, omega: float):
    """s = (1 + i sigma/omega)^{-1} (Section 2)."""
    return 1.0 / (1.0 + 1j * np.asarray(sigma, dtype=np.float64) / omega)


@dataclass
class Grid:
    n: int
    b: int
    omega: float
    C: float = 10.0

    @property
    def N(self) -> int:
        return self.n + 2 * self.b

    @property
    def h(self) -> float:
        return 1.0 / (self.n + 1)

    def global_sigma(self, pos):
        """sigma at (half-)integer padded positions: PML at both ends of the axis."""
        pos = np.asarray(pos, dtype=np.float64)
        eta = self.b * self.h
        return (pml_sigma((pos + 1.0) * self.h, eta, self.C)
                + pml_sigma((self.N - pos) * self.h, eta, self.C))


@dataclass
class AxisProfile:
    """Stretching on one axis of a box: nodes lo..lo+L-1.

    s_node[l] is s at node lo+l; s_half[l] is s at the half point lo+l-1/2
    (l = 0..L), so s_half[0] and s_half[L] sit between the box and its walls.
    """
    lo: int
    s_node: np.ndarray
    s_half: np.ndarray

    @property
    def L(self) -> int:
        return len(self.s_node)


def profile_from_sigma(lo: int, L: int, sigma_fn, omega: float) -> AxisProfile:
    nodes = lo + np.arange(L, dtype=np.float64)
    halves = lo - 0.5 + np.arange(L + 1, dtype=np.float64)
    return AxisProfile(lo, stretch(sigma_fn(nodes), omega), stretch(sigma_fn(halves), omega))


def global_profile(grid: Grid) -> AxisProfile:
    return profile_from_sigma(0, grid.N, grid.global_sigma, grid.omega)


def kappa_field(c: np.ndarray, omega: float) -> np.ndarray:
    """(omega^2 / c^2) at every node (Eq. system, last term)."""
    return omega ** 2 / np.asarray(c, dtype=np.float64) ** 2


def assemble_box(kappa_box: np.ndarray, px: AxisProfile, py: AxisProfile, pz: AxisProfile,
                 h: float) -> sp.csr_matrix:
    """Sparse matrix of Eq. (system) on a box with zero Dirichlet data outside it.

    kappa_box has shape (Lz, Ly, Lx); unknowns are numbered l = lx + Lx (ly + Ly lz)
    (x fastest, the paper's column-major order).  Row (lx,ly,lz) holds, per axis,
      s_node/h * [ s_{+1/2}/h (u_{+1} - u) - s_{-1/2}/h (u - u_{-1}) ]
    plus kappa u; neighbours outside the box are zero.
    """
    Lz, Ly, Lx = kappa_box.shape
    assert (px.L, py.L, pz.L) == (Lx, Ly, Lz)
    n_unk = Lx * Ly * Lz
    idx = np.arange(n_unk).reshape(Lz, Ly, Lx)
    rows, cols, vals = [], [], []
    diag = kappa_box.astype(np.complex128).copy()
    inv_h2 = 1.0 / (h * h)
    # (axis of the array, profile, shape broadcaster)
    for axis, prof in ((2, px), (1, py), (0, pz)):
        L = prof.L
        shape = [1, 1, 1]
        shape[axis] = L
        sn = prof.s_node.reshape(shape)
        sp_ = prof.s_half[1:].reshape(shape)     # s at +1/2
        sm_ = prof.s_half[:-1].reshape(shape)    # s at -1/2
        diag = diag - inv_h2 * sn * (sp_ + sm_)
        coef_up = np.broadcast_to(inv_h2 * sn * sp_, (Lz, Ly, Lx))
        coef_dn = np.broadcast_to(inv_h2 * sn * sm_, (Lz, Ly, Lx))
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[axis] = slice(0, L - 1)
        sl_hi[axis] = slice(1, L)
        # row at l couples to l+1 with s_node[l] s_half(l+1/2)
        rows.append(idx[tuple(sl_lo)].ravel())
        cols.append(idx[tuple(sl_hi)].ravel())
        vals.append(coef_up[tuple(sl_lo)].ravel())
        # row at l couples to l-1 with s_node[l] s_half(l-1/2)
        rows.append(idx[tuple(sl_hi)].ravel())
        cols.append(idx[tuple(sl_lo)].ravel())
        vals.append(coef_dn[tuple(sl_hi)].ravel())
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_unk, n_unk))
    return A.tocsr()


def assemble_full(c: np.ndarray, grid: Grid) -> sp.csr_matrix:
    """The full padded operator A of Eq. (system) (PML on all faces)."""
    g = global_profile(grid)
    return assemble_box(kappa_field(c, grid.omega), g, g, g, grid.h)


def apply_operator(u: np.ndarray, kappa: np.ndarray, px: AxisProfile, py: AxisProfile,
                   pz: AxisProfile, h: float) -> np.ndarray:
    """Matrix-free Eq. (system): u has shape (..., Lz, Ly, Lx); returns A u.

    Written independently of assemble_box: the flux differences are formed by
    padding u with its zero Dirichlet neighbours and slicing.
    """
    u = np.asarray(u, dtype=np.complex128)
    out = kappa * u
    inv_h2 = 1.0 / (h * h)
    nd = u.ndim
    for ax_from_end, prof in ((1, px), (2, py), (3, pz)):
        axis = nd - ax_from_end
        pad = [(0, 0)] * nd
        pad[axis] = (1, 1)
        up = np.pad(u, pad)
        L = u.shape[axis]
        take = lambda a, s: np.take(a, np.arange(s, s + L), axis=axis)  # noqa: E731
        u_plus, u_mid, u_minus = take(up, 2), take(up, 1), take(up, 0)
        shape = [1] * nd
        shape[axis] = L
        sn = prof.s_node.reshape(shape)
        s_p = prof.s_half[1:].reshape(shape)
        s_m = prof.s_half[:-1].reshape(shape)
        out = out + inv_h2 * sn * (s_p * (u_plus - u_mid) - s_m * (u_mid - u_minus))
    return out


def apply_full(u: np.ndarray, c: np.ndarray, grid: Grid) -> np.ndarray:
    g = global_profile(grid)
    return apply_operator(u, kappa_field(c, grid.omega), g, g, g, grid.h)

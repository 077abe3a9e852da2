"""Recursive moving-PML sweeping preconditioner, step by step in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Section 3 (moving-PML auxiliary problems H_m, the operator |T_m|,
Algorithms 1/2), Section 4.1 (inner sweep along x2: H~_m, |T~_m|, Algorithms
3/4) and Section 4.2 (|[T_m]|, Algorithms 5/6), with the first implementation
modification (several layers, d, per auxiliary problem) and the second (an
auxiliary PML width b_aux that may differ from b).

Readings (the paper leaves these open; both the oracle and the CUDA path use
them):
  * Blocks on a swept axis: block 0 is the boundary-PML slab g = 0..b-1, then
    blocks of d layers from g = b on; the last block is shorter when
    (N - b) mod d != 0.
  * Auxiliary window of block M >= 1 (first layer m, end e): the b_aux layers
    below the block plus the block itself, g = m-b_aux .. e-1, with a moving
    PML whose Dirichlet wall is at m-b_aux-1 (s(x - (m-b)h) of Section 3 with
    b replaced by b_aux), plus the global PML of the far face where the window
    reaches it.  If m - b_aux < 0 the window is clipped to g = 0 and keeps the
    global profile, i.e. it is the leading part of the real operator.  Zero
    Dirichlet at g = e.  Block 0's window is itself with the global profile.
  * One front, low to high then back, exactly as Algorithms 4 and 6 print
    (schedule='one_front').
  * Two fronts (schedule='two_front', Section 4.2's third modification, used in
    both loops in Section 5's experiments; the paper gives no formulas): the
    interior g = b .. N-b-1 is cut into q blocks of d layers from each end and
    a centre block of the remaining 1 .. 2d layers, q = (N - 2b - 1) // (2d);
    the boundary slabs g = 0..b-1 and N-b..N-1 are blocks of their own.  The
    lower front's blocks (the low slab and the q blocks above it) have the
    moving PML below, as in one front; the upper front's blocks mirror them
    (window: the block plus b_aux layers above, moving PML above, Dirichlet
    below); the centre block's window extends b_aux layers to both sides with
    a moving PML on each.  Forward: the lower front upward, the upper front
    downward, then the centre with the couplings of both neighbours; backward:
    the lower front downward, the upper front upward.  This is the block LDU
    factorisation eliminated from both ends towards the centre (a twisted
    factorisation), with every Schur complement replaced by its auxiliary
    problem; with windows reaching the faces (b_aux >= N) it is exact.
  * A window side without a moving PML keeps the global profile of that side
    (the real operator's coefficients; nonzero only inside the boundary PML).
  * The quasi-2D problems are solved by one inner sweep (Section 5 states one
    application of the inner preconditioner).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as spla

from .operator import (AxisProfile, Grid, assemble_box, global_profile, kappa_field,
                       pml_sigma, profile_from_sigma)


def axis_blocks(N: int, b: int, d: int):
    """[(start, end)] of the swept-axis blocks: the PML slab, then d layers each."""
    if not (N > b >= 1 and d >= 1):
        raise ValueError("need N > b >= 1 and d >= 1")
    out = [(0, b)]
    m = b
    while m < N:
        out.append((m, min(m + d, N)))
        m += d
    return out


def axis_blocks_two_front(N: int, b: int, d: int):
    """[(start, end)] and roles of the two-front blocks in axis order: the low
    PML slab and q blocks of d layers ('L'), the centre ('C'), q blocks of d
    layers and the high PML slab ('U')."""
    if not (N > 2 * b >= 2 and d >= 1):
        raise ValueError("need N > 2b >= 2 and d >= 1")
    q = (N - 2 * b - 1) // (2 * d)
    lower = [(0, b)] + [(b + i * d, b + (i + 1) * d) for i in range(q)]
    upper = [(N - b - (i + 1) * d, N - b - i * d) for i in range(q)][::-1] + [(N - b, N)]
    centre = (b + q * d, N - b - q * d)
    return lower + [centre] + upper, ["L"] * len(lower) + ["C"] + ["U"] * len(upper)


def axis_schedule(N: int, b: int, d: int, schedule: str = "one_front"):
    """(blocks, roles, centre index) of a swept axis.  One front: every block
    is swept from below and the last block ends the forward pass (its window
    is a lower-front window: it has no upper neighbour)."""
    if schedule == "one_front":
        blocks = axis_blocks(N, b, d)
        return blocks, ["L"] * (len(blocks) - 1) + ["C"], len(blocks) - 1
    if schedule == "two_front":
        blocks, roles = axis_blocks_two_front(N, b, d)
        return blocks, roles, roles.index("C")
    raise ValueError("schedule must be 'one_front' or 'two_front'")


def axis_window(grid: Grid, blocks, M: int, b_aux: int, role: str = "L"):
    """Auxiliary window of block M on a swept axis.

    A side gets b_aux extra layers and a moving PML when the block's role
    eliminates towards it ('L': below, 'U': above, 'C': both) and the
    block is not at that face; a window clipped by a face keeps that side's
    global profile, as does a side without a moving PML.  Returns (profile,
    (ia, ib)) where the profile covers the window and [ia, ib) are the
    block's own layers inside the window.
    """
    m, e = blocks[M]
    N = grid.N
    low_mov = role in ("L", "C") and m > 0
    high_mov = role in ("U", "C") and e < N
    lo = m - b_aux if low_mov else m
    hi = e + b_aux if high_mov else e
    if lo < 0:
        lo, low_mov = 0, False
    if hi > N:
        hi, high_mov = N, False
    eta_aux = b_aux * grid.h
    eta = grid.b * grid.h

    def fn(pos):
        pos = np.asarray(pos, dtype=np.float64)
        s_lo = (pml_sigma((pos - (lo - 1)) * grid.h, eta_aux, grid.C) if low_mov
                else pml_sigma((pos + 1.0) * grid.h, eta, grid.C))
        s_hi = (pml_sigma((hi - pos) * grid.h, eta_aux, grid.C) if high_mov
                else pml_sigma((N - pos) * grid.h, eta, grid.C))
        return s_lo + s_hi
    prof = profile_from_sigma(lo, hi - lo, fn, grid.omega)
    return prof, (m - lo, e - lo)


@dataclass
class Quasi1D:
    """Block-tridiagonal (along x1) auxiliary problem H~ for slab M, line block M'.

    Unknowns of one x-block are ordered a = lz + Lz*ly (dimension 3, then 2;
    dimension 1 last, Section 4.1).  D[i] are the k x k diagonal blocks; the
    x-couplings are scalar multiples of the identity because s_1 depends on
    x1 only: row block i couples to i-1 with lower[i] and to i+1 with upper[i].
    """
    D: np.ndarray            # (Nx, k, k)
    lower: np.ndarray        # (Nx,)  entry (i, i-1); lower[0] unused
    upper: np.ndarray        # (Nx,)  entry (i, i+1); upper[-1] unused
    Ly: int
    Lz: int
    y_interest: tuple        # [ia, ib) lines of the block inside the y-window
    T: list | None = None    # T_i = S_i^{-1}
    fmt: str | None = None   # None: LDU from x = 0 (Section 3 as printed); else the
                             # twisted form below with T_i stored in this format

    @property
    def k(self) -> int:
        return self.Ly * self.Lz

    @property
    def Nx(self) -> int:
        return self.D.shape[0]

    def factor(self):
        """Block LDU along x1 (the Section 3 recursion at the quasi-1D level):
        S_0 = D_0, S_i = D_i - A_{i,i-1} T_{i-1} A_{i-1,i}, T_i = S_i^{-1}."""
        if self.fmt is not None:
            return self.factor_twisted()
        T = []
        S = self.D[0]
        for i in range(self.Nx):
            if i > 0:
                S = self.D[i] - (self.lower[i] * self.upper[i - 1]) * T[i - 1]
            T.append(np.linalg.inv(S))
        self.T = T
        return self

    def factor_twisted(self):
        """The same recursion run from both ends, meeting at m = (Nx-1)//2:
        S_0 = D_0,       S_i = D_i - A_{i,i-1} T_{i-1} A_{i-1,i}            (i < m)
        S_{Nx-1} = D_{Nx-1}, S_i = D_i - A_{i,i+1} T_{i+1} A_{i+1,i}        (i > m)
        S_m = D_m - A_{m,m-1} T_{m-1} A_{m-1,m} - A_{m,m+1} T_{m+1} A_{m+1,m}
        (a twisted block factorisation: the same inverse as the one-sided LDU,
        with two independent elimination chains).  The chains use the exact
        T_i; only the stored copies are rounded to self.fmt."""
        from .precision import round_factor
        Nx, m = self.Nx, (self.Nx - 1) // 2
        T = [None] * Nx
        for i in range(m):
            S = self.D[i] if i == 0 else self.D[i] - (self.lower[i] * self.upper[i - 1]) * T[i - 1]
            T[i] = np.linalg.inv(S)
        for i in range(Nx - 1, m, -1):
            S = self.D[i] if i == Nx - 1 else self.D[i] - (self.upper[i] * self.lower[i + 1]) * T[i + 1]
            T[i] = np.linalg.inv(S)
        S = self.D[m].copy()
        if m > 0:
            S = S - (self.lower[m] * self.upper[m - 1]) * T[m - 1]
        if m + 1 < Nx:
            S = S - (self.upper[m] * self.lower[m + 1]) * T[m + 1]
        T[m] = np.linalg.inv(S)
        if self.fmt != "fp64":
            T = [round_factor(t, self.fmt) for t in T]
        self.T = T
        return self

    def solve_twisted(self, q: np.ndarray) -> np.ndarray:
        """x = H~^{-1} q with the twisted factors: eliminate towards m from both
        ends, solve the middle block, substitute back outwards."""
        T, Nx, m = self.T, self.Nx, (self.Nx - 1) // 2
        lo, up = self.lower, self.upper
        y = np.empty_like(q)
        for i in range(m):
            y[i] = T[i] @ (q[i] if i == 0 else q[i] - lo[i] * y[i - 1])
        for i in range(Nx - 1, m, -1):
            y[i] = T[i] @ (q[i] if i == Nx - 1 else q[i] - up[i] * y[i + 1])
        r = q[m].copy()
        if m > 0:
            r = r - lo[m] * y[m - 1]
        if m + 1 < Nx:
            r = r - up[m] * y[m + 1]
        x = np.empty_like(q)
        x[m] = T[m] @ r
        for i in range(m - 1, -1, -1):
            x[i] = y[i] - up[i] * (T[i] @ x[i + 1])
        for i in range(m + 1, Nx):
            x[i] = y[i] - lo[i] * (T[i] @ x[i - 1])
        return x

    def solve(self, q: np.ndarray) -> np.ndarray:
        """u = U^{-1} diag(T) L^{-1} q for q of shape (Nx, k, R)."""
        if self.T is None:
            self.factor()
        if self.fmt is not None:
            return self.solve_twisted(q)
        T, Nx = self.T, self.Nx
        y = np.empty_like(q)
        y[0] = T[0] @ q[0]
        for i in range(1, Nx):
            y[i] = T[i] @ (q[i] - self.lower[i] * y[i - 1])
        x = np.empty_like(q)
        x[Nx - 1] = y[Nx - 1]
        for i in range(Nx - 2, -1, -1):
            x[i] = y[i] - self.upper[i] * (T[i] @ x[i + 1])
        return x

    def restricted_apply(self, alpha: np.ndarray) -> np.ndarray:
        """|T~|: embed alpha on the block lines, solve, restrict (Section 4.1 procedure).

        alpha has shape (R, Lz, nl, Nx) (slab layout [z, y, x] per RHS).
        """
        R = alpha.shape[0]
        ia, ib = self.y_interest
        q = np.zeros((self.Nx, self.Ly, self.Lz, R), dtype=np.complex128)
        q[:, ia:ib, :, :] = np.transpose(alpha, (3, 2, 1, 0))
        x = self.solve(q.reshape(self.Nx, self.k, R)).reshape(self.Nx, self.Ly, self.Lz, R)
        return np.transpose(x[:, ia:ib, :, :], (3, 2, 1, 0))


def block_tridiagonal_x(H, Nx: int, Ly: int, Lz: int):
    """Split the box matrix (natural x-fastest order) into x-blocks of size Ly*Lz."""
    k = Ly * Lz
    coo = H.tocoo()
    r, c, v = coo.row, coo.col, coo.data
    # natural numbering l = x + Nx (y + Ly z)  ->  block x, local a = z + Lz y
    rx, ry, rz = r % Nx, (r // Nx) % Ly, r // (Nx * Ly)
    cx, cy, cz = c % Nx, (c // Nx) % Ly, c // (Nx * Ly)
    ra, ca = rz + Lz * ry, cz + Lz * cy
    D = np.zeros((Nx, k, k), dtype=np.complex128)
    lower = np.zeros(Nx, dtype=np.complex128)
    upper = np.zeros(Nx, dtype=np.complex128)
    same = rx == cx
    D[rx[same], ra[same], ca[same]] = v[same]
    dn = cx == rx - 1
    up = cx == rx + 1
    assert np.all(ra[dn] == ca[dn]) and np.all(ra[up] == ca[up]), "x-coupling not diagonal"
    assert np.all(same | dn | up)
    lower[rx[dn]] = v[dn]
    upper[rx[up]] = v[up]
    # the coupling is the same scalar for every (y, z) of a block: check it
    assert np.allclose(v[dn], lower[rx[dn]]) and np.allclose(v[up], upper[rx[up]])
    return D, lower, upper


class SweepPreconditioner:
    """Algorithm 5 (setup) and Algorithm 6 (apply) of Section 4.2.

    b_aux_z / b_aux_y set the auxiliary PML width of the outer (x3) and inner
    (x2) sweeps; inner='sweep' uses Algorithm 4 for the quasi-2D problems
    (the recursive method), inner='exact' solves them with a sparse direct
    solver (the non-recursive method of Section 3, Algorithm 2).
    keep_factors=False refactors a slab's problems each time it is used
    (for grids whose factors do not fit in host memory).
    factor_format=None factors each quasi-1D problem from x = 0 as Section 3
    prints it; 'fp64' uses the twisted factorisation (Quasi1D.factor_twisted)
    and 'fp32', 'fp16', 'split_fp16' additionally round every stored T_i
    (oracle.precision).
    """

    def __init__(self, c: np.ndarray, grid: Grid, d: int = 1, b_aux: int | None = None,
                 b_aux_z: int | None = None, b_aux_y: int | None = None,
                 inner: str = "sweep", keep_factors: bool = True, factor_format: str | None = None,
                 schedule: str = "one_front"):
        self.grid = grid
        self.factor_format = factor_format
        self.d = d
        b_aux = grid.b if b_aux is None else b_aux
        self.b_aux_z = b_aux if b_aux_z is None else b_aux_z
        self.b_aux_y = b_aux if b_aux_y is None else b_aux_y
        self.inner = inner
        self.keep = keep_factors
        self.N = grid.N
        self.kappa = kappa_field(c, grid.omega)
        self.gprof = global_profile(grid)
        self.schedule = schedule
        self.blocks, self.roles, self.centre = axis_schedule(self.N, grid.b, d, schedule)
        self.B = len(self.blocks)
        h2 = grid.h ** 2
        g = self.gprof
        # A's couplings between consecutive layers (Eq. system): row g to g-1 and g to g+1
        self.c_dn = g.s_node * g.s_half[:-1] / h2
        self.c_up = g.s_node * g.s_half[1:] / h2
        self.zwin = [axis_window(grid, self.blocks, M, self.b_aux_z, self.roles[M]) for M in range(self.B)]
        self.ywin = [axis_window(grid, self.blocks, M, self.b_aux_y, self.roles[M]) for M in range(self.B)]
        self._slab_cache = {}

    # ---- auxiliary problems -------------------------------------------------
    def quasi1d(self, M: int, Mp: int) -> Quasi1D:
        pz, _ = self.zwin[M]
        py, yi = self.ywin[Mp]
        kap = self.kappa[pz.lo:pz.lo + pz.L, py.lo:py.lo + py.L, :]
        H = assemble_box(kap, self.gprof, py, pz, self.grid.h)
        D, lo, up = block_tridiagonal_x(H, self.N, py.L, pz.L)
        return Quasi1D(D, lo, up, py.L, pz.L, yi, fmt=self.factor_format)

    def slab_problems(self, M: int):
        """Algorithm 3 for the quasi-2D problem of slab M: factor every H~_{M'}."""
        if M in self._slab_cache:
            return self._slab_cache[M]
        probs = [self.quasi1d(M, Mp).factor() for Mp in range(self.B)]
        if self.keep:
            self._slab_cache[M] = probs
        return probs

    def restricted_operator(self, M: int, Mp: int, rows, cols) -> np.ndarray:
        """The map |T~_{M'}| of Section 4.1 on slab M between chosen entries:
        embed a unit value at each column entry, solve the quasi-1D problem
        H~_{M'} (its LDU, Section 3), read the row entries.  rows and cols are
        sequences of (x, line, z row) with the line a global y index inside the
        line block's window and the z row a row of slab M's window.  Returns
        G[len(rows), len(cols)] = (H~^{-1})[rows, cols]."""
        q1 = self.quasi1d(M, Mp)
        q1.factor()
        py, _ = self.ywin[Mp]
        Lz = q1.Lz

        def block_row(line, lz):
            return lz + Lz * (line - py.lo)

        E = np.zeros((q1.Nx, q1.k, len(cols)), dtype=np.complex128)
        for j, (x, line, lz) in enumerate(cols):
            E[x, block_row(line, lz), j] = 1.0
        X = q1.solve(E)
        G = np.empty((len(rows), len(cols)), dtype=np.complex128)
        for i, (x, line, lz) in enumerate(rows):
            G[i] = X[x, block_row(line, lz)]
        return G

    def setup(self):
        """Algorithm 5: all quasi-1D factorizations (independent problems)."""
        if self.inner == "sweep":
            for M in range(self.B):
                self.slab_problems(M)
        return self

    def slab_matrix(self, M: int):
        """The quasi-2D auxiliary matrix H_M on slab M's window (natural order)."""
        pz, _ = self.zwin[M]
        kap = self.kappa[pz.lo:pz.lo + pz.L, :, :]
        return assemble_box(kap, self.gprof, self.gprof, pz, self.grid.h)

    # ---- Algorithm 4: inner sweep along x2 ----------------------------------
    def sweep(self, solve, g: np.ndarray, axis: int) -> np.ndarray:
        """The block sweep shared by Algorithms 4 and 6 along array axis `axis`
        of g: forward over the lower front upward and the upper front downward,
        the centre block last, then backward over the lower front downward and
        the upper front upward (one front: the lower front is every block but
        the last, which is the centre).  solve(M, rhs) applies block M's
        restricted auxiliary inverse to rhs (the block's own layers)."""
        v = np.zeros_like(g)
        B, c = self.B, self.centre

        def sl(lo, hi):
            idx = [slice(None)] * g.ndim
            idx[axis] = slice(lo, hi)
            return tuple(idx)

        def lay(q):
            idx = [slice(None)] * g.ndim
            idx[axis] = q
            return tuple(idx)
        for M in list(range(c)) + list(range(B - 1, c, -1)) + [c]:
            m, e = self.blocks[M]
            rhs = g[sl(m, e)].copy()
            if M > 0 and M <= c:                         # lower front and centre: the block below
                rhs[lay(0)] -= self.c_dn[m] * v[lay(m - 1)]
            if M < B - 1 and M >= c:                     # upper front and centre: the block above
                rhs[lay(e - 1 - m)] -= self.c_up[e - 1] * v[lay(e)]
            v[sl(m, e)] = solve(M, rhs)
        for M in list(range(c - 1, -1, -1)) + list(range(c + 1, B)):
            m, e = self.blocks[M]
            rhs = np.zeros_like(g[sl(m, e)])
            if M < c:
                rhs[lay(e - 1 - m)] = self.c_up[e - 1] * v[lay(e)]
            else:
                rhs[lay(0)] = self.c_dn[m] * v[lay(m - 1)]
            v[sl(m, e)] -= solve(M, rhs)
        return v

    def inner_sweep(self, M: int, g: np.ndarray) -> np.ndarray:
        """v ~= H_M^{-1} g for g of shape (R, Lz, N, N) (Algorithm 4)."""
        probs = self.slab_problems(M)
        return self.sweep(lambda Mp, rhs: probs[Mp].restricted_apply(rhs), g, axis=2)

    def exact_slab_solve(self, M: int, g: np.ndarray) -> np.ndarray:
        H = self.slab_matrix(M).tocsc()
        lu = spla.splu(H)
        R = g.shape[0]
        out = np.empty_like(g)
        for r in range(R):
            out[r] = lu.solve(g[r].ravel()).reshape(g[r].shape)
        return out

    def slab_apply(self, M: int, alpha: np.ndarray) -> np.ndarray:
        """|[T_M]| (or |T_M| with inner='exact'): embed on the block layers,
        solve the slab problem, restrict.  alpha: (R, nz, N, N)."""
        pz, (za, zb) = self.zwin[M]
        R = alpha.shape[0]
        g = np.zeros((R, pz.L, self.N, self.N), dtype=np.complex128)
        g[:, za:zb] = alpha
        if self.inner == "sweep":
            v = self.inner_sweep(M, g)
        else:
            v = self.exact_slab_solve(M, g)
        return v[:, za:zb]

    # ---- Algorithm 6: outer sweep along x3 ----------------------------------
    def apply(self, f: np.ndarray) -> np.ndarray:
        """u ~= A^{-1} f for f of shape (R, N, N, N) or (N, N, N) (Algorithm 6)."""
        single = f.ndim == 3
        f = np.asarray(f, dtype=np.complex128)
        if single:
            f = f[None]
        u = self.sweep(self.slab_apply, f, axis=1)
        return u[0] if single else u

"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

Each test states which part of the oracle it pins and why a plausible slip
(a dropped term, a wrong sign, a shifted index) would fail it.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.exact import sweeping_factorization, sweeping_solve
from oracle.krylov import gmres
from oracle.operator import (Grid, apply_full, assemble_box, assemble_full, global_profile,
                             kappa_field)
from oracle.sweep import SweepPreconditioner, axis_blocks, axis_blocks_two_front, axis_window
from paper_1502_07266_gb300 import workloads as W


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# ---------------------------------------------------------------- operator ---

def test_profile_endpoints():
    """Section 2: sigma vanishes from the PML's inner edge on and equals C/eta at the wall.

    The innermost PML node (the physical face g = b-1) must carry sigma = 0
    and every physical node s = 1; the wall half-point carries the largest
    damping.  A PML shifted by one node fails the first two checks."""
    g = Grid(15, 4, W.omega_for(15))
    prof = global_profile(g)
    sig = g.global_sigma(np.arange(g.N))
    assert sig[g.b - 1] == 0.0 and sig[g.N - g.b] == 0.0
    assert np.all(prof.s_node[g.b - 1:g.N - g.b + 1] == 1.0)
    assert sig[0] > 0 and sig[g.N - 1] > 0
    # at the wall (t = 0) sigma = C/eta, mirrored on both faces
    assert g.global_sigma(-1.0) == pytest.approx(g.C / (g.b * g.h))
    assert g.global_sigma(g.N) == pytest.approx(g.C / (g.b * g.h))
    # monotone decay into the domain
    assert np.all(np.diff(sig[:g.b]) < 0)


def test_matrix_free_equals_assembled():
    """The slicing form and the COO assembly of Eq. (system) agree to rounding."""
    n, b = 5, 2
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=4)
    A = assemble_full(c, g)
    x = W.random_rhs(1, n, b, seed=5)[0]
    assert _rel(apply_full(x, c, g), A @ x.ravel()) < 1e-14


def test_symmetrised_operator_is_complex_symmetric():
    """A = D A_sym with D = diag(s1 s2 s3) and A_sym complex symmetric.

    Holds because s_d depends on x_d only; an s at the wrong half point (e.g.
    s_{i+1/2} in the lower coupling) breaks the symmetry."""
    n, b = 5, 3
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    A = assemble_full(c, g)
    s = global_profile(g).s_node
    Dv = (s[None, None, :] * s[None, :, None] * s[:, None, None]).ravel()
    Asym = (A.multiply(1.0 / Dv[:, None])).toarray()
    assert np.abs(Asym - Asym.T).max() < 1e-12 * np.abs(Asym).max()


def test_stencil_consistent_with_stretched_pde():
    """Eq. (system) is a second-order approximation of the PML'd PDE.

    The continuous operator sum_d (s_d d_d)(s_d d_d) u + omega^2/c^2 u is built
    symbolically (sympy) from the Section 2 sigma; the maximum pointwise error
    over the nodes (PML included) falls by ~4 when h halves with the PML width
    eta fixed.  The innermost PML layer (t = eta) is checked separately: sigma
    is only C^1 there, so its local error is first order.  A dropped or
    mis-signed term leaves an O(1) error."""
    sympy = pytest.importorskip("sympy")
    om, C, eta = 9.0, 10.0, 0.25
    t = sympy.Symbol("t", real=True)
    xs = sympy.symbols("x0:3", real=True)
    errs = []
    for n in (15, 31):
        b = int(round(eta * (n + 1)))
        g = Grid(n, b, om, C)
        h, N = g.h, g.N
        L = 1.0 + 2 * b * h          # wall to wall
        lo = -b * h
        # sigma of one face as a function of the distance t from its wall
        sig_face = sympy.Piecewise(((C / eta) * ((t - eta) / eta) ** 2, t <= eta), (0, True))
        expr = 0
        u = 1
        for q in range(3):
            u = u * sympy.sin(sympy.pi * (xs[q] - lo) / L)
        for q in range(3):
            sq = (sig_face.subs(t, xs[q] - lo) + sig_face.subs(t, lo + L - xs[q]))
            s = 1 / (1 + sympy.I * sq / om)
            expr = expr + s * sympy.diff(s * sympy.diff(u, xs[q]), xs[q])
        kap = om ** 2
        expr = expr + kap * u
        fn = sympy.lambdify(xs, expr, "numpy")
        fu = sympy.lambdify(xs, u, "numpy")
        x = lo + (np.arange(N) + 1) * h
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        U = fu(X, Y, Z).astype(np.complex128)
        exact = np.broadcast_to(fn(X, Y, Z), U.shape)
        disc = apply_full(U, np.ones((N, N, N)), g)
        kink1 = np.isin(np.arange(N), (b - 1, N - b))
        kink = kink1[:, None, None] | kink1[None, :, None] | kink1[None, None, :]
        err = np.abs(disc - exact) / np.abs(exact).max()
        errs.append(err[~kink].max())
        assert err[kink].max() < 0.05
    ratio = errs[0] / errs[1]
    assert errs[1] < 1e-2
    assert 3.0 < ratio < 5.0, (errs, ratio)


@pytest.mark.slow
def test_green_function_constant_velocity():
    """Physics pin: for c = 1 the direct solution is the outgoing free-space field.

    (Delta + omega^2) G = delta gives G = -exp(i omega r)/(4 pi r); the Gaussian
    source exp(-alpha r^2) scales it by (pi/alpha)^{3/2} exp(-omega^2/(4 alpha)).
    The PML with s = (1 + i sigma/omega)^{-1} absorbs exp(+i omega r).  Away from
    the source the error must fall like h^2 (12 vs 8 points per wavelength at a
    fixed omega and PML width); a wrong sign of sigma or of the stencil gives an
    incoming or reflected field and an O(1) error."""
    om = 2 * math.pi * 2.0
    errs = []
    for n, b in ((15, 4), (23, 6)):
        g = Grid(n, b, om)
        N = g.N
        c = W.velocity_constant(n, b)
        f = W.gaussian_sources(n, b, om, [(0.5, 0.5, 0.5)])[0]
        u = spla.spsolve(assemble_full(c, g).tocsc(), f.ravel()).reshape(N, N, N)
        x = W.physical_coords(n, b)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        r = np.sqrt((X - .5) ** 2 + (Y - .5) ** 2 + (Z - .5) ** 2)
        alpha = (4 * om / math.pi) ** 2
        G = (-(math.pi / alpha) ** 1.5 * math.exp(-om ** 2 / (4 * alpha))
             * np.exp(1j * om * r) / (4 * math.pi * np.maximum(r, 1e-12)))
        sel = (r >= 0.2) & (r <= 0.35)
        errs.append(_rel(u[sel], G[sel]))
    assert errs[1] < 0.05
    # h ratio 24/16: second order predicts 2.25
    assert 1.8 < errs[0] / errs[1] < 3.0, errs


def test_direct_dense_lu_matches_sparse():
    """Dense LU of the assembled matrix (a library special case) vs sparse LU."""
    n, b = 5, 2
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    A = assemble_full(c, g)
    f = W.random_rhs(1, n, b, seed=8)[0].ravel()
    u1 = np.linalg.solve(A.toarray(), f)
    u2 = spla.spsolve(A.tocsc(), f)
    assert _rel(u1, u2) < 1e-12
    assert _rel(A @ u1, f) < 1e-12


# ------------------------------------------------- exact sweeping (Sec. 3) ---

def test_exact_block_ldu_reproduces_inverse():
    """Section 3: the plane-block LDU with exact Schur complements gives A^{-1} f."""
    n, b = 3, 2
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=2)
    A = assemble_full(c, g)
    f = W.random_rhs(1, n, b, seed=9)[0].ravel()
    T, lo, up = sweeping_factorization(A, g.N)
    u = sweeping_solve(T, lo, up, f, g.N)
    assert _rel(u, spla.spsolve(A.tocsc(), f)) < 1e-10


def test_T_m_is_half_space_green_function():
    """Section 3: T_m is the lower-right block of (A_{1:m,1:m})^{-1}."""
    n, b = 3, 2
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    A = assemble_full(c, g).toarray()
    P = g.N * g.N
    T, _, _ = sweeping_factorization(assemble_full(c, g), g.N)
    for m in (1, 3, g.N - 1):
        lead = np.linalg.inv(A[:(m + 1) * P, :(m + 1) * P])
        assert _rel(T[m], lead[m * P:, m * P:]) < 1e-10


# ------------------------------------------------ quasi-1D block LDU (a4/a5) ---

@pytest.mark.parametrize("M,Mp", [(0, 0), (0, 3), (2, 0), (3, 4)])
def test_quasi1d_factor_solve_matches_sparse_solve(M, Mp):
    """The x1 block LDU of an auxiliary quasi-1D problem equals a sparse LU solve."""
    n, b, d = 7, 3, 1
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=1)
    P = SweepPreconditioner(c, g, d=d)
    q1 = P.quasi1d(M, Mp).factor()
    pz, _ = P.zwin[M]
    py, _ = P.ywin[Mp]
    kap = kappa_field(c, g.omega)[pz.lo:pz.lo + pz.L, py.lo:py.lo + py.L, :]
    H = assemble_box(kap, global_profile(g), py, pz, g.h)
    rng = np.random.default_rng(5)
    q = rng.standard_normal((g.N, q1.k, 2)) + 1j * rng.standard_normal((g.N, q1.k, 2))
    x = q1.solve(q)
    # q is ordered (x, y, z) with z fastest; H's natural order is x fastest
    Lz, Ly = q1.Lz, q1.Ly
    for r in range(2):
        qn = q[:, :, r].reshape(g.N, Ly, Lz).transpose(2, 1, 0).ravel()
        xn = spla.spsolve(H.tocsc(), qn)
        assert _rel(x[:, :, r].reshape(g.N, Ly, Lz).transpose(2, 1, 0).ravel(), xn) < 1e-11


@pytest.mark.parametrize("fmt", [None, "fp64"])
def test_quasi1d_factors_are_symmetric_after_column_scaling(fmt):
    """The window operator is D A_sym with D = s_1 s_2 s_3 at the nodes (each
    axis term carries its own node stretch), so every Schur complement is
    S_i = D_i S_i^sym and T_i D_i = (S_i^sym)^{-1} is complex symmetric, for the
    one-sided and the twisted factorisation alike.  A wrong coupling product
    in the recursion (e.g. A_{i,i-1} A_{i,i-1}) or a window profile on the wrong
    axis breaks it."""
    n, b, d = 7, 3, 1
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=3)
    P = SweepPreconditioner(c, g, d=d, factor_format=fmt)
    s1 = global_profile(g).s_node
    for M, Mp in [(0, 0), (2, 3), (4, 1)]:
        q1 = P.quasi1d(M, Mp).factor()
        pz, _ = P.zwin[M]
        py, _ = P.ywin[Mp]
        dyz = (py.s_node[:, None] * pz.s_node[None, :]).ravel()     # a = lz + Lz ly
        for i in range(g.N):
            X = q1.T[i] * (s1[i] * dyz)[None, :]
            assert np.abs(X - X.T).max() <= 1e-12 * np.abs(X).max()
        # and the plain T_i itself is not symmetric (the scaling matters)
        T = q1.T[g.N // 2]
        assert np.abs(T - T.T).max() > 1e-6 * np.abs(T).max()


def test_moving_pml_window_is_translated_boundary_problem():
    """Section 3: H_m is the boundary problem translated (s_3^m(x) = s(x_3 - (m-b)h)).

    For constant velocity the window of an interior block equals, entry by
    entry, the first b+d layers of the real operator (wall at g = -1).  A
    moving wall off by one layer changes every PML coefficient."""
    n, b, d = 9, 3, 2
    g = Grid(n, b, W.omega_for(n))
    blocks = axis_blocks(g.N, b, d)
    glob = global_profile(g)
    for M in (1, 2, 3):
        prof, (ia, ib) = axis_window(g, blocks, M, b)
        L = prof.L
        assert (ia, ib) == (b, L)
        np.testing.assert_allclose(prof.s_node, glob.s_node[:L], rtol=0, atol=1e-15)
        np.testing.assert_allclose(prof.s_half, glob.s_half[:L + 1], rtol=0, atol=1e-15)


def test_moving_window_keeps_the_far_face_pml():
    """Windows that reach the high face (Section 3's moving PML on the low side,
    the real PML of the opposite face kept, as in H_m of Section 3 whose other
    faces carry the original boundary conditions).

    On the block's own layers the window profile must equal the global one
    (those nodes see the far-face PML and no moving PML).  Below them it must
    equal the low-face profile translated to the moving wall wherever the
    far-face sigma is zero, and where both PMLs cover a node the two sigmas
    add.  Dropping the far-face term fails the first check near the high face;
    adding it twice or measuring it from the window's end fails the first or
    the third."""
    n, b, d = 9, 3, 1
    g = Grid(n, b, W.omega_for(n))
    N = g.N
    blocks = axis_blocks(N, b, d)
    glob = global_profile(g)

    def sig(s):                             # s = 1/(1 + i sigma/omega)  ->  sigma
        return g.omega * np.imag(1.0 / np.asarray(s))

    reached = 0
    for M in range(1, len(blocks)):
        m, e = blocks[M]
        prof, (ia, ib) = axis_window(g, blocks, M, b)
        lo = prof.lo
        if lo == 0:
            continue                        # clipped windows are the leading block of A
        nodes = lo + np.arange(prof.L)
        # the block's own layers: the global profile, far face included
        np.testing.assert_allclose(prof.s_node[ia:ib], glob.s_node[m:e], rtol=0, atol=1e-15)
        np.testing.assert_allclose(prof.s_half[ia + 1:ib + 1], glob.s_half[m + 1:e + 1], rtol=0, atol=1e-15)
        # the moving layers: translated low-face profile where the far face has no PML
        far = np.where(nodes[:ia] >= N // 2, sig(glob.s_node[nodes[:ia]]), 0.0)   # high face only
        trans = glob.s_node[:ia]
        free = far == 0.0
        np.testing.assert_allclose(prof.s_node[:ia][free], trans[free], rtol=0, atol=1e-15)
        both = ~free
        np.testing.assert_allclose(sig(prof.s_node[:ia][both]), sig(trans[both]) + far[both], rtol=1e-12, atol=1e-9)
        if m > N - b:                       # node N-b is the far PML's sigma = 0 node
            reached += 1
            assert np.any(sig(prof.s_node[ia:ib]) > 0)      # the far-face PML is really there
    assert reached >= b - 1


def test_block_partition():
    assert axis_blocks(10, 3, 1) == [(0, 3)] + [(m, m + 1) for m in range(3, 10)]
    assert axis_blocks(10, 3, 3) == [(0, 3), (3, 6), (6, 9), (9, 10)]


# ------------------------------------------------- sweeps (a6/a7, Alg 4/6) ---

@pytest.mark.parametrize("n,b,d", [(3, 2, 1), (3, 2, 2), (4, 2, 3)])
def test_exact_limit_gives_inverse(n, b, d):
    """With b_aux >= N every window clips to the leading block of the real
    operator, each |T| is the exact Schur-complement operator of Section 3 at
    both levels, and the preconditioner equals A^{-1}.  Pins embedding,
    restriction, coupling signs, first-block handling and sweep order."""
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=1)
    A = assemble_full(c, g)
    f = W.random_rhs(2, n, b, seed=3)
    P = SweepPreconditioner(c, g, d=d, b_aux=g.N + 1).setup()
    z = P.apply(f)
    for r in range(2):
        assert _rel(z[r], spla.spsolve(A.tocsc(), f[r].ravel())) < 1e-11


def test_recursive_with_exact_inner_limit_equals_nonrecursive():
    """Inner b_aux >= N makes Algorithm 4 exact, so |[T_m]| = |T_m| and the
    recursive apply equals the non-recursive Algorithm 2 with exact quasi-2D
    solves (sparse LU of H_m).  Pins the outer moving PML independently of
    the inner level."""
    n, b, d = 5, 2, 1
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    f = W.random_rhs(1, n, b, seed=11)
    rec = SweepPreconditioner(c, g, d=d, b_aux_z=b, b_aux_y=g.N + 1).apply(f)
    nonrec = SweepPreconditioner(c, g, d=d, b_aux_z=b, inner="exact").apply(f)
    assert _rel(rec, nonrec) < 1e-11


def test_preconditioner_is_close_to_inverse():
    """The approximate preconditioner is a good approximation of A^{-1}."""
    n, b = 7, 3
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    A = assemble_full(c, g)
    f = W.random_rhs(1, n, b, seed=12)[0]
    z = SweepPreconditioner(c, g, d=1).apply(f)
    u = spla.spsolve(A.tocsc(), f.ravel())
    assert _rel(z, u) < 0.2


# ------------------------------------------------------------- GMRES (a8) ---

def test_gmres_matches_direct_solve():
    """GMRES with the sweep preconditioner converges to A^{-1} f (the solution
    does not depend on the preconditioner) in few iterations."""
    n, b = 7, 3
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    f = W.gaussian_sources(n, b, g.omega, [(0.5, 0.5, 0.25)])[0]
    P = SweepPreconditioner(c, g, d=1).setup()
    u, its, hist = gmres(lambda v: apply_full(v, c, g), P.apply, f, tol=1e-10)
    ud = spla.spsolve(assemble_full(c, g).tocsc(), f.ravel())
    assert hist[-1] <= 1e-10
    assert its <= 15
    assert _rel(u, ud) < 1e-8


def test_gmres_identity_preconditioner_small():
    """Unpreconditioned GMRES (M = I) on a tiny system reaches the direct solution."""
    n, b = 3, 2
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_constant(n, b)
    f = W.random_rhs(1, n, b, seed=1)[0]
    u, its, hist = gmres(lambda v: apply_full(v, c, g), lambda v: v, f, tol=1e-12,
                         restart=400, maxit=400)
    ud = spla.spsolve(assemble_full(c, g).tocsc(), f.ravel())
    assert _rel(u, ud) < 1e-9


# ------------------------------------------------------ adjoint / gradient (a11) ---

def test_transpose_identity_adjoint_solve():
    """A^T = D^{-1} A D (A = D A_sym): the identity-based adjoint solve equals a
    sparse LU solve of the transposed matrix (a library special case)."""
    from oracle.adjoint import adjoint_solve_via_identity
    n, b = 5, 2
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=6)
    rhs = W.random_rhs(1, n, b, seed=13)[0]
    lam = adjoint_solve_via_identity(c, g, rhs)
    A = assemble_full(c, g)
    lam_ref = spla.spsolve(A.T.tocsc(), rhs.ravel())
    assert _rel(lam, lam_ref) < 1e-11


def test_velocity_gradient_matches_central_differences():
    """dL/dc = Re(lambda * 2 omega^2 c^-3 * u) against central finite differences
    (step 1e-4, direct FP64 solves) at seeded points, one of them in the PML
    padding; a wrong sign or a missing conjugate fails by O(1)."""
    from oracle.adjoint import loss, solve_all, velocity_gradient
    n, b = 5, 2
    g = Grid(n, b, W.omega_for(n))
    N = g.N
    c = W.velocity_lens(n, b)
    c_obs = W.velocity_bump(n, b, seed=1)
    centers = [(0.3, 0.5, 0.2), (0.6, 0.4, 0.2)]
    f = W.gaussian_sources(n, b, g.omega, centers)
    rec = np.zeros((N, N, N), dtype=bool)
    rec[b + n - 2, b:b + n, b:b + n] = True          # a receiver plane near the top
    d = solve_all(c_obs, g, f)[:, rec]
    L0, grad = velocity_gradient(c, g, f, rec, d)
    rng = np.random.default_rng(2)
    pts = [tuple(rng.integers(b, b + n, size=3)) for _ in range(4)] + [(0, b + 1, b + 2)]
    eps = 1e-4
    for p in pts:
        cp, cm = c.copy(), c.copy()
        cp[p] += eps
        cm[p] -= eps
        fd = (loss(solve_all(cp, g, f), rec, d) - loss(solve_all(cm, g, f), rec, d)) / (2 * eps)
        assert abs(fd - grad[p]) <= 1e-5 * max(abs(grad).max(), 1e-30), (p, fd, grad[p])


def test_restricted_operator_is_the_embed_solve_restrict_map():
    """|T~_{M'}| of Section 4.1 written as a matrix between chosen entries.

    Pinned twice: (1) on the block's own lines it reproduces the embed /
    solve / restrict procedure (restricted_apply) on random data, so the
    line and z-row bookkeeping of both agree; (2) each entry is an entry of
    the inverse of the assembled quasi-1D matrix, computed by a library
    sparse LU (a library routine as the special case).  A transposed index
    (rows and columns swapped) or a line offset by one fails (2)."""
    import scipy.sparse as sp
    n, b, d = 5, 2, 1
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=6)
    P = SweepPreconditioner(c, g, d=d)
    N = g.N
    rng = np.random.default_rng(11)
    for M, Mp in ((0, 0), (2, 3), (P.B - 1, 1)):
        py, (ia, ib) = P.ywin[Mp]
        pz, _ = P.zwin[M]
        lines = range(py.lo + ia, py.lo + ib)
        ent = [(x, line, lz) for line in lines for lz in range(pz.L) for x in range(N)]
        G = P.restricted_operator(M, Mp, ent, ent)
        alpha = rng.standard_normal((2, pz.L, ib - ia, N)) + 1j * rng.standard_normal((2, pz.L, ib - ia, N))
        q1 = P.quasi1d(M, Mp)
        ref = q1.restricted_apply(alpha)                       # (R, Lz, nl, N)
        vec = np.array([[alpha[r, lz, line - py.lo - ia, x] for (x, line, lz) in ent] for r in range(2)])
        got = vec @ G.T
        want = np.array([[ref[r, lz, line - py.lo - ia, x] for (x, line, lz) in ent] for r in range(2)])
        assert _rel(got, want) < 1e-12
        # (2) entries of the inverse of the assembled quasi-1D matrix
        k = q1.k
        A = sp.lil_matrix((N * k, N * k), dtype=np.complex128)
        for i in range(N):
            A[i * k:(i + 1) * k, i * k:(i + 1) * k] = q1.D[i]
            if i > 0:
                A[i * k + np.arange(k), (i - 1) * k + np.arange(k)] = q1.lower[i]
            if i < N - 1:
                A[i * k + np.arange(k), (i + 1) * k + np.arange(k)] = q1.upper[i]
        cols = ent[::7][:6]
        rows = ent[::5]
        Gs = P.restricted_operator(M, Mp, rows, cols)
        lu = spla.splu(A.tocsc())
        for j, (x, line, lz) in enumerate(cols):
            e = np.zeros(N * k, dtype=np.complex128)
            e[x * k + lz + pz.L * (line - py.lo)] = 1.0
            col = lu.solve(e)
            want = np.array([col[xr * k + lzr + pz.L * (liner - py.lo)] for (xr, liner, lzr) in rows])
            assert _rel(Gs[:, j], want) < 1e-11


def test_lens63_golden_is_the_oracle_solution_of_the_workload():
    """The stored n = 63 lens solution (written by tests/golden/make_lens63.py
    from the oracle) belongs to the workload the GPU test builds: same grid,
    frequency and source norm, a converged FP64 solve (relres <= 1e-10),
    distinct in-range sample indices, and its largest value sits at the
    source centre (0.5, 0.5, 0.25)."""
    import json
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "lens63_solution.json")))
    wl = W.lens_one_source(gold["n"], gold["b"], gold["d"])
    assert (gold["n"], gold["b"], gold["d"], gold["N"]) == (63, 6, 1, wl.N)
    assert abs(gold["omega"] - W.omega_for(63)) < 1e-12
    assert gold["relres_fp64"] <= 1e-10
    assert abs(gold["norm_f"] - np.linalg.norm(wl.f[0].astype(np.complex64))) <= 1e-6 * gold["norm_f"]
    idx = np.asarray(gold["index"])
    assert idx.min() >= 0 and idx.max() < wl.N ** 3 and len(set(idx.tolist())) == len(idx)
    u = np.abs(np.asarray(gold["re"]) + 1j * np.asarray(gold["im"]))
    z, y, x = np.unravel_index(idx[np.argmax(u)], (wl.N,) * 3)
    src = np.array([0.25, 0.5, 0.5]) * (wl.n + 1) + wl.b - 1        # (z, y, x) index of the source centre
    assert np.max(np.abs(np.array([z, y, x]) - src)) <= 3


# ---------------------------------------- two fronts (Sec. 4.2, third mod.) ---

def test_two_front_partition():
    """The two-front blocks tile the axis: the PML slabs, q blocks of d from
    each end, a centre of 1..2d layers, roles L..C..U in axis order."""
    for N, b, d in [(13, 3, 1), (14, 3, 2), (17, 2, 3), (9, 4, 1), (20, 3, 4)]:
        blocks, roles = axis_blocks_two_front(N, b, d)
        assert blocks[0] == (0, b) and blocks[-1] == (N - b, N)
        assert all(blocks[i][1] == blocks[i + 1][0] for i in range(len(blocks) - 1))
        c = roles.index("C")
        assert roles == ["L"] * c + ["C"] + ["U"] * (len(blocks) - c - 1)
        assert c == len(blocks) - 1 - c                          # as many blocks above as below
        assert 1 <= blocks[c][1] - blocks[c][0] <= 2 * d
        assert all(e - m == d for m, e in blocks[1:c] + blocks[c + 1:-1])


@pytest.mark.parametrize("n,d", [(15, 1), (15, 2)])
@pytest.mark.parametrize("b_aux", [1, 2, 3])
def test_two_front_windows_are_translated_boundary_problems(n, d, b_aux):
    """Section 3's translation argument for the windows of the two-front schedule
    (Sec. 4.2, third modification) with constant velocity, for auxiliary PMLs
    thinner than the boundary PML (Sec. 4.2, second modification) and as thick.

    The reference is the global profile of a grid with the same h and a PML of
    b_aux layers.  A lower-front window [m - b_aux, e) is that grid's first
    layers, an upper-front window [m, e + b_aux) its last layers, and the centre
    window [m - b_aux, e + b_aux) its first b_aux layers, interior layers, and
    last b_aux layers.  A moving PML measured from the wrong end, one layer off,
    of the boundary PML's thickness, or missing on one side fails it."""
    b = 3
    g = Grid(n, b, W.omega_for(n))
    N = g.N
    ga = Grid(n, b_aux, g.omega)                 # same h, PML of b_aux layers
    Na = ga.N
    ref = global_profile(ga)
    blocks, roles = axis_blocks_two_front(N, b, d)
    c = roles.index("C")
    checked = {"L": 0, "U": 0}
    for M in range(1, len(blocks) - 1):
        if M == c:
            continue
        m, e = blocks[M]
        role = roles[M]
        if m - b_aux < b or e + b_aux > N - b:
            continue                              # the window meets a real PML
        prof, (ia, ib) = axis_window(g, blocks, M, b_aux, role)
        L = prof.L
        if role == "L":
            assert (prof.lo, ia, ib, L) == (m - b_aux, b_aux, b_aux + e - m, e - m + b_aux)
            np.testing.assert_allclose(prof.s_node, ref.s_node[:L], rtol=0, atol=1e-15)
            np.testing.assert_allclose(prof.s_half, ref.s_half[:L + 1], rtol=0, atol=1e-15)
        else:
            assert (prof.lo, ia, ib, L) == (m, 0, e - m, e - m + b_aux)
            np.testing.assert_allclose(prof.s_node, ref.s_node[Na - L:], rtol=0, atol=1e-15)
            np.testing.assert_allclose(prof.s_half, ref.s_half[Na - L:], rtol=0, atol=1e-15)
        checked[role] += 1
    assert checked["L"] >= 1 and checked["U"] >= 1
    m, e = blocks[c]
    dc = e - m
    prof, (ia, ib) = axis_window(g, blocks, c, b_aux, "C")
    L = prof.L
    assert (prof.lo, ia, ib, L) == (m - b_aux, b_aux, b_aux + dc, 2 * b_aux + dc)
    assert m - b_aux >= b and e + b_aux <= N - b   # an interior centre: no real PML inside the window
    want_node = np.concatenate([ref.s_node[:b_aux], ref.s_node[b_aux:b_aux + dc], ref.s_node[Na - b_aux:]])
    want_half = np.concatenate([ref.s_half[:b_aux + 1], ref.s_half[b_aux + 1:b_aux + dc],
                                ref.s_half[Na - b_aux:]])
    np.testing.assert_allclose(ref.s_node[b_aux:b_aux + dc], 1.0, rtol=0, atol=0)   # interior: no stretching
    np.testing.assert_allclose(prof.s_node, want_node, rtol=0, atol=1e-15)
    np.testing.assert_allclose(prof.s_half, want_half, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n,b,d", [(3, 2, 1), (4, 2, 2), (5, 2, 1)])
@pytest.mark.parametrize("inner", ["sweep", "exact"])
def test_two_front_exact_limit_gives_inverse(n, b, d, inner):
    """With b_aux >= N every two-front window reaches the faces: the lower
    front's problems are the leading blocks of the real operator, the upper
    front's the trailing blocks, the centre's the whole operator, so each
    |T| is an exact Schur-complement operator of the block LDU eliminated from
    both ends (a twisted factorisation), at both levels, and the
    preconditioner equals A^{-1}.  Pins the upper front's couplings and
    order and the centre's two couplings."""
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=2)
    A = assemble_full(c, g)
    f = W.random_rhs(2, n, b, seed=5)
    P = SweepPreconditioner(c, g, d=d, b_aux=g.N + 1, inner=inner, schedule="two_front").setup()
    z = P.apply(f)
    for r in range(2):
        assert _rel(z[r], spla.spsolve(A.tocsc(), f[r].ravel())) < 1e-11


@pytest.mark.parametrize("n,b,d,b_aux", [(7, 3, 1, 3), (8, 2, 2, 2), (7, 3, 2, 1)])
def test_two_front_is_mirror_symmetric(n, b, d, b_aux):
    """The discretisation (Section 2: the same PML on both faces) and the
    two-front schedule are symmetric under reflecting x3 and x2: the upper
    front's windows, moving PMLs and couplings are the mirror images of the
    lower front's.  So M applied to the reflected velocity and right-hand
    side gives the reflected result.  (One front is not symmetric.)  A slip
    in an upper-front window (wall position, profile direction) or coupling
    (c_up / c_dn, layer) breaks the symmetry."""
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_random(n, b, seed=9)
    f = W.random_rhs(1, n, b, seed=10)
    flip = lambda a: a[..., ::-1, ::-1, :]                     # (z, y, x): reflect z and y
    z1 = SweepPreconditioner(c, g, d=d, b_aux=b_aux, schedule="two_front").apply(f)
    z2 = SweepPreconditioner(np.ascontiguousarray(flip(c)), g, d=d, b_aux=b_aux,
                             schedule="two_front").apply(np.ascontiguousarray(flip(f)))
    assert _rel(flip(z2), z1) < 1e-12
    z3 = SweepPreconditioner(np.ascontiguousarray(flip(c)), g, d=d, b_aux=b_aux).apply(
        np.ascontiguousarray(flip(f)))
    z4 = SweepPreconditioner(c, g, d=d, b_aux=b_aux).apply(f)
    assert _rel(flip(z3), z4) > 1e-6                            # the one-front schedule is not


def test_two_front_gmres_converges_like_one_front():
    """Right-preconditioned GMRES with the two-front preconditioner reaches
    the direct solution; the iteration count stays close to one front's."""
    n, b = 9, 3
    g = Grid(n, b, W.omega_for(n))
    c = W.velocity_lens(n, b)
    f = W.gaussian_sources(n, b, g.omega, [(0.5, 0.5, 0.25)])[0]
    ud = spla.spsolve(assemble_full(c, g).tocsc(), f.ravel())
    its = {}
    for sched in ("one_front", "two_front"):
        P = SweepPreconditioner(c, g, d=1, schedule=sched).setup()
        u, its[sched], hist = gmres(lambda v: apply_full(v, c, g), P.apply, f, tol=1e-10)
        assert _rel(u, ud) < 1e-8
    assert its["two_front"] <= its["one_front"] + 4

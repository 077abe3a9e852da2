"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerances (complex FP32 kernels against FP64):
  * stencil c64: max |y - y_oracle| <= 2e-6 max |y_oracle|; c128: 1e-12
  * preconditioner apply: ||z - z_oracle|| / ||z_oracle|| <= 1e-5 per RHS
  * solve at tol 1e-6: ||u - u_direct|| / ||u_direct|| <= 1e-5 per RHS
The oracle receives the FP32-rounded velocity and sources the GPU receives,
so both sides discretise the same operator.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.krylov import gmres
from oracle.operator import Grid, apply_full, assemble_full
from oracle.sweep import SweepPreconditioner
from paper_1502_07266_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import helm as H
    return H


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def _inputs(n, b, kind="lens", R=2, seed=0):
    om = W.omega_for(n)
    if kind == "lens":
        c = W.velocity_lens(n, b)
    elif kind == "random":
        c = W.velocity_random(n, b, seed=seed)
    else:
        c = W.velocity_constant(n, b)
    c32 = c.astype(np.float32)
    f = W.random_rhs(R, n, b, seed=seed + 100).astype(np.complex64)
    return om, c32, f


def _solver(helm, c32, om, n, b, d, **kw):
    return helm.Solver(torch.from_numpy(c32).cuda(), om, n, b, d, **kw)


# ---------------------------------------------------------------- stencil ---

@pytest.mark.parametrize("n,b", [(7, 3), (10, 2), (33, 4)])
def test_matvec_parity(helm, n, b):
    om, c32, f = _inputs(n, b, "random", R=3)
    S = _solver(helm, c32, om, n, b, 1)
    g = Grid(n, b, om)
    c64 = c32.astype(np.float64)
    y = S.matvec(torch.from_numpy(f).cuda()).cpu().numpy()
    yo = apply_full(f.astype(np.complex128), c64, g)
    assert np.abs(y - yo).max() <= 2e-6 * np.abs(yo).max()
    y64 = S.matvec(torch.from_numpy(f.astype(np.complex128)).cuda()).cpu().numpy()
    assert np.abs(y64 - yo).max() <= 1e-12 * np.abs(yo).max()
    S.close()


# ------------------------------------------------------ preconditioner apply ---

@pytest.mark.parametrize("n,b,d,kind", [(7, 3, 1, "lens"), (8, 2, 3, "random"), (15, 4, 1, "random"),
                                        (5, 2, 2, "const"), (6, 3, 1, "random"), (1, 1, 1, "lens")])
def test_apply_parity(helm, n, b, d, kind):
    """Algorithm 6 on the GPU equals the oracle's, several tiles and a ragged last block."""
    om, c32, f = _inputs(n, b, kind, R=3, seed=n)
    S = _solver(helm, c32, om, n, b, d)
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    assert S.status() == helm.HELM_OK
    zo = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d).apply(f.astype(np.complex128))
    for r in range(f.shape[0]):
        assert _rel(z[r], zo[r]) <= 1e-5
    S.close()


@pytest.mark.parametrize("n,b", [(7, 3), (7, 4), (9, 4), (4, 6), (1, 1), (2, 1)])
def test_apply_rhs_batch(helm, n, b):
    """A batch gives the single-RHS results; shared-memory layouts with an odd
    N*k (n=7, b=4: N=15, k=25), block sizes above 32 (b=6: k up to 49), and the
    smallest grids (N=3, 4: one elimination step per half)."""
    om, c32, f = _inputs(n, b, "lens", R=5, seed=3)
    S = _solver(helm, c32, om, n, b, 1)
    ft = torch.from_numpy(f).cuda()
    zb = S.apply(ft).cpu().numpy()
    for r in range(5):
        z1 = S.apply(ft[r:r + 1].contiguous()).cpu().numpy()[0]
        assert _rel(zb[r], z1) <= 1e-6
    S.close()


def test_apply_exact_limit_is_inverse(helm):
    """b_aux >= N: every window is the leading block of A and M = A^{-1}."""
    n, b = 3, 2
    om, c32, f = _inputs(n, b, "random", R=2, seed=7)
    N = n + 2 * b
    S = _solver(helm, c32, om, n, b, 1, b_aux=N + 1)
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    A = assemble_full(c32.astype(np.float64), Grid(n, b, om)).tocsc()
    for r in range(2):
        assert _rel(z[r], spla.spsolve(A, f[r].astype(np.complex128).ravel())) <= 1e-5
    S.close()


def test_apply_zero_and_linearity(helm):
    n, b = 7, 3
    om, c32, f = _inputs(n, b, "lens", R=2, seed=5)
    S = _solver(helm, c32, om, n, b, 1)
    ft = torch.from_numpy(f).cuda()
    z0 = S.apply(torch.zeros_like(ft)).cpu().numpy()
    assert np.all(z0 == 0)
    za = S.apply(ft).cpu().numpy()
    zs = S.apply((2.0 * ft).contiguous()).cpu().numpy()
    assert _rel(zs, 2.0 * za) <= 1e-6
    S.close()


# ---------------------------------------------------------------- solves ---

@pytest.mark.parametrize("n,b,kind", [(7, 3, "lens"), (9, 3, "random")])
def test_solve_matches_direct(helm, n, b, kind):
    om, c32, f = _inputs(n, b, kind, R=3, seed=11)
    S = _solver(helm, c32, om, n, b, 1)
    u, its, rel, code = S.solve(torch.from_numpy(f).cuda(), tol=1e-6)
    assert code == helm.HELM_OK and max(rel) <= 1e-6
    A = assemble_full(c32.astype(np.float64), Grid(n, b, om)).tocsc()
    u = u.cpu().numpy()
    for r in range(3):
        ud = spla.spsolve(A, f[r].astype(np.complex128).ravel())
        assert _rel(u[r], ud) <= 1e-5
        # the FP64 residual the solver reports is the true one
        rr = np.linalg.norm(f[r].ravel() - A @ u[r].ravel().astype(np.complex128)) / np.linalg.norm(f[r])
        assert rr <= 2e-6
    assert max(its) <= 30
    S.close()


@pytest.mark.slow
def test_solve_small_constant_config(helm):
    """n=31, b=6, c=1, one centred Gaussian source (the small configuration):
    the GPU solution matches the oracle's GMRES solution (tol 1e-10)."""
    wl = W.small_constant()
    c32 = wl.c.astype(np.float32)
    f = wl.f.astype(np.complex64)
    S = _solver(helm, c32, wl.omega, wl.n, wl.b, wl.d)
    u, its, rel, code = S.solve(torch.from_numpy(f).cuda(), tol=1e-6)
    assert code == helm.HELM_OK
    g = Grid(wl.n, wl.b, wl.omega)
    c64 = c32.astype(np.float64)
    P = SweepPreconditioner(c64, g, d=wl.d).setup()
    uo, its_o, hist = gmres(lambda v: apply_full(v, c64, g), P.apply, f[0].astype(np.complex128),
                            tol=1e-10)
    assert _rel(u.cpu().numpy()[0], uo) <= 1e-5
    # same preconditioner: iteration counts agree closely at the same tolerance
    S.close()


# ------------------------------------------------------ full size, sampled ---

@pytest.mark.slow
def test_full_size_slab_and_matvec_sampled(helm):
    """n=127, b=6 (139^3 unknowns, the 64-source workload's grid): the matvec on
    two RHS, and one interior slab's Algorithm 4 apply, against the oracle."""
    n, b, d = 127, 6, 1
    om = W.omega_for(n)
    c32 = W.velocity_random(n, b, seed=0).astype(np.float32)
    S = _solver(helm, c32, om, n, b, d)
    N = n + 2 * b
    rng = np.random.default_rng(1)
    x = (rng.standard_normal((2, N, N, N)) + 1j * rng.standard_normal((2, N, N, N))).astype(np.complex64)
    y = S.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    g = Grid(n, b, om)
    c64 = c32.astype(np.float64)
    yo = apply_full(x.astype(np.complex128), c64, g)
    assert np.abs(y - yo).max() <= 2e-6 * np.abs(yo).max()
    P = SweepPreconditioner(c64, g, d=d, keep_factors=False)
    for M in (1, 70):
        Lz = helm.helm_slab_layers(S.handle, M)
        gs = (rng.standard_normal((1, Lz, N, N)) + 1j * rng.standard_normal((1, Lz, N, N))).astype(np.complex64)
        v = S.apply_slab(M, torch.from_numpy(gs).cuda()).cpu().numpy()
        vo = P.inner_sweep(M, gs.astype(np.complex128))
        assert _rel(v, vo) <= 1e-5
    S.close()


# ------------------------------------------------------------ edge cases ---

def test_invalid_arguments(helm):
    n, b = 5, 2
    om, c32, f = _inputs(n, b, "lens", R=1)
    ct = torch.from_numpy(c32).cuda()
    with pytest.raises(helm.HelmError) as e:
        helm.helm_setup(ct.data_ptr(), om, 0, b, 1)
    assert e.value.code == helm.HELM_EINVAL
    with pytest.raises(helm.HelmError) as e:
        helm.helm_setup(ct.data_ptr(), -om, n, b, 1)
    assert e.value.code == helm.HELM_EINVAL
    bad = ct.clone()
    bad[2, 2, 2] = -1.0
    with pytest.raises(helm.HelmError) as e:
        helm.helm_setup(bad.data_ptr(), om, n, b, 1)
    assert e.value.code == helm.HELM_EINVAL
    # (b + d)^2 > 64 is valid mathematics but not supported by the kernels
    c9 = torch.ones((3 + 18) ** 3, device="cuda", dtype=torch.float32)
    with pytest.raises(helm.HelmError) as e:
        helm.helm_setup(c9.data_ptr(), om, 3, 9, 1)
    assert e.value.code == helm.HELM_ENOTSUP
    S = _solver(helm, c32, om, n, b, 1)
    with pytest.raises(helm.HelmError):
        helm.helm_apply_precond(S.handle, 0, 0, 1)
    with pytest.raises(helm.HelmError):
        helm.helm_apply_slab(S.handle, 10 ** 6, 16, 32, 1)
    S.close()


def test_apply_more_clusters_than_sms(helm):
    """200 right-hand sides launch 400 CTAs, more than the GPU holds at once: the
    clusters that wait for an SM must not hold back the pacing of the running
    ones.  Each right-hand side's result is independent of the others (equal to
    the chunked applies bit for bit) and matches the oracle; the whole apply
    stays within a few waves of one chunk's time (a stalled pacing would cost
    about 0.2 ms per solve, tens of times more).  Times are CUDA-event device
    times, so host jitter does not enter."""
    n, b, R = 5, 2, 200
    om, c32, f = _inputs(n, b, "random", R=R, seed=9)
    S = _solver(helm, c32, om, n, b, 1)
    x = torch.from_numpy(f).cuda()

    def timed_apply(xx, zz):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        zz = S.apply(xx, zz)
        e1.record()
        torch.cuda.synchronize()
        return zz, e0.elapsed_time(e1) * 1e-3

    z = S.apply(x)
    torch.cuda.synchronize()
    z, t_all = timed_apply(x, z)
    assert S.status() == helm.HELM_OK
    parts, t_chunk = [], 0.0
    for q in range(0, R, 20):
        xc = x[q:q + 20].contiguous()
        zc = S.apply(xc)
        torch.cuda.synchronize()
        zc, t = timed_apply(xc, zc)
        t_chunk = max(t_chunk, t)
        parts.append(zc)
    assert torch.equal(z, torch.cat(parts))
    zo = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=1).apply(f[:2].astype(np.complex128))
    zz = z[:2].cpu().numpy()
    for r in range(2):
        assert _rel(zz[r], zo[r]) <= 1e-5
    assert t_all <= 20 * t_chunk + 0.05
    S.close()


@pytest.mark.parametrize("n,b,d,b_aux", [(7, 3, 1, 2), (8, 2, 2, 4), (9, 3, 1, 5)])
def test_apply_parity_auxiliary_pml_width(helm, n, b, d, b_aux):
    """Section 4.2's second modification: a moving-PML width b_aux different from
    b (windows of b_aux + d layers) on both sides of the comparison."""
    om, c32, f = _inputs(n, b, "random", R=2, seed=n + b_aux)
    S = _solver(helm, c32, om, n, b, d, b_aux=b_aux)
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    assert S.status() == helm.HELM_OK
    zo = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d,
                             b_aux=b_aux).apply(f.astype(np.complex128))
    for r in range(f.shape[0]):
        assert _rel(z[r], zo[r]) <= 1e-5
    S.close()


def test_apply_parity_pml_constant(helm):
    """A PML constant C other than 10 reaches the coefficients (Section 2)."""
    n, b = 7, 3
    om, c32, f = _inputs(n, b, "lens", R=2, seed=3)
    S = _solver(helm, c32, om, n, b, 1, pml_C=5.0)
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    y = S.matvec(torch.from_numpy(f).cuda()).cpu().numpy()
    g = Grid(n, b, om, C=5.0)
    c64 = c32.astype(np.float64)
    zo = SweepPreconditioner(c64, g, d=1).apply(f.astype(np.complex128))
    yo = apply_full(f.astype(np.complex128), c64, g)
    for r in range(f.shape[0]):
        assert _rel(z[r], zo[r]) <= 1e-5
    assert np.abs(y - yo).max() <= 2e-6 * np.abs(yo).max()
    S.close()


def test_solve_short_restart_matches_direct(helm):
    """GMRES(10): more restarts, each from the FP64 true residual, same answer."""
    n, b = 9, 3
    om = W.omega_for(n)
    c32 = W.velocity_random(n, b, seed=5).astype(np.float32)
    f = W.gaussian_sources(n, b, om, [(0.4, 0.5, 0.5)]).astype(np.complex64)
    S = _solver(helm, c32, om, n, b, 1, restart=10)
    u, its, rel, code = S.solve(torch.from_numpy(f).cuda(), tol=1e-6)
    assert code == helm.HELM_OK and max(rel) <= 1e-6
    A = assemble_full(c32.astype(np.float64), Grid(n, b, om)).tocsc()
    ud = spla.spsolve(A, f[0].astype(np.complex128).ravel()).reshape(f[0].shape)
    assert _rel(u.cpu().numpy()[0], ud) <= 1e-5
    S.close()

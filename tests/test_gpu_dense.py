"""Dense restricted-operator form (HELM_DENSE) against the FP64 oracle, through the C ABI.

The dense form stores, per quasi-1D problem, the map |T~_{M'}| of Section 4.1
between the entries Algorithms 4 and 6 feed and read, and applies each
quasi-1D solve as one matrix product.  It is the same preconditioner M as the
substitution chain, so the oracle's Algorithm 6 is the reference.

Tolerances (against FP64):
  * stored operator (FP32, split FP16): max |G - G_oracle| <= 1e-5 max |G_oracle|
    on every compared operator; FP16 hi: 2^-10 relative to each row's largest part
  * preconditioner apply (FP32, split FP16): ||z - z_oracle|| / ||z_oracle|| <= 1e-5
    per RHS; FP16 hi operators: <= 3e-3 (their storage rounding, 2^-11 per entry)
  * solve at tol 1e-6: ||u - u_direct|| / ||u_direct|| <= 1e-5 per RHS
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.operator import Grid, assemble_full
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
    c = {"lens": W.velocity_lens, "random": lambda n, b: W.velocity_random(n, b, seed=seed),
         "const": W.velocity_constant}[kind](n, b)
    c32 = c.astype(np.float32)
    f = W.random_rhs(R, n, b, seed=seed + 100).astype(np.complex64)
    return om, c32, f


def _solver(helm, c32, om, n, b, d, **kw):
    return helm.Solver(torch.from_numpy(c32).cuda(), om, n, b, d, apply_form="dense", **kw)


def _entries(rect_in, rects_out, N):
    line0, nl, z0, nz = rect_in
    cols = []
    for j in range(nl * nz * N):
        per = nz * nl
        x, r = divmod(j, per)
        cols.append((x, line0 + r // nz, z0 + r % nz))
    rows = []
    for (l0, nlr, zr0, nzr) in rects_out:
        for o in range(nlr * nzr * N):
            x, t = o % N, o // N
            rows.append((x, l0 + t // nzr, zr0 + t % nzr))
    return rows, cols


# ----------------------------------------------------------- stored operators ---

@pytest.mark.parametrize("n,b,d", [(7, 3, 1), (8, 2, 3), (9, 6, 1)])
@pytest.mark.parametrize("precision", ["fp32", "split_fp16", "fp16"])
def test_operator_matches_oracle(helm, n, b, d, precision):
    """Each stored G equals R_out H~^{-1} R_in^T of the oracle's quasi-1D problem
    (interior blocks, the first line block's forward and backward maps, the
    first slab and the last line block)."""
    om, c32, _ = _inputs(n, b, "random", R=1, seed=3)
    S = _solver(helm, c32, om, n, b, d, precision=precision)
    P = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d)
    B = P.B
    for M, Mp, dr in ((1, 2, 0), (B - 1, B - 1, 0), (0, 0, 0), (2, 0, 0), (2, 0, 1), (0, 0, 1), (B // 2, 1, 0)):
        Gt, rin, rout = S.dense_operator(M, Mp, dr)
        G = Gt.cpu().numpy().astype(np.complex128)
        rows, cols = _entries(rin, rout, S.N)
        Go = P.restricted_operator(M, Mp, rows, cols)
        assert G.shape == Go.shape
        if precision == "fp16":
            # per real row: error within 2^-10 of the row's largest part
            for part in (np.real, np.imag):
                mx = np.abs(part(Go)).max(axis=1, keepdims=True)
                assert np.all(np.abs(part(G) - part(Go)) <= 2.0 ** -10 * mx + 1e-30)
        else:
            assert np.abs(G - Go).max() <= 1e-5 * np.abs(Go).max(), (M, Mp, dr)
    S.close()


def test_full_size_operators_sampled(helm):
    """n = 127, b = 6, d = 1 (the 64-source workload's grid, k = 49, 973 x 973
    interior operators): sampled rows and columns of three stored operators of
    one slab against the oracle's quasi-1D solves (FP32 form)."""
    wl = W.random_64_sources(n=127, b=6, d=1, seed=0, per_side=1)
    c32 = wl.c.astype(np.float32)
    S = _solver(helm, c32, wl.omega, wl.n, wl.b, wl.d)
    P = SweepPreconditioner(c32.astype(np.float64), Grid(wl.n, wl.b, wl.omega), d=wl.d, keep_factors=False)
    rng = np.random.default_rng(5)
    for M, Mp, dr in ((67, 40, 0), (67, 0, 0), (67, 0, 1), (130, 133, 0)):
        Gt, rin, rout = S.dense_operator(M, Mp, dr)
        rows, cols = _entries(rin, rout, S.N)
        ri = np.sort(rng.choice(len(rows), size=24, replace=False))
        ci = np.sort(rng.choice(len(cols), size=12, replace=False))
        G = Gt[torch.as_tensor(ri).cuda()][:, torch.as_tensor(ci).cuda()].cpu().numpy()
        Go = P.restricted_operator(M, Mp, [rows[i] for i in ri], [cols[j] for j in ci])
        scale = float(Gt.abs().max())             # the operator's largest entry sets the FP32 error scale
        assert scale > 0 and np.abs(G - Go).max() <= 1e-5 * scale, (M, Mp, dr)
        del Gt
    S.close()


# ----------------------------------------------------------------- applies ---

CASES = [(7, 3, 1, "lens"), (8, 2, 3, "random"), (15, 4, 1, "random"), (5, 2, 2, "const"),
         (9, 6, 1, "random"), (1, 1, 1, "lens"), (6, 3, 1, "random")]


@pytest.mark.parametrize("n,b,d,kind", CASES)
@pytest.mark.parametrize("precision", ["fp32", "split_fp16"])
def test_apply_parity(helm, n, b, d, kind, precision):
    """Algorithm 6 with dense operators equals the oracle's, per RHS."""
    om, c32, f = _inputs(n, b, kind, R=3, seed=n)
    S = _solver(helm, c32, om, n, b, d, precision=precision)
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    assert S.status() == helm.HELM_OK
    zo = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d).apply(f.astype(np.complex128))
    for r in range(f.shape[0]):
        assert _rel(z[r], zo[r]) <= 1e-5, (r, _rel(z[r], zo[r]))
    S.close()


def test_apply_parity_fp16_operators(helm):
    """FP16 hi operators: within their storage rounding of the oracle, and the
    split form within 1e-5."""
    n, b, d = 9, 6, 1
    om, c32, f = _inputs(n, b, "random", R=2, seed=4)
    zo = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d).apply(f.astype(np.complex128))
    S = _solver(helm, c32, om, n, b, d, precision="fp16")
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    S.close()
    errs = [_rel(z[r], zo[r]) for r in range(2)]
    assert max(errs) <= 3e-3 and min(errs) > 1e-7, errs      # rounded, and not the FP32 result


def test_apply_many_rhs_and_padding(helm):
    """70 right-hand sides (two launches of <= 64) and 20 (padded to 32)."""
    n, b, d = 5, 2, 1
    om, c32, f = _inputs(n, b, "random", R=70, seed=9)
    zo = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d).apply(f.astype(np.complex128))
    for precision in ("fp32", "split_fp16"):
        S = _solver(helm, c32, om, n, b, d, precision=precision)
        for R in (70, 20):
            z = S.apply(torch.from_numpy(np.ascontiguousarray(f[:R])).cuda()).cpu().numpy()
            errs = [_rel(z[r], zo[r]) for r in range(R)]
            assert max(errs) <= 1e-5, (precision, R, max(errs))
        S.close()


def test_dense_equals_chain(helm):
    """The two apply forms give the same M (FP32 rounding apart)."""
    n, b, d = 15, 4, 1
    om, c32, f = _inputs(n, b, "lens", R=2, seed=2)
    ft = torch.from_numpy(f).cuda()
    Sd = _solver(helm, c32, om, n, b, d)
    Sc = helm.Solver(torch.from_numpy(c32).cuda(), om, n, b, d)
    zd, zc = Sd.apply(ft).cpu().numpy(), Sc.apply(ft).cpu().numpy()
    for r in range(2):
        assert _rel(zd[r], zc[r]) <= 2e-6
    Sd.close()
    Sc.close()


# ------------------------------------------------------------------- solves ---

@pytest.mark.parametrize("precision", ["fp32", "split_fp16", "fp16"])
def test_solve_matches_direct(helm, precision):
    n, b, d = 15, 6, 1
    om, c32, f = _inputs(n, b, "random", R=2, seed=12)
    S = _solver(helm, c32, om, n, b, d, precision=precision)
    u, its, rel, code = S.solve(torch.from_numpy(f).cuda(), tol=1e-6)
    assert code == helm.HELM_OK and max(rel) <= 1e-6
    A = assemble_full(c32.astype(np.float64), Grid(n, b, om)).tocsc()
    u = u.cpu().numpy()
    for r in range(2):
        ud = spla.spsolve(A, f[r].astype(np.complex128).ravel())
        assert _rel(u[r].ravel(), ud) <= 1e-5
    S.close()


# ----------------------------------------------------------- failure paths ---

def test_unmet_wait_times_out_and_reports(helm):
    """A wait whose arrival never comes (the test hook) expires after its bound:
    the kernel returns, helm_status reports HELM_ETIMEOUT, and the GPU context
    stays usable (a normal apply afterwards matches the oracle)."""
    n, b, d = 5, 2, 1
    om, c32, f = _inputs(n, b, "lens", R=2, seed=1)
    ft = torch.from_numpy(f).cuda()
    for precision in ("fp32", "split_fp16"):
        S = _solver(helm, c32, om, n, b, d, precision=precision, debug_unmet_wait=True, wait_cycles=20_000_000)
        S.apply(ft)
        with pytest.raises(helm.HelmError) as e:
            S.status()
        assert e.value.code == helm.HELM_ETIMEOUT
        S.close()
    S = _solver(helm, c32, om, n, b, d)
    z = S.apply(ft).cpu().numpy()
    assert S.status() == helm.HELM_OK
    zo = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d).apply(f.astype(np.complex128))
    assert _rel(z, zo) <= 1e-5
    S.close()


def test_gmres_reports_no_convergence(helm):
    """maxit = 2: HELM_ENOCONV, with the solution, iteration counts and the
    true residual still written (both apply forms)."""
    n, b, d = 9, 3, 1
    om, c32, f = _inputs(n, b, "random", R=2, seed=7)
    for form in ("chain", "dense"):
        S = helm.Solver(torch.from_numpy(c32).cuda(), om, n, b, d, maxit=2, apply_form=form)
        u = torch.full_like(torch.from_numpy(f).cuda(), float("nan"))
        u, its, rel, code = S.solve(torch.from_numpy(f).cuda(), tol=1e-12, u=u)
        assert code == helm.HELM_ENOCONV
        assert its == [2, 2] and all(0 < r < 1 for r in rel)
        assert torch.isfinite(torch.view_as_real(u)).all()
        S.close()


def test_wave_packet_source(helm):
    """The paper's second force, a Gaussian wave packet along (0, 1, 1)/sqrt 2
    (this library's definition of it): the split-precision dense solve
    matches a direct solve, and at c = 1 the field a distance ahead of the
    packet along its direction is far larger than the same distance behind."""
    n, b, d = 31, 6, 1
    om = W.omega_for(n)
    c32 = W.velocity_constant(n, b).astype(np.float32)
    f = W.wave_packet(n, b, om).astype(np.complex64)
    S = _solver(helm, c32, om, n, b, d, precision="split_fp16")
    u, its, rel, code = S.solve(torch.from_numpy(f).cuda(), tol=1e-6)
    S.close()
    assert code == helm.HELM_OK
    u = u.cpu().numpy()[0]
    A = assemble_full(c32.astype(np.float64), Grid(n, b, om)).tocsc()
    ud = spla.spsolve(A, f[0].astype(np.complex128).ravel()).reshape(u.shape)
    assert _rel(u, ud) <= 1e-5
    x = W.padded_coords(n, b)

    def amp(p):
        iz, iy, ix = (int(np.argmin(np.abs(x - v))) for v in (p[2], p[1], p[0]))
        return np.abs(u[iz - 1:iz + 2, iy - 1:iy + 2, ix - 1:ix + 2]).mean()

    s = 0.2 / np.sqrt(2.0)
    ahead, behind = amp((0.5, 0.25 + s, 0.25 + s)), amp((0.5, 0.25 - s, 0.25 - s))
    assert ahead > 10 * behind, (ahead, behind)


@pytest.mark.parametrize("n,b,clusters", [(18, 4, 2), (31, 4, 3)])
@pytest.mark.parametrize("precision", ["fp32", "split_fp16"])
def test_tiles_with_extra_rows(helm, n, b, clusters, precision):
    """Operators of 65 rows per resident cluster (130 rows on 2 clusters, 195 on
    3) are tiled as 64 tensor-core rows plus one FP32 row: the stored
    operators and the apply still match the oracle."""
    d = 1
    om, c32, f = _inputs(n, b, "random", R=3, seed=n + clusters)
    S = _solver(helm, c32, om, n, b, d, precision=precision, dense_clusters=clusters)
    P = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d)
    Gt, rin, rout = S.dense_operator(3, 2, 0)
    assert Gt.shape[0] == 65 * clusters
    rows, cols = _entries(rin, rout, S.N)
    Go = P.restricted_operator(3, 2, rows, cols)
    assert np.abs(Gt.cpu().numpy() - Go).max() <= 1e-5 * np.abs(Go).max()
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    assert S.status() == helm.HELM_OK
    zo = P.apply(f.astype(np.complex128))
    for r in range(f.shape[0]):
        assert _rel(z[r], zo[r]) <= 1e-5
    S.close()


@pytest.mark.parametrize("precision", ["split_fp16", "fp16"])
def test_tiny_columns_keep_their_scale(helm, precision):
    """A right-hand side of magnitude 1e-36 (its gathered columns near the
    bottom of the FP32 range, where 2^(15 - e) would overflow): the
    power-of-two column scales stay finite and the apply matches the oracle
    to the same relative accuracy as an O(1) right-hand side."""
    n, b, d = 9, 6, 1
    om, c32, f = _inputs(n, b, "random", R=2, seed=17)
    f[1] *= np.float32(1e-36)
    S = _solver(helm, c32, om, n, b, d, precision=precision)
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    S.close()
    zo = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d).apply(f.astype(np.complex128))
    tol = 1e-5 if precision == "split_fp16" else 3e-3
    assert np.all(np.isfinite(z))
    for r in range(2):
        assert _rel(z[r], zo[r]) <= tol, (r, _rel(z[r], zo[r]))

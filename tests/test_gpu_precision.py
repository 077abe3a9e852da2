"""Precision pattern on the GPU: stored-factor formats against the oracle.

The oracle applies the same twisted factorisation with its FP64 factors
rounded to the same stored form (oracle.precision).  Tolerances:
  * HELM_SPLIT_FP16: as the FP32 path, ||z - z_oracle|| / ||z_oracle|| <= 1e-5
    (the pair keeps about 22 bits; the FP32 setup's own error dominates).
  * HELM_FP16 against the FP16 oracle: <= 1e-4.  The GPU rounds its FP32 T_i,
    the oracle its FP64 T_i; the two agree to about 1e-6 relative, so an entry's
    FP16 value differs only where that difference crosses a rounding boundary
    (a fraction ~1e-6 / 2^-11 of the entries, by one unit of 2^-11).  Against
    the FP64 oracle the same result differs by the FP16 rounding itself
    (a few 1e-4), which the test also requires, so a path that skipped the
    rounding would fail.
  * solves reach the FP64 true residual tolerance in every format.
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


def _case(n, b, kind, R=3):
    om = W.omega_for(n)
    c = W.velocity_lens(n, b) if kind == "lens" else W.velocity_random(n, b, seed=n)
    return om, c.astype(np.float32), W.random_rhs(R, n, b, seed=n + 100).astype(np.complex64)


@pytest.mark.parametrize("n,b,d,kind", [(7, 3, 1, "lens"), (8, 2, 3, "random"), (15, 4, 1, "random"),
                                        (1, 1, 1, "lens")])
def test_apply_parity_fp16(helm, n, b, d, kind):
    om, c32, f = _case(n, b, kind)
    S = helm.Solver(torch.from_numpy(c32).cuda(), om, n, b, d, precision="fp16")
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    assert S.status() == helm.HELM_OK
    g = Grid(n, b, om)
    c64, f64 = c32.astype(np.float64), f.astype(np.complex128)
    z16 = SweepPreconditioner(c64, g, d=d, factor_format="fp16").apply(f64)
    z64 = SweepPreconditioner(c64, g, d=d).apply(f64)
    for r in range(f.shape[0]):
        assert _rel(z[r], z16[r]) <= 1e-4
        if n > 1:
            assert _rel(z[r], z64[r]) > 3 * _rel(z[r], z16[r])
    S.close()


@pytest.mark.parametrize("n,b,d,kind", [(7, 3, 1, "lens"), (8, 2, 3, "random"), (15, 4, 1, "random")])
def test_apply_parity_split_fp16(helm, n, b, d, kind):
    om, c32, f = _case(n, b, kind)
    S = helm.Solver(torch.from_numpy(c32).cuda(), om, n, b, d, precision="split_fp16")
    z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
    assert S.status() == helm.HELM_OK
    zs = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d,
                             factor_format="split_fp16").apply(f.astype(np.complex128))
    for r in range(f.shape[0]):
        assert _rel(z[r], zs[r]) <= 1e-5
    S.close()


def test_factor_bytes_per_format(helm):
    """Stored bytes follow the layout: k rows of ldk entries, ldk = ceil8(k) + 2
    (8-byte entries) or ceil8(k) + 4 (4-byte FP16 entries), N blocks per problem."""
    n, b = 9, 3
    om, c32, _ = _case(n, b, "random", R=1)
    c = torch.from_numpy(c32).cuda()
    sizes = {}
    for fmt in ("fp32", "fp16", "split_fp16"):
        S = helm.Solver(c, om, n, b, 1, precision=fmt)
        sizes[fmt] = helm.helm_factor_bytes(S.handle)
        S.close()
    P = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=1)
    N = n + 2 * b
    ks = [P.zwin[M][0].L * P.ywin[Mp][0].L for M in range(P.B) for Mp in range(P.B)]
    c8 = [8 * ((k + 7) // 8) for k in ks]
    assert sizes["fp32"] == sum(N * k * (c + 2) * 8 for k, c in zip(ks, c8))
    assert sizes["split_fp16"] == sizes["fp32"]
    assert sizes["fp16"] == sum(N * k * (c + 4) * 4 for k, c in zip(ks, c8))


@pytest.mark.parametrize("fmt", ["fp16", "split_fp16"])
def test_solve_per_format_reaches_tolerance(helm, fmt):
    n, b = 9, 3
    om = W.omega_for(n)
    c32 = W.velocity_random(n, b, seed=3).astype(np.float32)
    f = W.gaussian_sources(n, b, om, [(0.5, 0.5, 0.3), (0.3, 0.6, 0.5)]).astype(np.complex64)
    c = torch.from_numpy(c32).cuda()
    ft = torch.from_numpy(f).cuda()
    its, us = {}, {}
    for p in ("fp32", fmt):
        S = helm.Solver(c, om, n, b, 1, precision=p)
        u, it, rel, code = S.solve(ft, tol=1e-6)
        assert code == helm.HELM_OK and max(rel) <= 1e-6
        its[p], us[p] = it, u.cpu().numpy()
        S.close()
    A = assemble_full(c32.astype(np.float64), Grid(n, b, om)).tocsc()
    for r in range(f.shape[0]):
        ud = spla.spsolve(A, f[r].astype(np.complex128).ravel()).reshape(f[r].shape)
        assert _rel(us[fmt][r], ud) <= 1e-5
        assert its[fmt][r] <= its["fp32"][r] + 1


def test_precision_arguments(helm):
    n, b = 5, 2
    om, c32, f = _case(n, b, "lens", R=1)
    c = torch.from_numpy(c32).cuda()
    o = helm.helm_default_opts()
    o.precision = 7
    with pytest.raises(helm.HelmError) as e:
        helm.helm_setup(c.data_ptr(), om, n, b, 1, o, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == helm.HELM_EINVAL
    S32 = helm.Solver(c, om, n, b, 1, precision="fp32")
    S16 = helm.Solver(c, om, n, b, 1, precision="fp16")
    x = torch.from_numpy(f).cuda()
    z = [torch.empty_like(x), torch.empty_like(x)]
    with pytest.raises(helm.HelmError) as e:
        helm.helm_apply_batch([S32.handle, S16.handle], [x.data_ptr(), x.data_ptr()],
                              [z[0].data_ptr(), z[1].data_ptr()], [1, 1],
                              torch.cuda.current_stream().cuda_stream)
    assert e.value.code == helm.HELM_ENOTSUP
    S32.close()
    S16.close()


def test_slab_apply_and_noalloc_fp16(helm):
    """The single-slab launch (Algorithm 4 alone) and the no-allocation apply
    with FP16-stored factors: the slab against the oracle's inner sweep over
    FP16-rounded twisted factors, the no-allocation apply against the
    allocating one (same kernel instance, identical results)."""
    n, b, d = 9, 3, 1
    om, c32, f = _case(n, b, "random", R=2)
    S = helm.Solver(torch.from_numpy(c32).cuda(), om, n, b, d, precision="fp16")
    P = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d, factor_format="fp16")
    N = n + 2 * b
    rng = np.random.default_rng(2)
    for M in (0, 4):
        Lz = helm.helm_slab_layers(S.handle, M)
        gs = (rng.standard_normal((1, Lz, N, N)) + 1j * rng.standard_normal((1, Lz, N, N))).astype(np.complex64)
        v = S.apply_slab(M, torch.from_numpy(gs).cuda()).cpu().numpy()
        vo = P.inner_sweep(M, gs.astype(np.complex128))
        assert _rel(v, vo) <= 1e-4
    x = torch.from_numpy(f).cuda()
    z = S.apply(x)
    z2 = torch.empty_like(x)
    st = torch.cuda.current_stream().cuda_stream
    helm.helm_apply_precond_noalloc(S.handle, x.data_ptr(), z2.data_ptr(), x.shape[0], st)
    assert helm.helm_status(S.handle, st) == helm.HELM_OK
    assert torch.equal(z, z2)
    S.close()

"""Batching of uneven problems, concurrent solves, ring autotuning and CUDA-graph
capture of the preconditioner apply (the serving patterns of the library)."""
import numpy as np
import pytest

from paper_1502_07266_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

PROBLEMS = [  # (n, b, d, velocity, nrhs): uneven sizes, widths, layer counts
    (5, 2, 1, "lens", 2),
    (9, 3, 2, "random", 3),
    (7, 4, 1, "waveguide", 1),
]


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300 import helm as H
    return H


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module")
def batch(helm):
    st = torch.cuda.current_stream().cuda_stream
    hs, fs, cs = [], [], []
    for q, (n, b, d, kind, R) in enumerate(PROBLEMS):
        om = W.omega_for(n)
        c = {"lens": W.velocity_lens, "waveguide": W.velocity_waveguide,
             "random": lambda n, b: W.velocity_random(n, b, seed=4)}[kind](n, b)
        ct = torch.from_numpy(c.astype(np.float32)).cuda()
        cs.append(ct)
        hs.append(helm.helm_setup(ct.data_ptr(), om, n, b, d, None, st))
        fs.append(torch.from_numpy(W.random_rhs(R, n, b, seed=40 + q).astype(np.complex64)).cuda())
    yield hs, fs
    for h in hs:
        helm.helm_destroy(h)


def test_batched_apply_equals_separate_applies(helm, batch):
    hs, fs = batch
    st = torch.cuda.current_stream().cuda_stream
    zs = [torch.empty_like(f) for f in fs]
    helm.helm_apply_batch(hs, [f.data_ptr() for f in fs], [z.data_ptr() for z in zs],
                          [p[4] for p in PROBLEMS], st)
    for h, f, z in zip(hs, fs, zs):
        zr = torch.empty_like(f)
        helm.helm_apply_precond(h, f.data_ptr(), zr.data_ptr(), f.shape[0], st)
        helm.helm_status(h, st)
        assert _rel(z.cpu().numpy(), zr.cpu().numpy()) <= 1e-6


def test_batched_apply_matches_oracle_per_problem(helm, batch):
    """One batched launch over the uneven problems: each problem's result is
    the oracle's Algorithm 6 apply on that problem's own grid, velocity and d
    (complex FP32 against FP64, 1e-5 relative)."""
    from oracle.operator import Grid
    from oracle.sweep import SweepPreconditioner
    hs, fs = batch
    st = torch.cuda.current_stream().cuda_stream
    zs = [torch.empty_like(f) for f in fs]
    helm.helm_apply_batch(hs, [f.data_ptr() for f in fs], [z.data_ptr() for z in zs],
                          [p[4] for p in PROBLEMS], st)
    for h in hs:
        helm.helm_status(h, st)
    for q, ((n, b, d, kind, R), f, z) in enumerate(zip(PROBLEMS, fs, zs)):
        c = {"lens": W.velocity_lens, "waveguide": W.velocity_waveguide,
             "random": lambda n, b: W.velocity_random(n, b, seed=4)}[kind](n, b)
        P = SweepPreconditioner(c.astype(np.float32).astype(np.float64), Grid(n, b, W.omega_for(n)), d=d)
        zo = P.apply(f.cpu().numpy().astype(np.complex128))
        zg = z.cpu().numpy()
        for r in range(R):
            assert _rel(zg[r], zo[r]) <= 1e-5, (q, r, _rel(zg[r], zo[r]))


def test_concurrent_batch_solve_equals_separate_solves(helm, batch):
    hs, fs = batch
    st = torch.cuda.current_stream().cuda_stream
    us = [torch.empty_like(f) for f in fs]
    nr = [p[4] for p in PROBLEMS]
    code, its, rel = helm.helm_solve_batch(hs, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], nr,
                                           1e-6, st)
    assert code == helm.HELM_OK and max(rel) <= 1e-6 and len(its) == sum(nr)
    for h, f, u in zip(hs, fs, us):
        ur = torch.empty_like(f)
        code1, its1, rel1 = helm.helm_solve(h, f.data_ptr(), ur.data_ptr(), f.shape[0], 1e-6, st)
        assert code1 == helm.HELM_OK
        assert _rel(u.cpu().numpy(), ur.cpu().numpy()) <= 1e-6


def test_autotune_keeps_results(helm, batch):
    hs, fs = batch
    st = torch.cuda.current_stream().cuda_stream
    h, f = hs[1], fs[1]
    z0 = torch.empty_like(f)
    helm.helm_apply_precond(h, f.data_ptr(), z0.data_ptr(), f.shape[0], st)
    stages = helm.helm_autotune(h, f.shape[0], st)
    assert 2 <= stages <= 8
    z1 = torch.empty_like(f)
    helm.helm_apply_precond(h, f.data_ptr(), z1.data_ptr(), f.shape[0], st)
    helm.helm_status(h, st)
    assert _rel(z1.cpu().numpy(), z0.cpu().numpy()) <= 1e-6


def test_apply_captured_in_cuda_graph(helm, batch):
    """The apply launches no allocation once its work space exists, so it can be
    captured in a CUDA graph and replayed on new inputs."""
    hs, fs = batch
    h, f = hs[0], fs[0]
    R = f.shape[0]
    static_in = f.clone()
    static_out = torch.empty_like(f)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        helm.helm_apply_precond(h, static_in.data_ptr(), static_out.data_ptr(), R, s.cuda_stream)  # work space
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        helm.helm_apply_precond(h, static_in.data_ptr(), static_out.data_ptr(), R,
                                torch.cuda.current_stream().cuda_stream)
    new = (2.0 * f + 1.0).contiguous()
    static_in.copy_(new)
    g.replay()
    torch.cuda.synchronize()
    ref = torch.empty_like(f)
    st = torch.cuda.current_stream().cuda_stream
    helm.helm_apply_precond(h, new.data_ptr(), ref.data_ptr(), R, st)
    helm.helm_status(h, st)
    assert _rel(static_out.cpu().numpy(), ref.cpu().numpy()) <= 1e-6


def test_batch_handle_matches_separate_handles(helm, batch):
    """helm_setup_batch: one handle over the three problems, vectors back to back.
    Its apply (one launch), solve (concurrent) and matvec equal the separate
    handles' results; single-problem queries and calls are refused."""
    hs, fs = batch
    st = torch.cuda.current_stream().cuda_stream
    cs, probs = [], []
    for q, (n, b, d, kind, R) in enumerate(PROBLEMS):
        c = {"lens": W.velocity_lens, "waveguide": W.velocity_waveguide,
             "random": lambda n, b: W.velocity_random(n, b, seed=4)}[kind](n, b)
        cs.append(torch.from_numpy(c.astype(np.float32)).cuda())
        probs.append((cs[-1].data_ptr(), W.omega_for(n), n, b, d, R))
    hb = helm.helm_setup_batch(probs, None, st)
    try:
        total = sum(p[4] for p in PROBLEMS)
        fcat = torch.cat([f.reshape(-1) for f in fs])
        z = torch.empty_like(fcat)
        helm.helm_apply_precond(hb, fcat.data_ptr(), z.data_ptr(), total, st)
        assert helm.helm_status(hb, st) == helm.HELM_OK
        off = 0
        for h, f in zip(hs, fs):
            zr = torch.empty_like(f)
            helm.helm_apply_precond(h, f.data_ptr(), zr.data_ptr(), f.shape[0], st)
            helm.helm_status(h, st)
            assert torch.equal(z[off:off + f.numel()].reshape(f.shape), zr)
            off += f.numel()
        # matvec, c64 and c128
        y = torch.empty_like(fcat)
        helm.helm_matvec(hb, fcat.data_ptr(), y.data_ptr(), total, 0, st)
        f128 = fcat.to(torch.complex128)
        y128 = torch.empty_like(f128)
        helm.helm_matvec(hb, f128.data_ptr(), y128.data_ptr(), total, 1, st)
        off = 0
        for h, f in zip(hs, fs):
            yr = torch.empty_like(f)
            helm.helm_matvec(h, f.data_ptr(), yr.data_ptr(), f.shape[0], 0, st)
            assert torch.equal(y[off:off + f.numel()].reshape(f.shape), yr)
            fr = f.to(torch.complex128)
            yr128 = torch.empty_like(fr)
            helm.helm_matvec(h, fr.data_ptr(), yr128.data_ptr(), f.shape[0], 1, st)
            assert torch.equal(y128[off:off + f.numel()].reshape(f.shape), yr128)
            off += f.numel()
        # solve: every problem's right-hand sides reach the tolerance and agree
        u = torch.empty_like(fcat)
        code, its, rel = helm.helm_solve(hb, fcat.data_ptr(), u.data_ptr(), total, 1e-6, st)
        assert code == helm.HELM_OK and len(its) == total and max(rel) <= 1e-6
        off = 0
        for h, f in zip(hs, fs):
            ur = torch.empty_like(f)
            code1, _, _ = helm.helm_solve(h, f.data_ptr(), ur.data_ptr(), f.shape[0], 1e-6, st)
            assert code1 == helm.HELM_OK
            assert _rel(u[off:off + f.numel()].reshape(f.shape).cpu().numpy(), ur.cpu().numpy()) <= 1e-6
            off += f.numel()
        # sizes and refusals
        assert helm.helm_factor_bytes(hb) == sum(helm.helm_factor_bytes(h) for h in hs)
        assert helm.helm_grid_size(hb) == -1 and helm.helm_num_blocks(hb) == -1
        for call, code in [
            (lambda: helm.helm_apply_precond(hb, fcat.data_ptr(), z.data_ptr(), total - 1, st), helm.HELM_EINVAL),
            (lambda: helm.helm_apply_precond_noalloc(hb, fcat.data_ptr(), z.data_ptr(), total, st),
             helm.HELM_ENOTSUP),
            (lambda: helm.helm_apply_batch([hb], [fcat.data_ptr()], [z.data_ptr()], [total], st), helm.HELM_EINVAL),
        ]:
            with pytest.raises(helm.HelmError) as e:
                call()
            assert e.value.code == code
    finally:
        helm.helm_destroy(hb)


def test_batched_apply_fp16_equals_separate_applies(helm):
    """The batched launch with FP16-stored factors (its own kernel instance)
    gives the separate applies' results."""
    st = torch.cuda.current_stream().cuda_stream
    o = helm.helm_default_opts()
    o.precision = helm.HELM_FP16
    hs, fs, cs = [], [], []
    try:
        for q, (n, b, d, kind, R) in enumerate(PROBLEMS):
            c = {"lens": W.velocity_lens, "waveguide": W.velocity_waveguide,
                 "random": lambda n, b: W.velocity_random(n, b, seed=4)}[kind](n, b)
            cs.append(torch.from_numpy(c.astype(np.float32)).cuda())
            hs.append(helm.helm_setup(cs[-1].data_ptr(), W.omega_for(n), n, b, d, o, st))
            fs.append(torch.from_numpy(W.random_rhs(R, n, b, seed=60 + q).astype(np.complex64)).cuda())
        zs = [torch.empty_like(f) for f in fs]
        helm.helm_apply_batch(hs, [f.data_ptr() for f in fs], [z.data_ptr() for z in zs],
                              [p[4] for p in PROBLEMS], st)
        for h, f, z in zip(hs, fs, zs):
            zr = torch.empty_like(f)
            helm.helm_apply_precond(h, f.data_ptr(), zr.data_ptr(), f.shape[0], st)
            assert helm.helm_status(h, st) == helm.HELM_OK
            assert torch.equal(z, zr)
    finally:
        for h in hs:
            helm.helm_destroy(h)

"""The no-allocation preconditioner apply gives the allocating apply's result.

helm_apply_precond_noalloc serves callers that must not allocate device memory
during a call (captured streams, fixed memory budgets): its slab work space is
a fixed array compiled into the library instead of a cudaMalloc.  This file is
collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

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


def _dirty_scratch(helm, st):
    """Fill the shared scratch from another geometry (other N and window
    length) with large values, so that the calls below start from
    another call's leftovers."""
    n, b, d = 9, 2, 2
    om = W.omega_for(n)
    c = torch.from_numpy(W.velocity_random(n, b, seed=3).astype(np.float32)).cuda()
    f = torch.from_numpy((1e6 * W.random_rhs(4, n, b, seed=5)).astype(np.complex64)).cuda()
    h = helm.helm_setup(c.data_ptr(), om, n, b, d, None, st)
    try:
        z = torch.empty_like(f)
        helm.helm_apply_precond_noalloc(h, f.data_ptr(), z.data_ptr(), 4, st)
        helm.helm_status(h, st)
    finally:
        helm.helm_destroy(h)


def test_noalloc_apply_matches_allocating_apply_twice(helm):
    n, b, R = 7, 3, 3
    om = W.omega_for(n)
    c = torch.from_numpy(W.velocity_lens(n, b).astype(np.float32)).cuda()
    f = torch.from_numpy(W.random_rhs(R, n, b, seed=21).astype(np.complex64)).cuda()
    st = torch.cuda.current_stream().cuda_stream
    _dirty_scratch(helm, st)
    h = helm.helm_setup(c.data_ptr(), om, n, b, 1, None, st)
    try:
        z_ref = torch.empty_like(f)
        helm.helm_apply_precond(h, f.data_ptr(), z_ref.data_ptr(), R, st)
        ref = z_ref.cpu().numpy()
        for _ in range(2):                        # the shared scratch keeps the last call's contents
            z = torch.full_like(f, float("nan"))
            helm.helm_apply_precond_noalloc(h, f.data_ptr(), z.data_ptr(), R, st)
            helm.helm_status(h, st)
            out = z.cpu().numpy()
            for r in range(R):
                err = np.linalg.norm(out[r] - ref[r]) / np.linalg.norm(ref[r])
                assert err <= 1e-6, err
        # a request beyond the fixed scratch is refused before any launch
        N = n + 2 * b
        per_rhs = N * N * (b + 1) * 8
        too_many = helm.HELM_NOALLOC_SCRATCH_BYTES // per_rhs + 1
        big = torch.zeros((too_many, N, N, N), dtype=torch.complex64, device="cuda")
        with pytest.raises(helm.HelmError) as e:
            helm.helm_apply_precond_noalloc(h, big.data_ptr(), torch.empty_like(big).data_ptr(), too_many, st)
        assert e.value.code == helm.HELM_EINVAL
    finally:
        helm.helm_destroy(h)


def test_noalloc_apply_replays_from_a_cuda_graph(helm):
    """The allocation-free apply captured in a CUDA graph (after one call
    outside the capture) replays to the allocating apply's result, twice."""
    n, b, R = 6, 3, 2
    om = W.omega_for(n)
    c = torch.from_numpy(W.velocity_random(n, b, seed=8).astype(np.float32)).cuda()
    f = torch.from_numpy(W.random_rhs(R, n, b, seed=22).astype(np.complex64)).cuda()
    st = torch.cuda.current_stream().cuda_stream
    h = helm.helm_setup(c.data_ptr(), om, n, b, 1, None, st)
    try:
        z_ref = torch.empty_like(f)
        helm.helm_apply_precond(h, f.data_ptr(), z_ref.data_ptr(), R, st)
        ref = z_ref.cpu().numpy()
        z = torch.empty_like(f)
        helm.helm_apply_precond_noalloc(h, f.data_ptr(), z.data_ptr(), R, st)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            helm.helm_apply_precond_noalloc(h, f.data_ptr(), z.data_ptr(), R,
                                            torch.cuda.current_stream().cuda_stream)
        _dirty_scratch(helm, st)
        for _ in range(2):
            z.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            out = z.cpu().numpy()
            for r in range(R):
                assert np.linalg.norm(out[r] - ref[r]) / np.linalg.norm(ref[r]) <= 1e-6
        helm.helm_status(h, st)
    finally:
        helm.helm_destroy(h)


def test_noalloc_apply_dense_handle(helm):
    """A dense-form handle (split FP16 operators, tensor-core products): the
    allocation-free apply gives the allocating apply's result, twice."""
    n, b, R = 7, 3, 3
    om = W.omega_for(n)
    c = torch.from_numpy(W.velocity_lens(n, b).astype(np.float32)).cuda()
    f = torch.from_numpy(W.random_rhs(R, n, b, seed=23).astype(np.complex64)).cuda()
    st = torch.cuda.current_stream().cuda_stream
    _dirty_scratch(helm, st)
    o = helm.helm_default_opts()
    o.apply_form = helm.HELM_DENSE
    o.precision = helm.HELM_SPLIT_FP16
    h = helm.helm_setup(c.data_ptr(), om, n, b, 1, o, st)
    try:
        z_ref = torch.empty_like(f)
        helm.helm_apply_precond(h, f.data_ptr(), z_ref.data_ptr(), R, st)
        ref = z_ref.cpu().numpy()
        for _ in range(2):
            z = torch.full_like(f, float("nan"))
            helm.helm_apply_precond_noalloc(h, f.data_ptr(), z.data_ptr(), R, st)
            helm.helm_status(h, st)
            out = z.cpu().numpy()
            for r in range(R):
                assert np.linalg.norm(out[r] - ref[r]) / np.linalg.norm(ref[r]) <= 1e-6
    finally:
        helm.helm_destroy(h)

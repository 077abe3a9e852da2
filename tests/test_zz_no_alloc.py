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


def test_noalloc_apply_matches_allocating_apply_twice(helm):
    n, b, R = 7, 3, 3
    om = W.omega_for(n)
    c = torch.from_numpy(W.velocity_lens(n, b).astype(np.float32)).cuda()
    f = torch.from_numpy(W.random_rhs(R, n, b, seed=21).astype(np.complex64)).cuda()
    st = torch.cuda.current_stream().cuda_stream
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

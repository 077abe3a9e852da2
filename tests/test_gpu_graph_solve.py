"""GMRES iterations as CUDA graphs: each iteration of a cycle (apply, matvec,
CGS2, norms, Givens and the device-side convergence test) is captured once per
handle and right-hand-side count and replayed.  A second solve on the same
handle replays the cached graphs and gives the first solve's result bit for
bit; a solve with another right-hand-side count recaptures; timing statistics
and launch counts still cover every iteration; the solution is the direct
solution of Eq. (system) within 1e-5."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.operator import Grid, assemble_full
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


@pytest.mark.parametrize("form,precision", [("chain", "fp32"), ("dense", "split_fp16")])
def test_replayed_solves_are_identical_and_correct(helm, form, precision):
    n, b, R = 9, 3, 3
    om = W.omega_for(n)
    c = W.velocity_random(n, b, seed=6).astype(np.float32)
    f = W.random_rhs(R, n, b, seed=61).astype(np.complex64)
    ft = torch.from_numpy(f).cuda()
    S = helm.Solver(torch.from_numpy(c).cuda(), om, n, b, 1, precision=precision, apply_form=form)
    try:
        helm.helm_enable_timing(S.handle, True)
        l0 = S.launches
        u1, its1, rel1, code1 = S.solve(ft, tol=1e-7)
        l1 = S.launches
        u2, its2, rel2, code2 = S.solve(ft, tol=1e-7)
        l2 = S.launches
        assert code1 == code2 == helm.HELM_OK
        assert torch.equal(u1, u2) and list(its1) == list(its2)
        assert l2 - l1 == l1 - l0 > 0                    # replays count their kernels
        st = helm.helm_get_stats(S.handle)
        total_its = 2 * max(its1)                        # one apply per iteration of the slowest RHS
        assert st.sweep_launches >= total_its and st.rhs_applied == R * st.sweep_launches
        assert st.sweep_ms > 0.0
        A = assemble_full(c.astype(np.float64), Grid(n, b, om)).tocsc()
        ug = u1.cpu().numpy()
        for r in range(R):
            ud = spla.spsolve(A, f[r].astype(np.complex128).ravel())
            assert np.linalg.norm(ug[r].ravel() - ud) / np.linalg.norm(ud) <= 1e-5
        # another right-hand-side count: the cache is rebuilt, results stay right
        u3, its3, rel3, code3 = S.solve(ft[:1].contiguous(), tol=1e-7)
        assert code3 == helm.HELM_OK
        ud = spla.spsolve(A, f[0].astype(np.complex128).ravel())
        assert np.linalg.norm(u3.cpu().numpy()[0].ravel() - ud) / np.linalg.norm(ud) <= 1e-5
    finally:
        S.close()

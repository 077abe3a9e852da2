"""Iterative refinement in FP64 around the reduced-precision solve.

Restarted GMRES forms the true residual r = f - A u in FP64 (FP64 stencil,
FP64 solution u) at the start of every cycle, and each cycle solves for the
correction with the preconditioner and the Arnoldi basis in complex FP32 / FP16:
restarts are refinement steps.  So the solve reaches FP64 residuals far below
what one FP32 or FP16 cycle can (a cycle's own accuracy is limited by its basis
rounding, about 1e-7): to 1e-10 here (the residual of the FP64 iterate the
solver keeps); the returned complex FP32 solution then equals the FP64 direct
solution of Eq. (system) up to its own rounding.
"""
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


@pytest.mark.parametrize("form,precision", [("dense", "split_fp16"), ("dense", "fp16"), ("chain", "fp16")])
def test_restarts_refine_below_the_working_precision(helm, form, precision):
    n, b, R = 9, 3, 2
    om = W.omega_for(n)
    c = W.velocity_lens(n, b).astype(np.float32)
    f = W.random_rhs(R, n, b, seed=81).astype(np.complex64)
    S = helm.Solver(torch.from_numpy(c).cuda(), om, n, b, 1, precision=precision, apply_form=form, restart=8)
    try:
        u, its, rel, code = S.solve(torch.from_numpy(f).cuda(), tol=1e-10)
        assert code == helm.HELM_OK and max(rel) <= 1e-10, (code, rel)
        assert max(its) > 8                               # more than one cycle: the restarts refined
        # the FP32 output of the FP64 solution is compared with the FP64 direct solution
        A = assemble_full(c.astype(np.float64), Grid(n, b, om)).tocsc()
        ug = u.cpu().numpy()
        for r in range(R):
            ud = spla.spsolve(A, f[r].astype(np.complex128).ravel())
            assert np.linalg.norm(ug[r].ravel() - ud) / np.linalg.norm(ud) <= 1e-6
    finally:
        S.close()

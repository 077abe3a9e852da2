"""The setup-level autotuner (helm_tune): it times setup + solve for each
candidate (d, apply form, precision, schedule, b_aux), records candidates that
cannot be set up,
and names the lowest score; the named configuration solves to the direct
solution of Eq. (system) (the oracle's sparse LU) within 1e-5."""
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


def test_tune_picks_the_fastest_passing_candidate(helm):
    n, b, R = 9, 3, 2
    om = W.omega_for(n)
    c = W.velocity_lens(n, b).astype(np.float32)
    f = W.random_rhs(R, n, b, seed=44).astype(np.complex64)
    ct, ft = torch.from_numpy(c).cuda(), torch.from_numpy(f).cuda()
    cands = [(1, "chain", "fp32"), (2, "chain", "fp32"), (3, "chain", "fp32"), (5, "chain", "fp32"),
             (6, "chain", "fp32"), (1, "dense", "split_fp16"), (2, "dense", "split_fp16"),
             (1, "dense", "split_fp16", "two_front", 2), (1, "chain", "fp32", "two_front", 2)]
    best, res = helm.helm_tune(ct.data_ptr(), om, n, b, ft.data_ptr(), R, cands, tol=1e-6,
                               stream=torch.cuda.current_stream().cuda_stream)
    assert res[4]["status"] == helm.HELM_ENOTSUP                 # d = 6: block (6+3)^2 > 64
    assert res[8]["status"] == helm.HELM_ENOTSUP                 # two fronts need the dense form
    assert (res[7]["schedule"], res[7]["b_aux"]) == (helm.HELM_TWO_FRONT, 2)
    ok = [q for q, r in enumerate(res) if r["status"] == helm.HELM_OK]
    assert len(ok) == 7
    assert best == min(ok, key=lambda q: res[q]["score"])
    for q in ok:
        r = res[q]
        assert r["setup_ms"] > 0 and r["solve_ms"] > 0 and r["relres_max"] <= 1e-6 and r["stored_bytes"] > 0
    # d changes the preconditioner: the iteration counts are not all equal
    assert len({res[q]["iters_max"] for q in ok if cands[q][1] == "chain"}) > 1
    d, form, prec = cands[best][:3]
    sched, b_aux = cands[best][3:] if len(cands[best]) > 3 else ("one_front", 0)
    S = helm.Solver(ct, om, n, b, d, b_aux=b_aux, precision=prec, apply_form=form, schedule=sched)
    try:
        u, its, rel, code = S.solve(ft, tol=1e-7)
        assert code == helm.HELM_OK
        A = assemble_full(c.astype(np.float64), Grid(n, b, om)).tocsc()
        ug = u.cpu().numpy()
        for r in range(R):
            ud = spla.spsolve(A, f[r].astype(np.complex128).ravel())
            assert np.linalg.norm(ug[r].ravel() - ud) / np.linalg.norm(ud) <= 1e-5
    finally:
        S.close()

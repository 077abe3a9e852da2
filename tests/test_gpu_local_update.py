"""Local factor update on the GPU (Section 6): after helm_update_velocity the
handle equals a fresh helm_setup with the new velocity, bit for bit (apply and
matvec), in the chain and dense forms; the update rebuilds only the problems
helm_affected_problems names; the apply matches the oracle's Algorithm 6 with
the new velocity (complex FP32 against FP64, 1e-5 relative)."""
import numpy as np
import pytest

from oracle.operator import Grid
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


@pytest.mark.parametrize("form,precision", [("chain", "fp32"), ("chain", "split_fp16"), ("dense", "fp32"),
                                            ("dense", "split_fp16")])
def test_update_equals_fresh_setup(helm, form, precision):
    n, b, d, R = 9, 4, 1, 3
    om = W.omega_for(n)
    N = n + 2 * b
    c0 = W.velocity_random(n, b, seed=12).astype(np.float32)
    box = (2, 11, 6, 9, 10, 13)                      # x0, x1, y0, y1, z0, z1
    c1 = c0.copy()
    c1[box[4]:box[5], box[2]:box[3], box[0]:box[1]] *= np.float32(1.2)
    f = torch.from_numpy(W.random_rhs(R, n, b, seed=31).astype(np.complex64)).cuda()
    kw = dict(precision=precision, apply_form=form)
    S = helm.Solver(torch.from_numpy(c0).cuda(), om, n, b, d, **kw)
    F = helm.Solver(torch.from_numpy(c1).cuda(), om, n, b, d, **kw)
    try:
        z_old = S.apply(f).clone()
        nprob = S.update_velocity(torch.from_numpy(c1).cuda(), box)
        r = helm.helm_affected_problems(n, b, d, box)
        B = helm.helm_num_blocks(S.handle)
        assert nprob == (r[1] - r[0] + 1) * (r[3] - r[2] + 1)
        assert 0 < nprob < B * B
        z_upd, z_new = S.apply(f), F.apply(f)
        y_upd, y_new = torch.empty_like(f), torch.empty_like(f)
        st = torch.cuda.current_stream().cuda_stream
        helm.helm_matvec(S.handle, f.data_ptr(), y_upd.data_ptr(), R, 0, st)
        helm.helm_matvec(F.handle, f.data_ptr(), y_new.data_ptr(), R, 0, st)
        assert S.status() == helm.HELM_OK
        assert torch.equal(z_upd, z_new)
        assert torch.equal(y_upd, y_new)
        assert not torch.equal(z_upd, z_old)
        if precision in ("fp32", "split_fp16"):
            zo = SweepPreconditioner(c1.astype(np.float64), Grid(n, b, om), d=d).apply(
                f.cpu().numpy().astype(np.complex128))
            zg = z_upd.cpu().numpy()
            for q in range(R):
                assert _rel(zg[q], zo[q]) <= 1e-5
    finally:
        S.close()
        F.close()


def test_update_two_front_equals_fresh_setup(helm):
    """The local update of a two-front dense handle equals its fresh setup bit
    for bit and matches the oracle's two-front apply (1e-5)."""
    n, b, d, b_aux, R = 9, 3, 1, 3, 2
    om = W.omega_for(n)
    c0 = W.velocity_random(n, b, seed=13).astype(np.float32)
    box = (1, 10, 9, 12, 2, 5)
    c1 = c0.copy()
    c1[box[4]:box[5], box[2]:box[3], box[0]:box[1]] *= np.float32(0.9)
    f = torch.from_numpy(W.random_rhs(R, n, b, seed=32).astype(np.complex64)).cuda()
    kw = dict(precision="split_fp16", apply_form="dense", schedule="two_front", b_aux=b_aux)
    S = helm.Solver(torch.from_numpy(c0).cuda(), om, n, b, d, **kw)
    F = helm.Solver(torch.from_numpy(c1).cuda(), om, n, b, d, **kw)
    try:
        nprob = S.update_velocity(torch.from_numpy(c1).cuda(), box)
        r = helm.helm_affected_problems(n, b, d, box, b_aux=b_aux, schedule=helm.HELM_TWO_FRONT)
        assert nprob == (r[1] - r[0] + 1) * (r[3] - r[2] + 1)
        z_upd, z_new = S.apply(f), F.apply(f)
        assert S.status() == helm.HELM_OK
        assert torch.equal(z_upd, z_new)
        zo = SweepPreconditioner(c1.astype(np.float64), Grid(n, b, om), d=d, b_aux=b_aux,
                                 schedule="two_front").apply(f.cpu().numpy().astype(np.complex128))
        zg = z_upd.cpu().numpy()
        for q in range(R):
            assert _rel(zg[q], zo[q]) <= 1e-5
    finally:
        S.close()
        F.close()


def test_update_rejects_bad_input(helm):
    n, b = 7, 3
    c0 = W.velocity_random(n, b, seed=2).astype(np.float32)
    S = helm.Solver(torch.from_numpy(c0).cuda(), W.omega_for(n), n, b, 1)
    try:
        bad = c0.copy()
        bad[5, 5, 5] = -1.0
        with pytest.raises(helm.HelmError) as e:
            S.update_velocity(torch.from_numpy(bad).cuda(), (5, 6, 5, 6, 5, 6))
        assert e.value.code == helm.HELM_EINVAL
        with pytest.raises(helm.HelmError):
            S.update_velocity(torch.from_numpy(c0).cuda(), (0, 14, 0, 1, 0, 1))
    finally:
        S.close()

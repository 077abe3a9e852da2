"""Two-front sweeps (Section 4.2's third modification, in both loops as in
Section 5) in the dense form, against the FP64 oracle's two-front schedule.

The oracle's two-front preconditioner is pinned on the CPU (exact limit,
reflection symmetry, GMRES convergence, tests/test_oracle.py).  Here:
  * the stored restricted operators of every role (lower front, upper front,
    centre, both boundary slabs' forward and backward maps) equal the oracle's
    R_out H~^{-1} R_in^T (FP32 and split FP16: 1e-5 of the largest entry);
  * the full two-front apply equals the oracle's (1e-5 relative per RHS);
  * GMRES with it reaches the direct solution (1e-5).
The centre window extends b_aux layers to both sides; the quasi-1D block of
the centre problem (2 b_aux + centre)^2 must stay <= 64, so b_aux <= 3.
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


def _entries(rect_in, rects_out, N):
    line0, nl, z0, nz = rect_in
    cols = []
    for j in range(nl * nz * N):
        x, r = divmod(j, nz * nl)
        cols.append((x, line0 + r // nz, z0 + r % nz))
    rows = []
    for (l0, nlr, zr0, nzr) in rects_out:
        for o in range(nlr * nzr * N):
            x, t = o % N, o // N
            rows.append((x, l0 + t // nzr, zr0 + t % nzr))
    return rows, cols


def _setup(helm, n, b, d, b_aux, precision, kind="random", seed=3):
    om = W.omega_for(n)
    c = {"random": lambda: W.velocity_random(n, b, seed=seed), "lens": lambda: W.velocity_lens(n, b)}[kind]()
    c32 = c.astype(np.float32)
    S = helm.Solver(torch.from_numpy(c32).cuda(), om, n, b, d, b_aux=b_aux, precision=precision,
                    apply_form="dense", schedule="two_front")
    P = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d, b_aux=b_aux, schedule="two_front")
    return S, P, om, c32


@pytest.mark.parametrize("n,b,d,b_aux", [(7, 3, 1, 3), (9, 4, 2, 2), (8, 2, 3, 1)])
@pytest.mark.parametrize("precision", ["fp32", "split_fp16"])
def test_two_front_operators_match_oracle(helm, n, b, d, b_aux, precision):
    S, P, _, _ = _setup(helm, n, b, d, b_aux, precision)
    try:
        B, c = P.B, P.centre
        cases = [(1, 1, 0), (1, c, 0), (c, c, 0), (c, B - 2, 0), (B - 1, B - 1, 0), (0, 0, 0), (0, 0, 1),
                 (c, 0, 1), (2, B - 1, 0), (2, B - 1, 1), (B - 1, B - 1, 1), (B - 2, c - 1, 0)]
        for M, Mp, dr in cases:
            Gt, rin, rout = S.dense_operator(M, Mp, dr)
            G = Gt.cpu().numpy().astype(np.complex128)
            rows, cols = _entries(rin, rout, S.N)
            Go = P.restricted_operator(M, Mp, rows, cols)
            assert G.shape == Go.shape
            assert np.abs(G - Go).max() <= 1e-5 * np.abs(Go).max(), (M, Mp, dr)
    finally:
        S.close()


@pytest.mark.parametrize("n,b,d,b_aux,kind", [(7, 3, 1, 3, "random"), (9, 4, 2, 2, "lens"), (8, 2, 3, 1, "random"),
                                              (11, 3, 1, 3, "lens"), (13, 6, 1, 2, "random")])
@pytest.mark.parametrize("precision", ["fp32", "split_fp16"])
def test_two_front_apply_matches_oracle(helm, n, b, d, b_aux, kind, precision):
    S, P, om, c32 = _setup(helm, n, b, d, b_aux, precision, kind=kind)
    try:
        f = W.random_rhs(3, n, b, seed=70).astype(np.complex64)
        z = S.apply(torch.from_numpy(f).cuda()).cpu().numpy()
        assert S.status() == helm.HELM_OK
        zo = P.apply(f.astype(np.complex128))
        for r in range(3):
            assert _rel(z[r], zo[r]) <= 1e-5, (r, _rel(z[r], zo[r]))
        # not the one-front preconditioner
        z1 = SweepPreconditioner(c32.astype(np.float64), Grid(n, b, om), d=d, b_aux=b_aux).apply(
            f[:1].astype(np.complex128))
        assert _rel(z1[0], zo[0]) > 1e-4
    finally:
        S.close()


def test_two_front_solve_matches_direct(helm):
    n, b, d, b_aux = 11, 4, 1, 3
    S, P, om, c32 = _setup(helm, n, b, d, b_aux, "split_fp16", kind="lens")
    try:
        f = W.random_rhs(2, n, b, seed=71).astype(np.complex64)
        u, its, rel, code = S.solve(torch.from_numpy(f).cuda(), tol=1e-7)
        assert code == helm.HELM_OK
        A = assemble_full(c32.astype(np.float64), Grid(n, b, om)).tocsc()
        ug = u.cpu().numpy()
        for r in range(2):
            ud = spla.spsolve(A, f[r].astype(np.complex128).ravel())
            assert _rel(ug[r].ravel(), ud) <= 1e-5
    finally:
        S.close()


def test_two_front_setup_rules(helm):
    """Two fronts run in the dense form only, need n - 1 >= 2d (one block of d
    per front), and a centre block that fits (b_aux <= 3 for d = 1)."""
    n, b = 7, 3
    c = torch.from_numpy(W.velocity_random(n, b, seed=1).astype(np.float32)).cuda()
    om = W.omega_for(n)
    with pytest.raises(helm.HelmError) as e:
        helm.Solver(c, om, n, b, 1, b_aux=3, apply_form="chain", schedule="two_front")
    assert e.value.code == helm.HELM_ENOTSUP
    with pytest.raises(helm.HelmError) as e:
        helm.Solver(c, om, n, b, 4, b_aux=1, apply_form="dense", schedule="two_front")
    assert e.value.code == helm.HELM_ENOTSUP
    b4 = 4                                              # b_aux = b = 4: a 9 x 9-layer centre problem
    c4 = torch.from_numpy(W.velocity_random(n, b4, seed=1).astype(np.float32)).cuda()
    with pytest.raises(helm.HelmError) as e:
        helm.Solver(c4, om, n, b4, 1, b_aux=0, apply_form="dense", schedule="two_front")
    assert e.value.code == helm.HELM_ENOTSUP

"""Adjoint solve and velocity gradient on the GPU vs the FP64 oracle.

The finite-difference pin of the gradient formula runs in the oracle (FP64
direct solves, tests/test_oracle.py); here the GPU adjoint fields and the
autograd gradient are compared with the oracle's adjoint gradient on the same
FP32-rounded inputs, and a directional derivative is checked at n = 63.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.adjoint import velocity_gradient
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


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def test_adjoint_solve_matches_transposed_direct_solve(helm):
    n, b, R = 7, 3, 2
    om = W.omega_for(n)
    c32 = W.velocity_random(n, b, seed=5).astype(np.float32)
    g = W.random_rhs(R, n, b, seed=31).astype(np.complex64)
    st = torch.cuda.current_stream().cuda_stream
    h = helm.helm_setup(torch.from_numpy(c32).cuda().data_ptr(), om, n, b, 1, None, st)
    try:
        gt = torch.from_numpy(g).cuda()
        lam = torch.empty_like(gt)
        code, its, rel = helm.helm_solve_adjoint(h, gt.data_ptr(), lam.data_ptr(), R, 1e-7, st)
        assert code == helm.HELM_OK
        AT = assemble_full(c32.astype(np.float64), Grid(n, b, om)).T.tocsc()
        lam = lam.cpu().numpy()
        for r in range(R):
            assert _rel(lam[r], spla.spsolve(AT, g[r].astype(np.complex128).ravel())) <= 1e-5
    finally:
        helm.helm_destroy(h)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_autograd_gradient_matches_oracle_adjoint_gradient(helm, precision):
    """The stored factor form changes only the preconditioner: the gradient
    meets the same tolerance against the oracle with FP16 factors."""
    from paper_1502_07266_gb300.autograd import helmholtz_solve
    n, b = 9, 3
    wl = W.lens_bump_16_sources(n=n, b=b)
    N = wl.N
    c32 = wl.c.astype(np.float32)
    f = wl.f.astype(np.complex64)
    g = Grid(n, b, wl.omega)
    rec = np.zeros((N, N, N), dtype=bool)
    rec[wl.meta["rec_plane"], b:b + n, b:b + n] = True
    from oracle.adjoint import solve_all
    d = solve_all(wl.meta["c_obs"].astype(np.float32).astype(np.float64), g, f.astype(np.complex128))[:, rec]
    L_o, grad_o = velocity_gradient(c32.astype(np.float64), g, f.astype(np.complex128), rec, d)
    c_t = torch.from_numpy(c32).cuda().requires_grad_(True)
    u = helmholtz_solve(c_t, torch.from_numpy(f).cuda(), wl.omega, n, b, 1, 1e-7, precision=precision)
    rec_t = torch.from_numpy(rec).cuda()
    d_t = torch.from_numpy(d.astype(np.complex64)).cuda()
    L = 0.5 * (u[:, rec_t] - d_t).abs().pow(2).sum()
    L.backward()
    assert abs(L.item() - L_o) <= 1e-4 * abs(L_o)
    grad = c_t.grad.double().cpu().numpy()
    assert _rel(grad, grad_o) <= 1e-3
    assert np.abs(grad - grad_o).max() <= 1e-3 * np.abs(grad_o).max()


@pytest.mark.slow
def test_gradient_directional_derivative_lens_bump_n63(helm):
    """n = 63 lens + bump, 16 sources, receivers on the z = 0.9 plane, data from
    the unperturbed lens: <dL/dc, dc> equals the central difference of L along
    a smooth direction dc (step 1e-3 in c, solves to 1e-7)."""
    from paper_1502_07266_gb300.autograd import helmholtz_solve
    wl = W.lens_bump_16_sources()
    n, b, N = wl.n, wl.b, wl.N
    rec = torch.zeros((N, N, N), dtype=torch.bool)
    rec[wl.meta["rec_plane"], b:b + n, b:b + n] = True
    rec = rec.cuda()
    f = torch.from_numpy(wl.f.astype(np.complex64)).cuda()
    c_obs = torch.from_numpy(wl.meta["c_obs"].astype(np.float32)).cuda()
    with torch.no_grad():
        d = helmholtz_solve(c_obs, f, wl.omega, n, b, 1, 1e-7)[:, rec]
    c0 = torch.from_numpy(wl.c.astype(np.float32)).cuda()

    def loss(c, grad=False):
        c = c.clone().requires_grad_(grad)
        u = helmholtz_solve(c, f, wl.omega, n, b, 1, 1e-7)
        L = 0.5 * (u[:, rec] - d).abs().pow(2).sum()
        if grad:
            L.backward()
            return L.item(), c.grad.double()
        return L.item(), None

    L0, grad = loss(c0, grad=True)
    x = torch.from_numpy(W.physical_coords(n, b)).cuda()
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    dc = torch.exp(-40 * ((X - 0.45) ** 2 + (Y - 0.55) ** 2 + (Z - 0.5) ** 2)).float()
    eps = 1e-3
    Lp, _ = loss(c0 + eps * dc)
    Lm, _ = loss(c0 - eps * dc)
    fd = (Lp - Lm) / (2 * eps)
    an = float((grad * dc.double()).sum())
    assert abs(fd - an) <= 2e-2 * abs(an), (fd, an)

"""torch.autograd.Function for u = A(c)^{-1} f (Eq. system) on the GPU.

forward: helm_setup on c, then helm_solve (GMRES with the recursive sweep).
backward: given grad_u (PyTorch's conjugate-Wirtinger gradient of a real loss,
so dL = Re(grad_u^H du)), the adjoint fields solve A^T lambda = conj(grad_u)
with the forward factors (helm_solve_adjoint, A^T = D^{-1} A D), and the fused
kernel helm_velocity_gradient forms dL/dc = Re(sum_r lambda_r u_r) 2 omega^2/c^3.
The gradient with respect to f is conj(lambda).  All arithmetic runs in libhelm.
"""
from __future__ import annotations

import torch

from . import helm


class _Handle:
    """Owns a helm handle for the lifetime of one autograd graph node."""

    def __init__(self, h: int):
        self.h = h

    def close(self):
        if self.h:
            helm.helm_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HelmholtzSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, f, omega: float, n: int, b: int, d: int = 1, tol: float = 1e-6,
                precision: str = "fp32", b_aux: int = 0):
        if c.dtype != torch.float32 or not c.is_cuda or f.dtype != torch.complex64 or not f.is_cuda:
            raise ValueError("c must be float32 and f complex64 CUDA tensors")
        c = c.contiguous()
        f = f.resolve_conj().contiguous()
        N = n + 2 * b
        R = f.numel() // N ** 3
        st = torch.cuda.current_stream().cuda_stream
        opts = helm.helm_default_opts()
        if precision not in helm.PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(helm.PRECISIONS)}")
        opts.precision = helm.PRECISIONS[precision]
        opts.b_aux = b_aux
        hd = _Handle(helm.helm_setup(c.data_ptr(), omega, n, b, d, opts, st))
        u = torch.empty_like(f)
        code, its, rel = helm.helm_solve(hd.h, f.data_ptr(), u.data_ptr(), R, tol, st)
        ctx.hd, ctx.R, ctx.tol, ctx.N = hd, R, tol, N
        ctx.iters, ctx.relres = its, rel
        ctx.save_for_backward(c, u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        c, u = ctx.saved_tensors
        st = torch.cuda.current_stream().cuda_stream
        # conj() is a lazy view in PyTorch: materialise it before passing a raw pointer
        g = grad_u.conj().resolve_conj().to(torch.complex64).contiguous()
        lam = torch.empty_like(g)
        helm.helm_solve_adjoint(ctx.hd.h, g.data_ptr(), lam.data_ptr(), ctx.R, ctx.tol, st)
        grad_c = None
        if ctx.needs_input_grad[0]:
            grad = torch.empty(c.shape, dtype=torch.float64, device=c.device)
            helm.helm_velocity_gradient(ctx.hd.h, lam.data_ptr(), u.data_ptr(), ctx.R, grad.data_ptr(), st)
            grad_c = grad.to(c.dtype)
        grad_f = lam.conj() if ctx.needs_input_grad[1] else None
        ctx.hd.close()
        return grad_c, grad_f, None, None, None, None, None, None, None


def helmholtz_solve(c, f, omega: float, n: int, b: int, d: int = 1, tol: float = 1e-6,
                    precision: str = "fp32", b_aux: int = 0):
    """u = A(c)^{-1} f, differentiable in c (and f).  precision selects the stored
    factor form ("fp32", "fp16", "split_fp16"); b_aux the auxiliary PML width
    (0 = b).  Both change only the preconditioner: u and the gradient are set by
    the GMRES tolerance on the FP64 residual."""
    return HelmholtzSolve.apply(c, f, omega, n, b, d, tol, precision, b_aux)

"""Differentiable solve x = A(chi)^{-1} b on the GPU factors.

`solve(h2, chi, b)` returns x and records a torch.autograd node whose backward
reuses the factorization of `h2` for the adjoint solve mu = A^{-H} g (the
conjugate-transposed traversal of the same factors) and maps x and mu to the
per-cell derivative with h2_grad_chi:

    dL/dchi_i = Re( x_i conj(mu_i - g_i) ) / chi_i,      dL/db = mu,

with g the incoming gradient of x (PyTorch's conjugate-Wirtinger convention,
dL = Re sum conj(g) dx).  A = I + s K D_chi is the matrix of the context.  If
chi differs from the context's contrast (e.g. after an optimisation step),
the context is moved to the new chi with h2_set_chi (exact update of the H^2
form) and refactorized with the settings of its last factorization before
the solve.  Everything runs in libh2; this module marshals arguments.
"""
import numpy as np
import torch


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, chi, b, h2, refine, tol, max_iter):
        x = h2.solve(b, refine=refine, tol=tol, max_iter=max_iter)
        ctx.h2, ctx.refine, ctx.tol, ctx.max_iter = h2, refine, tol, max_iter
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        h2 = ctx.h2
        gx = gx.to(torch.complex128).contiguous()
        mu = h2.solve(gx, adjoint=True, refine=ctx.refine, tol=ctx.tol, max_iter=ctx.max_iter)
        gchi = h2.grad_chi(x, mu, gx) if ctx.needs_input_grad[0] else None
        gb = mu if ctx.needs_input_grad[1] else None
        return gchi, gb, None, None, None, None


def solve(h2, chi, b, refine=True, tol=1e-10, max_iter=30, eps_fill=None, precision=None):
    """x = A(chi)^{-1} b, differentiable in chi (float64, shape (N,)) and b.

    b: CUDA complex128 (N,) or (N, nrhs).  With refine=True both the forward
    and the adjoint solve are refined against the FP64 H^2 matvec to `tol`.
    A chi other than the context's triggers h2_set_chi + h2_factorize
    (eps_fill / precision default to those of the context's last
    factorization)."""
    if h2.chi is None:
        raise ValueError("the context carries no contrast (built without chi / loaded without dscale)")
    if chi.shape != (h2.N,):
        raise ValueError("chi must have shape (N,)")
    got = chi.detach().to("cpu", torch.float64).numpy()
    if not np.array_equal(got, np.asarray(h2.chi)):
        last = getattr(h2, "last_factorize", None)
        e = eps_fill if eps_fill is not None else (last[0] if last else None)
        p = precision if precision is not None else (last[1] if last else None)
        if e is None or p is None:
            raise ValueError("new chi: give eps_fill and precision (the context has no earlier factorization)")
        h2.set_chi(got)
        h2.factorize(e, p)
    return _Solve.apply(chi, b, h2, refine, tol, max_iter)

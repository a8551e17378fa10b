"""torch.autograd.Functions for x = D_DW^-1 b: on U(1) link angles theta
(DwfSolve), and on the links themselves for any group (DwfSolveLinks: 2-d
U(1) or 4-d SU(3); the gradient with respect to U follows PyTorch's complex
convention dL/dRe U + i dL/dIm U, so a parametrisation such as
U = exp(i omega) U_0 written in torch chains through it).

Forward: links U = exp(i theta) and the solve run in libdwfmg (FP64 CGNR, or
the multigrid K-cycle when a handle is given).  A multigrid handle solves with
the operator it was set up for, so it must come from mg_setup on exactly
exp(i theta), M5 and mf: the forward pass checks that (mg_check_operator) and
raises DwfError otherwise, e.g. once theta has moved in a training step.  Backward: one adjoint solve
lambda = D_DW^-dag g, done as Gamma_5 D_DW^-1 Gamma_5 g (Gamma_5 = gamma_5 R,
Sec. 2.1), then dL/db = lambda and dL/dtheta = -Re(lambda^dag dD_DW/dtheta x)
from the link-force kernel.  Only x is kept between forward and backward (the
solve iterates are not stored; the adjoint solve recomputes what it needs).
"""
from __future__ import annotations

import torch

from . import _lib


def _solve(geom, U, b, M5, mf, tol, maxiter, mg):
    x = torch.empty_like(b)
    if mg is not None:
        st, _ = _lib.mg_solve(mg, b.contiguous(), x, tol=tol, maxiter=maxiter)
    else:
        st, _ = _lib.cgne_solve(geom, U, b.contiguous(), x, M5, mf, tol=tol, maxiter=maxiter)
    return x, st


class DwfSolve(torch.autograd.Function):
    """x = D_DW(exp(i theta))^-1 b.  Inputs: theta (float64 [nd*V]), b (complex128)."""

    @staticmethod
    def forward(ctx, theta, b, geom, M5, mf, tol=1e-12, maxiter=200000, mg=None):
        U = _lib.links_from_angles(geom, theta.detach())
        if mg is not None:
            _lib.mg_check_operator(mg, U, M5, mf)
        x, st = _solve(geom, U, b.detach(), M5, mf, tol, maxiter, mg)
        ctx.save_for_backward(x)
        ctx.geom, ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg = geom, M5, mf, tol, maxiter, mg
        ctx.U = U
        ctx.stats = st
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        geom = ctx.geom
        g = gx.contiguous().to(torch.complex128)
        # lambda = D^-dag g = Gamma_5 D^-1 Gamma_5 g
        y, _ = _solve(geom, ctx.U, _lib.gamma5_reflect(geom, g), ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg)
        lam = _lib.gamma5_reflect(geom, y)
        F = _lib.link_force(geom, ctx.U, lam, x)
        return -F, lam, None, None, None, None, None, None


def solve(theta, b, geom, M5, mf, tol=1e-12, maxiter=200000, mg=None):
    """Differentiable x = D_DW^-1 b (see DwfSolve)."""
    return DwfSolve.apply(theta, b, geom, M5, mf, tol, maxiter, mg)


class DwfSolveLinks(torch.autograd.Function):
    """x = D_DW(U)^-1 b with U (complex128, canonical link layout) differentiable.

    Backward: lambda = D^-dag g by one adjoint solve (Gamma_5 D^-1 Gamma_5), then
    dL/db = lambda and dL/dU = -G with G the complex link gradient of
    Re(lambda^dag dD x) (dwf_link_grad: colour outer products of lambda and the
    spin-projected x along every link, summed over s).  With a multigrid handle
    the links must be those of its setup (checked)."""

    @staticmethod
    def forward(ctx, U, b, geom, M5, mf, tol=1e-12, maxiter=200000, mg=None):
        Ud = U.detach().contiguous()
        if mg is not None:
            _lib.mg_check_operator(mg, Ud, M5, mf)
        x, st = _solve(geom, Ud, b.detach(), M5, mf, tol, maxiter, mg)
        ctx.save_for_backward(x)
        ctx.geom, ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg = geom, M5, mf, tol, maxiter, mg
        ctx.U = Ud
        ctx.stats = st
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        geom = ctx.geom
        g = gx.contiguous().to(torch.complex128)
        y, _ = _solve(geom, ctx.U, _lib.gamma5_reflect(geom, g), ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg)
        lam = _lib.gamma5_reflect(geom, y)
        G = _lib.link_grad(geom, lam, x)
        return -G, lam, None, None, None, None, None, None


def solve_links(U, b, geom, M5, mf, tol=1e-12, maxiter=200000, mg=None):
    """Differentiable x = D_DW(U)^-1 b with respect to the links U and b (see DwfSolveLinks)."""
    return DwfSolveLinks.apply(U, b, geom, M5, mf, tol, maxiter, mg)

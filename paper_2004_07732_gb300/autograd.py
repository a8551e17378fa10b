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
from the link-force kernel.  The solve iterates are never stored: backward
needs only x, and the adjoint solve recomputes what it needs.  Where device
memory is short (many solves alive in one graph, large lattices), `checkpoint`
chooses how x is kept between forward and backward:
  "device"    (default) x stays on the GPU;
  "host"      x is copied to pinned host memory and brought back in backward,
              so its device memory is free between the two passes;
  "recompute" nothing is kept: backward solves for x again from the saved
              inputs (one extra solve; the solvers are deterministic, so the
              gradient is the same to the bit).
"""
from __future__ import annotations

import torch

from . import _lib


CHECKPOINT_MODES = ("device", "host", "recompute")


def _keep_x(ctx, x, checkpoint):
    """Store x in ctx as `checkpoint` asks (see the module docstring)."""
    if checkpoint not in CHECKPOINT_MODES:
        raise ValueError(f"checkpoint must be one of {CHECKPOINT_MODES}")
    ctx.checkpoint = checkpoint
    ctx.x_host = None
    if checkpoint == "device":
        ctx.save_for_backward(x)
    elif checkpoint == "host":
        xh = torch.empty(x.shape, dtype=x.dtype, device="cpu", pin_memory=True)
        xh.copy_(x)                                  # synchronous: x may be freed once forward returns
        ctx.x_host = xh


def _restore_x(ctx, recompute):
    """x for backward: from the device, from the host copy, or solved again (recompute())."""
    if ctx.checkpoint == "device":
        (x,) = ctx.saved_tensors
        return x
    if ctx.checkpoint == "host":
        return ctx.x_host.to(ctx.device, non_blocking=True)
    return recompute()


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
    def forward(ctx, theta, b, geom, M5, mf, tol=1e-12, maxiter=200000, mg=None, checkpoint="device"):
        U = _lib.links_from_angles(geom, theta.detach())
        if mg is not None:
            _lib.mg_check_operator(mg, U, M5, mf)
        x, st = _solve(geom, U, b.detach(), M5, mf, tol, maxiter, mg)
        _keep_x(ctx, x, checkpoint)
        ctx.geom, ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg = geom, M5, mf, tol, maxiter, mg
        ctx.device = x.device
        # the links are rebuilt from theta in backward unless x stays on the device
        ctx.U = U if checkpoint == "device" else None
        ctx.theta = theta.detach()
        ctx.b = b.detach() if checkpoint == "recompute" else None
        ctx.stats = st
        return x

    @staticmethod
    def backward(ctx, gx):
        geom = ctx.geom
        U = ctx.U if ctx.U is not None else _lib.links_from_angles(geom, ctx.theta)
        x = _restore_x(ctx, lambda: _solve(geom, U, ctx.b, ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg)[0])
        g = gx.contiguous().to(torch.complex128)
        # lambda = D^-dag g = Gamma_5 D^-1 Gamma_5 g
        y, _ = _solve(geom, U, _lib.gamma5_reflect(geom, g), ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg)
        lam = _lib.gamma5_reflect(geom, y)
        F = _lib.link_force(geom, U, lam, x)
        return -F, lam, None, None, None, None, None, None, None


def solve(theta, b, geom, M5, mf, tol=1e-12, maxiter=200000, mg=None, checkpoint="device"):
    """Differentiable x = D_DW^-1 b (see DwfSolve; checkpoint: how x is kept for backward)."""
    return DwfSolve.apply(theta, b, geom, M5, mf, tol, maxiter, mg, checkpoint)


class DwfSolveLinks(torch.autograd.Function):
    """x = D_DW(U)^-1 b with U (complex128, canonical link layout) differentiable.

    Backward: lambda = D^-dag g by one adjoint solve (Gamma_5 D^-1 Gamma_5), then
    dL/db = lambda and dL/dU = -G with G the complex link gradient of
    Re(lambda^dag dD x) (dwf_link_grad: colour outer products of lambda and the
    spin-projected x along every link, summed over s).  With a multigrid handle
    the links must be those of its setup (checked)."""

    @staticmethod
    def forward(ctx, U, b, geom, M5, mf, tol=1e-12, maxiter=200000, mg=None, checkpoint="device"):
        Ud = U.detach().contiguous()
        if mg is not None:
            _lib.mg_check_operator(mg, Ud, M5, mf)
        x, st = _solve(geom, Ud, b.detach(), M5, mf, tol, maxiter, mg)
        _keep_x(ctx, x, checkpoint)
        ctx.geom, ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg = geom, M5, mf, tol, maxiter, mg
        ctx.device = x.device
        ctx.U = Ud
        ctx.b = b.detach() if checkpoint == "recompute" else None
        ctx.stats = st
        return x

    @staticmethod
    def backward(ctx, gx):
        geom = ctx.geom
        x = _restore_x(ctx, lambda: _solve(geom, ctx.U, ctx.b, ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg)[0])
        g = gx.contiguous().to(torch.complex128)
        y, _ = _solve(geom, ctx.U, _lib.gamma5_reflect(geom, g), ctx.M5, ctx.mf, ctx.tol, ctx.maxiter, ctx.mg)
        lam = _lib.gamma5_reflect(geom, y)
        G = _lib.link_grad(geom, lam, x)
        return -G, lam, None, None, None, None, None, None, None


def solve_links(U, b, geom, M5, mf, tol=1e-12, maxiter=200000, mg=None, checkpoint="device"):
    """Differentiable x = D_DW(U)^-1 b with respect to the links U and b (see DwfSolveLinks;
    checkpoint: how x is kept for backward)."""
    return DwfSolveLinks.apply(U, b, geom, M5, mf, tol, maxiter, mg, checkpoint)

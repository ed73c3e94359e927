"""torch.autograd wrappers: the assembly as two graph nodes (Map+Reduce
forward, hand-written adjoint backward) and a Dirichlet solve whose backward
is the adjoint solve of Eq. (adj).

* ``assemble(p, coords, kappa, layout, c)``  -> CSR values (differentiable in
  coords and kappa).
* ``load(p, coords, f, layout, ncomp)``      -> load vector (differentiable in
  coords and f).
* ``solve(p, vals, F, dirichlet, rtol)``     -> u with K_II u_I = F_I, u_D = 0;
  backward solves K lam' = grad_u (K symmetric) and returns
  dL/dvals = -lam' u^T on the pattern and dL/dF = lam'.
* ``solve_assembled(p, coords, kappa, layout, f, f_layout, dirichlet)`` -> u
  in one node whose backward calls the fused adjoint kernel (lam U^T enters the
  backward assembly directly; the nnz-sized gradient is never formed).
* ``residual(p, coords, kappa, layout, c, x, f, f_layout, dirichlet)`` -> the
  residual vector y = K x - F of Eq. (res1) without storing K (zero on
  Dirichlet rows); differentiable in x, kappa, f and coords.  Backward, with
  g the upstream gradient masked to the free rows: dL/dx = K g (the same
  matrix-free call; K is symmetric), dL/dkappa and dL/dcoords from the fused
  adjoint backward with lam = g, U = x, and dL/df from the load backward
  with grad_F = -g.  With ``reaction`` (the four coefficients of r(u)) y
  gains the semilinear term N(x), dL/dx gains J(x) g, and dL/dcoords the
  reaction's |det J| term (a per-point load of r(u_q), load backward).
"""
from __future__ import annotations

import torch

from . import binding as B


class _Assemble(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, kappa, p, layout, c):
        ctx.p, ctx.layout, ctx.c = p, layout, c
        ctx.save_for_backward(coords, kappa)
        return B.tg_assemble_bilinear(p, coords.contiguous(), kappa.contiguous(), layout, c)

    @staticmethod
    def backward(ctx, gvals):
        coords, kappa = ctx.saved_tensors
        gk, gx, _ = B.tg_assemble_backward(ctx.p, coords.contiguous(), kappa.contiguous(), ctx.layout, ctx.c,
                                           grad_vals=gvals.contiguous(), grad_kappa=ctx.needs_input_grad[1],
                                           grad_coords=ctx.needs_input_grad[0], grad_c=False)
        return gx, gk, None, None, None


class _Load(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, f, p, layout, ncomp):
        ctx.p, ctx.layout, ctx.ncomp = p, layout, ncomp
        ctx.save_for_backward(coords, f)
        return B.tg_assemble_load(p, coords.contiguous(), f.contiguous(), layout, ncomp)

    @staticmethod
    def backward(ctx, gF):
        coords, f = ctx.saved_tensors
        gf, gx = B.tg_assemble_load_backward(ctx.p, coords.contiguous(), f.contiguous(), ctx.layout, ctx.ncomp,
                                             gF.contiguous(), grad_f=ctx.needs_input_grad[1],
                                             grad_coords=ctx.needs_input_grad[0])
        return gx, gf, None, None, None


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, F, p, dirichlet, rtol, maxit):
        u, it, rel = B.tg_cg_solve(p, vals.contiguous(), F.contiguous(), dirichlet, rtol=rtol, maxit=maxit)
        ctx.p, ctx.dirichlet, ctx.rtol, ctx.maxit = p, dirichlet, rtol, maxit
        ctx.save_for_backward(vals, u)
        ctx.info = (it, rel)
        return u

    @staticmethod
    def backward(ctx, gu):
        vals, u = ctx.saved_tensors
        # K symmetric: K^T lam' = grad_u on the interior, lam'_D = 0
        lam, _, _ = B.tg_cg_solve(ctx.p, vals, gu.contiguous(), ctx.dirichlet, rtol=ctx.rtol, maxit=ctx.maxit)
        gvals = B.tg_csr_outer(ctx.p, lam, u, alpha=-1.0) if ctx.needs_input_grad[0] else None
        return gvals, (lam if ctx.needs_input_grad[1] else None), None, None, None, None


class _SolveAssembled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, kappa, f, p, layout, f_layout, dirichlet, rtol, maxit):
        coords, kappa, f = coords.contiguous(), kappa.contiguous(), f.contiguous()
        vals = B.tg_assemble_bilinear(p, coords, kappa, layout, 0.0)
        F = B.tg_assemble_load(p, coords, f, f_layout, 1)
        u, it, rel = B.tg_cg_solve(p, vals, F, dirichlet, rtol=rtol, maxit=maxit)
        ctx.p, ctx.layout, ctx.f_layout, ctx.dirichlet, ctx.rtol, ctx.maxit = p, layout, f_layout, dirichlet, rtol, maxit
        ctx.save_for_backward(coords, kappa, f, vals, u)
        ctx.info = (it, rel)
        return u

    @staticmethod
    def backward(ctx, gu):
        coords, kappa, f, vals, u = ctx.saved_tensors
        p = ctx.p
        lam, _, _ = B.tg_cg_solve(p, vals, gu.contiguous(), ctx.dirichlet, rtol=ctx.rtol, maxit=ctx.maxit)
        # Eq. (adj) with lam_adj = -lam: dGamma/dK = -lam u^T, dGamma/dF = lam
        neg = B.tg_scale_masked(lam, -1.0)
        gk, gx, _ = B.tg_assemble_backward(p, coords, kappa, ctx.layout, 0.0, lam=neg, U=u,
                                           grad_kappa=ctx.needs_input_grad[1], grad_coords=True, grad_c=False)
        # accumulate adds into both outputs: grad_f starts from zero
        gf0 = torch.zeros_like(f) if ctx.needs_input_grad[2] else False
        gf, _ = B.tg_assemble_load_backward(p, coords, f, ctx.f_layout, 1, lam, grad_f=gf0, grad_coords=gx,
                                            accumulate=True)
        return (gx if ctx.needs_input_grad[0] else None), gk, gf, None, None, None, None, None, None


class _Residual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, kappa, x, f, p, layout, c, f_layout, dirichlet, reaction):
        coords, kappa, x = coords.contiguous(), kappa.contiguous(), x.contiguous()
        f = f.contiguous() if f is not None else None
        if reaction is None:
            y, _ = B.tg_residual(p, coords, kappa, layout, c, x, f, f_layout, dirichlet, loss=False)
        else:
            y, _ = B.tg_semilinear_residual(p, coords, kappa, layout, c, x, reaction, f, f_layout,
                                            dirichlet=dirichlet, loss=False)
        ctx.p, ctx.layout, ctx.c, ctx.f_layout, ctx.dirichlet = p, layout, c, f_layout, dirichlet
        ctx.reaction = reaction
        ctx.has_f = f is not None
        ctx.save_for_backward(coords, kappa, x, f if f is not None else x)
        return y

    @staticmethod
    def backward(ctx, gy):
        coords, kappa, x, f = ctx.saved_tensors
        p = ctx.p
        # the upstream gradient restricted to the free rows (the Dirichlet
        # rows of y are zero whatever x is)
        g = B.tg_scale_masked(gy.contiguous(), 1.0, ctx.dirichlet)
        need_x, need_k, need_f = ctx.needs_input_grad[2], ctx.needs_input_grad[1], ctx.needs_input_grad[3]
        need_c = ctx.needs_input_grad[0]
        gx_in = None
        if need_x and ctx.reaction is None:
            gx_in = B.tg_residual(p, coords, kappa, ctx.layout, ctx.c, g, loss=False)[0]
        elif need_x:  # K g + J(x) g (K and the reaction's Jacobian are symmetric)
            gx_in = B.tg_semilinear_residual(p, coords, kappa, ctx.layout, ctx.c, g, ctx.reaction, x_react=x,
                                             loss=False)[0]
        gk = gc = None
        if need_k or need_c:
            gk, gc, _ = B.tg_assemble_backward(p, coords, kappa, ctx.layout, ctx.c, lam=g, U=x, grad_kappa=need_k,
                                               grad_coords=need_c, grad_c=False)
        gf = None
        if ctx.has_f and (need_f or need_c):
            # accumulate adds into both outputs: grad_f starts from zero
            gf, _ = B.tg_assemble_load_backward(p, coords, f, ctx.f_layout, 1, B.tg_scale_masked(g, -1.0),
                                                grad_f=torch.zeros_like(f) if need_f else False,
                                                grad_coords=gc if need_c else False, accumulate=True)
        if need_c and ctx.reaction is not None:
            # the reaction term's |det J| scaling: a per-point load of r(u_q) with upstream gradient +g
            rq = B.tg_reaction_points(p, x, ctx.reaction)
            B.tg_assemble_load_backward(p, coords, rq, B.PER_QP, 1, g, grad_f=False, grad_coords=gc, accumulate=True)
        return gc, gk, gx_in, gf, None, None, None, None, None, None


def assemble(p, coords, kappa, layout, c=0.0):
    return _Assemble.apply(coords, kappa, p, layout, float(c))


def load(p, coords, f, layout, ncomp=1):
    return _Load.apply(coords, f, p, layout, int(ncomp))


def solve(p, vals, F, dirichlet=None, rtol=1e-12, maxit=100000):
    return _Solve.apply(vals, F, p, dirichlet, float(rtol), int(maxit))


def solve_assembled(p, coords, kappa, layout, f, f_layout, dirichlet=None, rtol=1e-12, maxit=100000):
    return _SolveAssembled.apply(coords, kappa, f, p, layout, f_layout, dirichlet, float(rtol), int(maxit))


def residual(p, coords, kappa, layout, c, x, f=None, f_layout=B.PER_NODE, dirichlet=None, reaction=None):
    r = tuple(float(v) for v in reaction) if reaction is not None else None
    return _Residual.apply(coords, kappa, x, f, p, layout, float(c), f_layout, dirichlet, r)

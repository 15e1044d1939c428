"""torch.autograd.Function over the assembly: (kappa, x, y, z) -> (values, rhs).

Forward calls fea_assemble; backward calls fea_assemble_backward, the
hand-written adjoint kernel (dL/dkappa per element, dL/dx per node), which
recomputes the local matrices instead of storing them.  Scalar forms only
(P1/P2 kappa-diffusion with optional mass term), FP64.
"""
from __future__ import annotations

import torch

from . import fea


class FeaAssemble(torch.autograd.Function):
    """values, rhs = FeaAssemble.apply(kappa, x, y, z, mesh, form, npts, f_kind, f_param)

    kappa: [E] float64 CUDA tensor (per-element coefficient); x, y, z: [N]
    float64 CUDA node coordinates (the mesh is re-pointed at them); mesh: an
    fea.Mesh whose pattern of form.order is built or buildable."""

    @staticmethod
    def forward(ctx, kappa, x, y, z, mesh, form, npts=4, f_kind=fea.FEA_LOAD_SINPROD, f_param=(1.0,)):
        x, y, z, kappa = (t.contiguous() for t in (x, y, z, kappa))
        mesh.set_coords(x, y, z)
        coeffs = fea.make_coeffs(kappa=kappa, f_kind=f_kind, f_param=f_param)
        quad = fea.make_quadrature(npts, fea.FEA_FP64)
        values, rhs = mesh.assemble(form, coeffs, quad)
        ctx.save_for_backward(kappa, x, y, z)
        ctx.mesh, ctx.form, ctx.npts, ctx.f_kind, ctx.f_param = mesh, form, npts, f_kind, f_param
        return values, rhs

    @staticmethod
    def backward(ctx, grad_values, grad_rhs):
        kappa, x, y, z = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_coords(x, y, z)
        need_k = ctx.needs_input_grad[0]
        need_x = any(ctx.needs_input_grad[1:4])
        gk = torch.empty_like(kappa) if need_k else None
        gx = torch.empty((3, x.numel()), dtype=torch.float64, device=x.device) if need_x else None
        gv = None if grad_values is None else grad_values.contiguous()
        gf = None if grad_rhs is None else grad_rhs.contiguous()
        coeffs = fea.make_coeffs(kappa=kappa, f_kind=ctx.f_kind, f_param=ctx.f_param)
        quad = fea.make_quadrature(ctx.npts, fea.FEA_FP64)
        fea.fea_assemble_backward(mesh.h, ctx.form, coeffs, quad, gv, gf, gk, gx)
        gxs = (gx[0], gx[1], gx[2]) if need_x else (None, None, None)
        return (gk, *gxs, None, None, None, None, None)

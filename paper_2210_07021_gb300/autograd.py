"""torch.autograd integration of the sFMM (forward: sfmm_deflection; backward:
the adjoint sFMM, sfmm_adjoint).

    psi, alpha = deflection(src, q, tgt, plan)

is differentiable with respect to the masses q and the source positions src.
The gradient with respect to src is the covariant gradient on the sphere
(a tangent 3-vector at each source), which is what a step that moves the
sources along the sphere (and renormalises) needs.  Gradients with respect
to the target positions would need second derivatives of the potential and
are not formed; asking for them raises.  The backward pass runs in FP64 for
an FP64 plan and in double-float otherwise (see sfmm_adjoint).
"""
import torch

from . import sfmm


class _Deflection(torch.autograd.Function):
    @staticmethod
    def forward(ctx, src, q, tgt, plan):
        psi, alpha = plan.deflection(src, q, tgt)
        ctx.save_for_backward(src, q, tgt)
        ctx.plan = plan
        return psi, alpha

    @staticmethod
    def backward(ctx, g_psi, g_alpha):
        src, q, tgt = ctx.saved_tensors
        if ctx.needs_input_grad[2]:
            raise NotImplementedError("gradients with respect to the target positions are not formed")
        want_src, want_q = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_src or want_q):
            return None, None, None, None
        gp = None if g_psi is None else g_psi.contiguous().to(torch.float64)
        ga = None if g_alpha is None else g_alpha.contiguous().to(torch.float64)
        gq, gs = ctx.plan.adjoint(src.detach(), q.detach(), tgt.detach(), g_psi=gp, g_alpha=ga,
                                  want_q=want_q, want_src=want_src)
        if gq is not None:
            gq = gq.to(q.dtype)
        return gs, gq, None, None


def deflection(src, q, tgt, plan: "sfmm.Plan"):
    """(psi [M], alpha [M, 2]) of the plan, differentiable in q and src."""
    return _Deflection.apply(src, q, tgt, plan)

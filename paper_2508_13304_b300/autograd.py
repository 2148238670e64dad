"""torch.autograd wrappers of the projector pair.

``forward_project(mu, pose, projector)`` -> projections; its backward gives
  * d/dpose through the fused pose-gradient march in residual mode
    (proj_forward_pose_grad with the incoming gradient as dL/dl), i.e. the
    paper's analytic gradient (Eqs. final_forward, dis_forward), and
  * d/dmu through the exact transpose of the forward projector
    (proj_forward_adjoint).
``back_project(proj, pose, projector, weight)`` -> volume; its backward gives
  * d/dpose through the back-projection pose-gradient kernel
    (proj_back_pose_grad with the incoming gradient as dL/dmu; Eqs.
    final_back, dis_back), and
  * d/dproj through the exact transpose of the back-projector
    (proj_back_adjoint).

Memory: only the inputs are saved for backward; the prepared (mu, grad mu)
volume is rebuilt from mu in backward (one stencil pass), so no per-sample
or per-channel intermediate is ever stored.  The pose gradients are the
paper's analytic ones, not the exact derivative of the discrete projector;
their agreement is the subject of the tests (cosine similarity with finite
differences, as in the paper's Sec. III-A).
"""
from __future__ import annotations

import torch

from . import (PROJ_LOSS_RESIDUAL, PROJ_OP_ADJOINT, PROJ_OP_BACK, PROJ_OP_BACK_GRAD, PROJ_OP_FORWARD,
               PROJ_OP_FORWARD_GRAD, PROJ_W_NONE, Projector)

FORWARD_OPS = PROJ_OP_FORWARD | PROJ_OP_FORWARD_GRAD | PROJ_OP_ADJOINT
BACK_OPS = PROJ_OP_BACK | PROJ_OP_BACK_GRAD


class _ForwardProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, pose, projector):
        mu = mu.detach().float().contiguous()
        pose = pose.detach().float().contiguous()
        projector.set_volume(mu)
        out = projector.forward(pose)
        ctx.projector = projector
        ctx.save_for_backward(mu, pose)
        return out

    @staticmethod
    def backward(ctx, g):
        mu, pose = ctx.saved_tensors
        P = ctx.projector
        g = g.float().contiguous()
        g_mu = g_pose = None
        if ctx.needs_input_grad[0]:
            g_mu = P.forward_adjoint(g, pose)
        if ctx.needs_input_grad[1]:
            P.set_volume(mu)
            g_pose, _ = P.forward_pose_grad(pose, PROJ_LOSS_RESIDUAL, g)
        return g_mu, g_pose, None


class _BackProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, proj, pose, projector, weight):
        proj = proj.detach().float().contiguous()
        pose = pose.detach().float().contiguous()
        out = projector.back(proj, pose, weight)
        ctx.projector = projector
        ctx.weight = weight
        ctx.save_for_backward(proj, pose)
        return out

    @staticmethod
    def backward(ctx, g):
        proj, pose = ctx.saved_tensors
        P = ctx.projector
        g = g.float().contiguous()
        g_proj = g_pose = None
        if ctx.needs_input_grad[0]:
            g_proj = P.back_adjoint(g, pose, ctx.weight)
        if ctx.needs_input_grad[1]:
            g_pose = P.back_pose_grad(proj, pose, g, ctx.weight)
        return g_proj, g_pose, None, None


def forward_project(mu, pose, projector: Projector):
    """Projections [n_inst][nv][nu] of mu at the poses [n_pose][6]; the
    projector must support FORWARD_OPS."""
    return _ForwardProject.apply(mu, pose, projector)


def back_project(proj, pose, projector: Projector, weight=PROJ_W_NONE):
    """Voxel-driven back-projection of proj [n_inst][nv][nu]; the projector
    must support BACK_OPS."""
    return _BackProject.apply(proj, pose, projector, weight)


def ncc_loss(proj, target, inst_view, inst_pose, n_pose):
    """-mean over each pose's instances of the Pearson NCC of projection and
    target (torch ops, differentiable); returns [n_pose]."""
    a = proj.reshape(proj.shape[0], -1)
    b = target[torch.as_tensor(inst_view, device=proj.device, dtype=torch.long)].reshape(a.shape)
    da = a - a.mean(dim=1, keepdim=True)
    db = b - b.mean(dim=1, keepdim=True)
    ncc = (da * db).sum(1) / torch.sqrt((da * da).sum(1) * (db * db).sum(1))
    ip = torch.as_tensor(inst_pose, device=proj.device, dtype=torch.long)
    out = torch.zeros(n_pose, device=proj.device, dtype=proj.dtype).index_add_(0, ip, -ncc)
    cnt = torch.zeros(n_pose, device=proj.device, dtype=proj.dtype).index_add_(0, ip, torch.ones_like(ncc))
    return out / cnt

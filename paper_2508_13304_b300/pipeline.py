"""Streaming the fused pose gradient from host memory.

``PoseGradPipeline`` runs one ``set_volume`` + ``forward_pose_grad`` per
submitted step on inputs that live in (pinned) host memory and writes the
gradients and losses back to host memory.  The host-to-device copies of
step k+1 run on a copy stream while step k computes, into a second set of
device buffers, so a stream of steps costs about max(copy, compute) per step
instead of their sum.  Every step still copies its own inputs and results;
only the overlap differs from calling the projector step by step.
"""
from __future__ import annotations

import torch

from . import proj_forward_pose_grad, proj_set_volume


class PoseGradPipeline:
    def __init__(self, projector, loss, n_target_images):
        """projector: a Projector with PROJ_OP_FORWARD_GRAD; loss: PROJ_LOSS_*;
        n_target_images: images per reference (views for L2/NCC, instances for
        the residual mode)."""
        P = projector
        g = P.geom
        dev = P.device
        self.P, self.loss = P, loss
        self.compute = torch.cuda.current_stream(dev)
        self.copy = torch.cuda.Stream(dev)
        self.mu = [torch.empty((g.nz, g.ny, g.nx), device=dev) for _ in range(2)]
        self.ref = [torch.empty((n_target_images, g.nv, g.nu), device=dev) for _ in range(2)]
        self.pose = [torch.empty((P.plan.n_pose, 6), device=dev) for _ in range(2)]
        self.grad = [torch.empty((P.plan.n_pose, 6), device=dev) for _ in range(2)]
        self.lossv = [torch.empty((P.plan.n_pose,), device=dev) for _ in range(2)]
        self.copied = [torch.cuda.Event() for _ in range(2)]
        self.used = [torch.cuda.Event() for _ in range(2)]
        self.k = 0

    def submit(self, mu_h, ref_h, pose_h, grad_h, loss_h=None):
        """Queue one step: copy mu_h, ref_h, pose_h (host, pinned for overlap)
        in, compute, copy the gradient (and loss) out to grad_h / loss_h.
        Returns immediately; call synchronize() before reading the results."""
        b = self.k & 1
        self.copy.wait_event(self.used[b])       # the step that last used buffer b has computed
        with torch.cuda.stream(self.copy):
            self.mu[b].copy_(mu_h, non_blocking=True)
            self.ref[b].copy_(ref_h, non_blocking=True)
            self.pose[b].copy_(pose_h, non_blocking=True)
            self.copied[b].record(self.copy)
        self.compute.wait_event(self.copied[b])
        s = self.compute
        proj_set_volume(self.P.plan, self.mu[b], self.P.ws, stream=s)
        proj_forward_pose_grad(self.P.plan, self.pose[b], self.loss, self.ref[b], self.grad[b], self.lossv[b], None,
                               self.P.ws, stream=s)
        with torch.cuda.stream(self.compute):
            grad_h.copy_(self.grad[b], non_blocking=True)
            if loss_h is not None:
                loss_h.copy_(self.lossv[b], non_blocking=True)
        self.used[b].record(self.compute)
        self.k += 1

    def synchronize(self):
        self.compute.synchronize()

"""Gradient-based 2D/3D rigid registration with the fused NCC pose gradient
(the registration experiment of Sec. II-D.3: maximise the NCC of the
digitally reconstructed radiographs with the observed projections, Adam with
step 2 deg for rotations and 10 mm for translations, stop when the loss
changes by less than 1e-5 or the NCC exceeds 0.999).

Batched: every start pose (candidate) is a pose of one plan, all candidates
advance together, one fused launch per iteration; a converged candidate
keeps its pose (masked update).  Plain: the same loop with one candidate per
launch.  The bookkeeping of an iteration (hit test against a known truth,
stopping test, masked Adam step, refill of the slots of stopped starts) is
one launch (proj_registration_step); the Adam step counters live on the
device, so whole iterations
(pose-gradient launches, stopping test, Adam step) can be captured in a CUDA
graph and replayed (graph_steps > 0): the host then looks at the stopping
state once per replay instead of once per iteration.  The trajectories are
those of the eager loop: after every candidate has stopped, further captured
iterations leave all poses unchanged.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import (PROJ_LOSS_NCC, PROJ_OP_FORWARD_GRAD, Projector, proj_forward_pose_grad, proj_pose_adam,
               proj_registration_step, proj_set_volume, reg_params)


class Adam:
    """Adam on an [n, 6] pose tensor with per-parameter step sizes, one launch
    per step (proj_pose_adam)."""

    def __init__(self, n, lr, betas=(0.9, 0.999), eps=1e-8, device="cuda"):
        self.lr = [float(x) for x in np.broadcast_to(np.asarray(lr, dtype=np.float64), (6,))]
        self.b1, self.b2 = betas
        self.eps = eps
        self.m = torch.zeros((n, 6), device=device)
        self.v = torch.zeros((n, 6), device=device)
        # step count of each pose, on the device: a pose's bias correction counts only its own
        # updates, so a start that joins a running batch later follows its own trajectory
        self.t = torch.zeros(n, dtype=torch.float32, device=device)

    def step(self, pose, grad, active):
        """Update the rows of pose whose active flag is set (active: [n] bool, or None for all)."""
        proj_pose_adam(pose, grad, self.m, self.v, self.t, active, self.lr, self.b1, self.b2, self.eps)


def paper_step_sizes():
    return [10.0, 10.0, 10.0, math.radians(2.0), math.radians(2.0), math.radians(2.0)]


def register(geom, mu, target, init_poses, max_iter=200, lr=None, ncc_stop=0.999, dloss_stop=1e-5,
             batched=True, device="cuda", true_pose=None, tol=(0.5, 0.5), graph_steps=0, inst_view=None,
             wave=None, stop_at_hit=False):
    """Register every start pose in init_poses [n][6] to the target images
    ([n_views][nv][nu]).  By default every pose sees every view; with
    inst_view ([n] view indices) pose i sees only view inst_view[i], i.e. n
    independent single-view registrations advancing together (batched).
    Returns dict(poses, ncc, iters, seconds, and, when true_pose is given,
    first_hit_s: wall time at which any candidate was first seen within
    tol = (mm, deg) of it, or None; true_pose may be [6] or [n][6]).
    graph_steps > 0 replays CUDA graphs of that many iterations (checked
    once per replay).  wave=B runs at most B starts at a time (see
    register_waves); stop_at_hit ends the run at the first hit."""
    if wave is not None and inst_view is None:
        return register_waves(geom, mu, target, init_poses, wave, max_iter=max_iter, lr=lr, ncc_stop=ncc_stop,
                              dloss_stop=dloss_stop, device=device, true_pose=true_pose, tol=tol,
                              stop_at_hit=stop_at_hit)
    lr = paper_step_sizes() if lr is None else lr
    init = torch.as_tensor(np.asarray(init_poses, dtype=np.float32), device=device)
    n = init.shape[0]
    nv = geom.views.shape[0]
    mu_d = torch.as_tensor(np.asarray(mu, dtype=np.float32), device=device).contiguous()
    tgt = torch.as_tensor(np.asarray(target, dtype=np.float32), device=device).contiguous()
    groups = [list(range(n))] if (batched or inst_view is not None) else [[c] for c in range(n)]
    projs = []
    for grp in groups:
        k = len(grp)
        if inst_view is not None:
            P = Projector(geom, n_pose=k, inst_view=np.asarray(inst_view, dtype=np.int32),
                          inst_pose=np.arange(k, dtype=np.int32), ops=PROJ_OP_FORWARD_GRAD, device=device)
        else:
            P = Projector(geom, n_pose=k, inst_view=np.tile(np.arange(nv), k),
                          inst_pose=np.repeat(np.arange(k), nv), ops=PROJ_OP_FORWARD_GRAD, device=device)
        proj_set_volume(P.plan, mu_d, P.ws)
        projs.append(P)
    pose = init.clone()
    opt = Adam(n, lr, device=device)
    active = torch.ones(n, dtype=torch.bool, device=device)
    last = torch.full((n,), float("inf"), device=device)
    grad = torch.empty((n, 6), device=device)
    loss = torch.empty((n,), device=device)
    iters = torch.zeros(n, dtype=torch.int64, device=device)
    hit_any = torch.zeros((), dtype=torch.bool, device=device)
    views = [(pose[grp[0]:grp[-1] + 1], grad[grp[0]:grp[-1] + 1], loss[grp[0]:grp[-1] + 1]) for grp in groups]
    tp = None
    if true_pose is not None:
        tp = torch.as_tensor(np.asarray(true_pose, dtype=np.float32), device=device).reshape(-1, 6).contiguous()
    # every start in a slot of its own; a stopped start's slot just empties (no start waits)
    slots = torch.arange(n, dtype=torch.int32, device=device)
    nxt = torch.full((), n, dtype=torch.int64, device=device)
    listed = torch.zeros(n, dtype=torch.bool, device=device)
    params = reg_params(opt.lr, opt.b1, opt.b2, opt.eps, ncc_stop, dloss_stop, max_iter, tol)

    def iteration():
        for (pg, g_out, l_out), P in zip(views, projs):
            proj_forward_pose_grad(P.plan, pg, PROJ_LOSS_NCC, tgt, g_out, l_out, None, P.ws)
        # hit test, stopping test, masked Adam step, loss history: one launch
        proj_registration_step(pose, grad, loss, last, opt.m, opt.v, opt.t, active, iters, slots, nxt, tp,
                               hit_any if tp is not None else None, listed, params)

    first_hit = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it = 0
    graph = None
    while it < max_iter:
        k = 1
        if graph_steps > 0 and it > 0 and max_iter - it >= graph_steps:
            if graph is None:
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    for _ in range(graph_steps):
                        iteration()
            graph.replay()
            k = graph_steps
        else:
            iteration()
        it += k
        if true_pose is not None and first_hit is None and bool(hit_any):
            first_hit = time.perf_counter() - t0
            if stop_at_hit:
                break
        if not bool(active.any()):
            break
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    return dict(poses=pose.cpu().numpy(), ncc=(-loss).cpu().numpy(), iters=iters.cpu().numpy(), seconds=seconds,
                first_hit_s=first_hit)


def register_waves(geom, mu, target, init_poses, wave, max_iter=200, lr=None, ncc_stop=0.999, dloss_stop=1e-5,
                   device="cuda", true_pose=None, tol=(0.5, 0.5), stop_at_hit=False):
    """Multi-start registration with at most `wave` starts in flight: one plan
    holds every start as a pose, and each iteration marches only the poses in
    a device-resident slot list (proj_forward_pose_grad_list).  A start that
    stops (NCC above ncc_stop, loss change below dloss_stop, or max_iter
    updates) leaves its slot and the next start in order takes it, on the
    device, without a host round trip.  Each start follows exactly the
    trajectory it has when registered alone (its Adam state and step count are
    its own).  Returns the dict of register() plus `started` (starts begun)."""
    from . import proj_forward_pose_grad_list
    lr = paper_step_sizes() if lr is None else lr
    init = torch.as_tensor(np.asarray(init_poses, dtype=np.float32), device=device)
    n = init.shape[0]
    B = max(1, min(int(wave), n))
    nv = geom.views.shape[0]
    mu_d = torch.as_tensor(np.asarray(mu, dtype=np.float32), device=device).contiguous()
    tgt = torch.as_tensor(np.asarray(target, dtype=np.float32), device=device).contiguous()
    P = Projector(geom, n_pose=n, inst_view=np.tile(np.arange(nv), n), inst_pose=np.repeat(np.arange(n), nv),
                  ops=PROJ_OP_FORWARD_GRAD, device=device)
    proj_set_volume(P.plan, mu_d, P.ws)
    pose = init.clone()
    opt = Adam(n, lr, device=device)
    alive = torch.ones(n, dtype=torch.bool, device=device)     # not yet stopped
    last = torch.full((n,), float("inf"), device=device)
    grad = torch.zeros((n, 6), device=device)
    loss = torch.zeros((n,), device=device)
    iters = torch.zeros(n, dtype=torch.int64, device=device)
    slots = torch.arange(B, dtype=torch.int32, device=device)    # pose of each slot, -1 = empty
    nxt = torch.full((), B, dtype=torch.int64, device=device)    # next start to begin
    hit_any = torch.zeros((), dtype=torch.bool, device=device)
    listed = torch.zeros(n, dtype=torch.bool, device=device)
    tp = None
    if true_pose is not None:
        tp = torch.as_tensor(np.asarray(true_pose, dtype=np.float32), device=device).reshape(-1, 6).contiguous()
    params = reg_params(opt.lr, opt.b1, opt.b2, opt.eps, ncc_stop, dloss_stop, max_iter, tol)

    def iteration():
        proj_forward_pose_grad_list(P.plan, pose, slots, PROJ_LOSS_NCC, tgt, grad, loss, None, P.ws)
        # hit test, stopping test, masked Adam step, loss history and the refill of the slots of stopped
        # starts with the next starts in order: one launch
        proj_registration_step(pose, grad, loss, last, opt.m, opt.v, opt.t, alive, iters, slots, nxt, tp,
                               hit_any if tp is not None else None, listed, params)

    first_hit = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while True:
        iteration()
        if true_pose is not None and first_hit is None and bool(hit_any):
            first_hit = time.perf_counter() - t0
            if stop_at_hit:
                break
        if not bool((slots >= 0).any()):
            break
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    return dict(poses=pose.cpu().numpy(), ncc=(-loss).cpu().numpy(), iters=iters.cpu().numpy(), seconds=seconds,
                first_hit_s=first_hit, started=int(min(int(nxt.item()), n)))


def pose_error(a, b):
    """Translation error (mm, max abs) and rotation error (deg, max abs)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a[..., :3] - b[..., :3]).max(-1), np.degrees(np.abs(a[..., 3:] - b[..., 3:]).max(-1))

"""Motion-compensated FDK reconstruction (the motion-compensated analytical
reconstruction experiment of Sec. II-D.3): estimate one rigid pose per view
by minimising an image-sharpness loss of the FDK reconstruction, with Adam
and the back-projection pose gradient.

Per iteration: FDK back-projection of the filtered projections at the
current poses (proj_back, FDK weight), the sharpness S = -Var(|grad mu|) and
dS/dmu (proj_sharpness), the per-view pose gradient (proj_back_pose_grad
with the FDK weight derivative), and an Adam step on the [n_views, 6] poses.
The paper uses gradient entropy as the sharpness criterion; this build uses
the negative variance of the gradient magnitude.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import PROJ_OP_BACK, PROJ_OP_BACK_GRAD, PROJ_OP_SHARPNESS, PROJ_W_FDK, Projector
from .registration import Adam


def moco_fdk(geom, proj, n_iter=80, lr=(0.5, 0.5, 0.5, math.radians(0.5), math.radians(0.5), math.radians(0.5)),
             init=None, device="cuda"):
    """Returns dict(poses [n_views][6], sharpness history, seconds, fdk0 (the
    uncompensated reconstruction), fdk (the final one))."""
    n = geom.views.shape[0]
    P = Projector(geom, n_pose=n, inst_view=np.arange(n), inst_pose=np.arange(n),
                  ops=PROJ_OP_BACK | PROJ_OP_BACK_GRAD | PROJ_OP_SHARPNESS, device=device)
    q = P.fdk_filter(torch.as_tensor(np.asarray(proj, dtype=np.float32), device=device), math.pi / n)
    pose = torch.zeros((n, 6), device=device) if init is None else \
        torch.as_tensor(np.asarray(init, dtype=np.float32), device=device).clone()
    opt = Adam(n, lr, device=device)
    active = torch.ones(n, dtype=torch.bool, device=device)
    hist = []
    fdk0 = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(n_iter):
        vol = P.back(q, pose, PROJ_W_FDK)
        if fdk0 is None:
            fdk0 = vol.clone()
        loss, dvol = P.sharpness(vol)
        grad = P.back_pose_grad(q, pose, dvol, PROJ_W_FDK)
        hist.append(loss)
        opt.step(pose, grad, active)
    vol = P.back(q, pose, PROJ_W_FDK)
    loss = P.sharpness(vol, want_grad=False)
    hist.append(loss)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    return dict(poses=pose.cpu().numpy(), sharpness=torch.cat(hist).cpu().numpy(), seconds=seconds,
                fdk0=fdk0.cpu().numpy(), fdk=vol.cpu().numpy())

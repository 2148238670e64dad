"""Learned pose proposal: a small convolutional regressor from two DRR views
to the six rigid-pose parameters, trained on digitally reconstructed
radiographs rendered on the fly by the forward projector, and used to start
the gradient-based registration near the answer.

The paper leaves learned, coarse-to-fine pose initialisation to future work
(Sec. V); this module builds it on the library's tensor-core kernels
(include/posenet.h).  Architecture: n_conv layers of 3x3, stride-2,
padding-1 convolutions with ReLU (default 2 -> 32 -> 64 -> 128 -> 128 ->
128 -> 128 channels on a 128 x 128 input, ending at 2 x 2), then a fully
connected layer of 256 with ReLU and a linear output of 6 (normalised pose:
translations / t_range, rotations / r_range).  Loss: mean squared error.

Every forward and backward step runs in the library's kernels: implicit-
GEMM convolutions (the tensor-core kernel gathers the 3x3 patches itself;
bias and ReLU fused) forward for layers whose input has a multiple of 8
channels and at least 8192 output pixels, im2col + GEMM for the others; the
input gradients as implicit GEMMs too (the kernel gathers the output
gradient's rows per input pixel and tap; ReLU mask fused), or GEMM + col2im
with implicit=False; im2col, transposes + split-K GEMM for the weight
gradients; column sums for the bias gradients.  Parameters are FP32 masters in one flat
buffer, updated by Adam in one launch that also writes their BF16 copies
(pn_adam_step), then transposed for the GEMMs after every update.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import (PROJ_OP_FORWARD, Projector, pn_col2im_3x3s2, pn_colsum_bf16, pn_colsum_scratch_floats,
               pn_adam_step, pn_conv3x3s2_bf16, pn_conv3x3s2_dgrad_bf16, pn_conv_dgrad_weights, pn_gemm_bf16, pn_gemm_split_hint, pn_im2col_3x3s2, pn_mse_loss, pn_prepare_images,
               pn_to_bf16, pn_transpose_bf16, proj_forward)

BF = torch.bfloat16


def _r8(n):
    return (n + 7) // 8 * 8


class PoseNet:
    """The network with its parameters, BF16 copies and activation buffers
    for a fixed batch size.  forward() then backward() compute the loss
    gradients of one batch into .grads (FP32, same shapes as .params)."""

    def __init__(self, batch, in_hw=128, n_views=2, channels=(32, 64, 128, 128, 128, 128), hidden=256, n_out=6,
                 device="cuda", seed=0, implicit=True):
        self.B, self.hw, self.n_views, self.n_out = batch, in_hw, n_views, n_out
        self.implicit = implicit
        self.dev = torch.device(device)
        g = torch.Generator(device="cpu").manual_seed(seed)
        self.layers = []
        cin, hw = n_views, in_hw
        for cout in channels:
            kp = _r8(9 * cin)
            w = torch.zeros((cout, kp))
            w[:, :9 * cin] = torch.randn((cout, 9 * cin), generator=g) * math.sqrt(2.0 / (9 * cin))
            self.layers.append(dict(cin=cin, cout=cout, H=hw, kp=kp, Ho=(hw + 1) // 2, w=w.to(self.dev),
                                    b=torch.zeros(cout, device=self.dev)))
            hw, cin = (hw + 1) // 2, cout
        self.out_hw = hw
        self.flat = hw * hw * cin
        self.n_pad = _r8(n_out)
        w1 = torch.randn((hidden, self.flat), generator=g) * math.sqrt(2.0 / self.flat)
        w2 = torch.zeros((self.n_pad, hidden))
        w2[:n_out] = torch.randn((n_out, hidden), generator=g) * math.sqrt(1.0 / hidden)
        self.fc = [dict(w=w1.to(self.dev), b=torch.zeros(hidden, device=self.dev), n_in=self.flat, n=hidden),
                   dict(w=w2.to(self.dev), b=torch.zeros(self.n_pad, device=self.dev), n_in=hidden, n=self.n_pad)]
        self.hidden = hidden
        self._alloc()
        self.refresh()

    # ---------------------------------------------------------------- buffers
    def _flatten(self):
        """Master weights, their gradients and their BF16 copies as views of three
        flat buffers (each tensor at a multiple of 8 elements, so every view is
        16-byte aligned for the tensor maps), so that one launch updates them all
        (pn_adam_step) and one converts them (pn_to_bf16)."""
        d = self.dev
        ts = [P[k] for P in self.layers + self.fc for k in ("w", "b")]
        offs, n = [], 0
        for t in ts:
            offs.append(n)
            n += _r8(t.numel())
        self.flat_p = torch.zeros(n, device=d)
        self.flat_g = torch.zeros(n, device=d)
        self.flat_b16 = torch.zeros(n, device=d, dtype=BF)
        i = 0
        for P in self.layers + self.fc:
            for k in ("w", "b"):
                t, o = P[k], offs[i]
                i += 1
                view = self.flat_p[o:o + t.numel()].view(t.shape)
                view.copy_(t)
                P[k] = view
                P["g" + k] = self.flat_g[o:o + t.numel()].view(t.shape)
                if k == "w":
                    P["wb"] = self.flat_b16[o:o + t.numel()].view(t.shape)

    def _alloc(self):
        B, d = self.B, self.dev
        self._flatten()
        self.x = torch.zeros((B, self.hw, self.hw, self.n_views), device=d, dtype=BF)
        biggest_t, biggest_dcol, biggest_part = 0, 0, 0
        for L in self.layers:
            M = B * L["Ho"] * L["Ho"]
            L["M"], L["Mp"] = M, _r8(M)
            L["col"] = torch.empty((M, L["kp"]), device=d, dtype=BF)
            L["a"] = torch.empty((M, L["cout"]), device=d, dtype=BF)       # post-ReLU output, NHWC
            L["d"] = torch.empty((M, L["cout"]), device=d, dtype=BF)       # gradient w.r.t. pre-activation
            L["wbT"] = torch.empty((L["kp"], L["cout"]), device=d, dtype=BF)
            if L["kp"] == 9 * L["cin"] and L["cout"] % 8 == 0:  # weights of the implicit input gradient
                L["wd"] = torch.empty((L["cin"], 9 * L["cout"]), device=d, dtype=BF)
            L["split"] = pn_gemm_split_hint(L["cout"], L["kp"], L["Mp"])
            biggest_t = max(biggest_t, L["kp"] * L["Mp"], L["cout"] * L["Mp"])
            biggest_dcol = max(biggest_dcol, M * L["kp"])
            biggest_part = max(biggest_part, L["split"] * L["cout"] * L["kp"])
        Bp = _r8(B)
        self.Bp = Bp
        for F in self.fc:
            F["wbT"] = torch.empty((F["n_in"], F["n"]), device=d, dtype=BF)
            F["split"] = pn_gemm_split_hint(F["n"], F["n_in"], Bp)
            biggest_t = max(biggest_t, F["n"] * Bp, F["n_in"] * Bp)
            biggest_part = max(biggest_part, F["split"] * F["n"] * F["n_in"])
        self.h = torch.empty((B, self.hidden), device=d, dtype=BF)
        self.dh = torch.empty((B, self.hidden), device=d, dtype=BF)
        self.out = torch.empty((B, self.n_pad), device=d)
        self.dout = torch.empty((B, self.n_pad), device=d, dtype=BF)
        self.loss = torch.zeros(1, device=d)
        self.tA = torch.empty(biggest_t, device=d, dtype=BF)
        self.tB = torch.empty(biggest_t, device=d, dtype=BF)
        self.dcol = torch.empty(biggest_dcol, device=d)
        self.part = torch.empty(max(1, biggest_part), device=d)
        cs = max(pn_colsum_scratch_floats(L["M"], L["cout"]) for L in self.layers)
        cs = max(cs, pn_colsum_scratch_floats(B, self.hidden), pn_colsum_scratch_floats(B, self.n_pad))
        self.cs = torch.empty(cs, device=d)

    @property
    def params(self):
        return [t for L in self.layers for t in (L["w"], L["b"])] + [t for F in self.fc for t in (F["w"], F["b"])]

    @property
    def grads(self):
        return [t for L in self.layers for t in (L["gw"], L["gb"])] + [t for F in self.fc for t in (F["gw"], F["gb"])]

    def refresh(self, convert=True):
        """BF16 copies (and transposes) of the FP32 weights for the GEMMs;
        convert=False when pn_adam_step has written the BF16 copies already."""
        if convert:
            pn_to_bf16(self.flat_p, self.flat_b16)
        for P in self.layers + self.fc:
            rows, cols = P["wb"].shape
            pn_transpose_bf16(P["wb"], rows, cols, P["wbT"], rows)
            if "wd" in P:
                pn_conv_dgrad_weights(P["wb"], P["cout"], P["cin"], P["wd"])

    # ---------------------------------------------------------------- passes
    def forward(self, x=None):
        """Outputs [B][n_pad] FP32 (columns n_out.. are zero) for the input
        in self.x (or x, BF16 NHWC [B][hw][hw][n_views])."""
        if x is not None:
            self.x.copy_(x)
        B = self.B
        a, cin = self.x, self.n_views
        for L in self.layers:
            # implicit GEMM where its grid has at least 64 tiles of 128 output pixels: on the two smallest
            # layers of the default network (8 and 32 tiles) im2col + GEMM measured faster
            if self.implicit and cin % 8 == 0 and L["M"] >= 64 * 128:
                pn_conv3x3s2_bf16(a, B, L["H"], L["H"], cin, L["wb"], L["cout"], bias=L["b"], relu=True, y16=L["a"])
                L["col_ready"] = False
            else:
                pn_im2col_3x3s2(a, B, L["H"], L["H"], cin, L["kp"], L["col"])
                pn_gemm_bf16(L["M"], L["cout"], L["kp"], L["col"], L["kp"], L["wb"], L["kp"], bias=L["b"],
                             relu=True, D16=L["a"])
                L["col_ready"] = True
            a, cin = L["a"], L["cout"]
        F1, F2 = self.fc
        pn_gemm_bf16(B, F1["n"], F1["n_in"], a, F1["n_in"], F1["wb"], F1["n_in"], bias=F1["b"], relu=True,
                     D16=self.h)
        pn_gemm_bf16(B, F2["n"], F2["n_in"], self.h, F2["n_in"], F2["wb"], F2["n_in"], bias=F2["b"], D32=self.out)
        return self.out

    def loss_grad(self, target):
        """MSE of the first n_out outputs against target [B][n_out] (FP32);
        writes self.loss and the output gradient."""
        pn_mse_loss(self.out, self.B, self.n_out, self.n_pad, target, self.loss, self.dout, self.n_pad)
        return self.loss

    def _wgrad(self, dy, M, N_out, inp, K_in, gw, split):
        """gw [N_out][K_in] = dy^T . inp over M rows (dy [M][N_out], inp [M][K_in])."""
        Mp = _r8(M)
        dyT = self.tA[:N_out * Mp]
        inT = self.tB[:K_in * Mp]
        pn_transpose_bf16(dy, M, N_out, dyT, Mp)
        pn_transpose_bf16(inp, M, K_in, inT, Mp)
        pn_gemm_bf16(N_out, K_in, Mp, dyT, Mp, inT, Mp, D32=gw, split_k=split, part=self.part)

    def backward(self):
        """Gradients of the loss (after loss_grad) into .grads."""
        B = self.B
        F1, F2 = self.fc
        last = self.layers[-1]
        # output layer
        self._wgrad(self.dout, B, F2["n"], self.h, F2["n_in"], F2["gw"], F2["split"])
        pn_colsum_bf16(self.dout, B, F2["n"], F2["n"], F2["gb"], self.cs)
        pn_gemm_bf16(B, F2["n_in"], F2["n"], self.dout, F2["n"], F2["wbT"], F2["n"], mask=self.h, ldm=F2["n_in"],
                     D16=self.dh)
        # hidden layer
        self._wgrad(self.dh, B, F1["n"], last["a"], F1["n_in"], F1["gw"], F1["split"])
        pn_colsum_bf16(self.dh, B, F1["n"], F1["n"], F1["gb"], self.cs)
        pn_gemm_bf16(B, F1["n_in"], F1["n"], self.dh, F1["n"], F1["wbT"], F1["n"], mask=last["a"],
                     ldm=F1["n_in"], D16=last["d"])
        # convolutions, last to first
        for i in reversed(range(len(self.layers))):
            L = self.layers[i]
            if not L.get("col_ready", False):     # the implicit forward did not store the patches
                inp = self.x if i == 0 else self.layers[i - 1]["a"]
                pn_im2col_3x3s2(inp, B, L["H"], L["H"], L["cin"], L["kp"], L["col"])
                L["col_ready"] = True
            self._wgrad(L["d"], L["M"], L["cout"], L["col"], L["kp"], L["gw"], L["split"])
            pn_colsum_bf16(L["d"], L["M"], L["cout"], L["cout"], L["gb"], self.cs)
            if i > 0 and self.implicit and "wd" in L:
                P = self.layers[i - 1]
                pn_conv3x3s2_dgrad_bf16(L["d"], B, L["H"], L["H"], L["cin"], L["wd"], L["cout"], mask=P["a"],
                                        dx16=P["d"])
            elif i > 0:
                P = self.layers[i - 1]
                dcol = self.dcol[:L["M"] * L["kp"]]
                pn_gemm_bf16(L["M"], L["kp"], L["cout"], L["d"], L["cout"], L["wbT"], L["cout"], D32=dcol)
                pn_col2im_3x3s2(dcol, B, L["H"], L["H"], L["cin"], L["kp"], mask=P["a"], dx16=P["d"])

    # ---------------------------------------------------------------- oracle view
    def as_oracle_params(self):
        """The BF16-rounded weights in the layout of oracle.posenet (numpy FP64):
        conv [Co][3][3][Ci], fc [n][n_in] (output rows n_out.. dropped)."""
        conv = []
        for L in self.layers:
            w = L["w"].bfloat16().float().cpu().numpy().astype(np.float64)[:, :9 * L["cin"]]
            conv.append((w.reshape(L["cout"], 3, 3, L["cin"]), L["b"].cpu().numpy().astype(np.float64)))
        F1, F2 = self.fc
        fc = [(F1["w"].bfloat16().float().cpu().numpy().astype(np.float64), F1["b"].cpu().numpy().astype(np.float64)),
              (F2["w"].bfloat16().float().cpu().numpy().astype(np.float64)[:self.n_out],
               F2["b"].cpu().numpy().astype(np.float64)[:self.n_out])]
        return dict(conv=conv, fc=fc)


class AdamW:
    """Adam (bias-corrected, decoupled weight decay optional) on a network's
    flat FP32 master weights, one launch per step (pn_adam_step), which also
    writes the BF16 copies the GEMMs read."""

    def __init__(self, net, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, wd=0.0):
        self.net = net
        self.m = torch.zeros_like(net.flat_p)
        self.v = torch.zeros_like(net.flat_p)
        self.lr, self.b1, self.b2, self.eps, self.wd = lr, betas[0], betas[1], eps, wd
        self.t = 0

    def step(self, lr=None):
        """One update from the gradients in net.flat_g; then net.refresh(convert=False)."""
        self.t += 1
        lr = self.lr if lr is None else lr
        c1 = 1 - self.b1 ** self.t
        c2 = 1 - self.b2 ** self.t
        n = self.net
        pn_adam_step(n.flat_p, n.flat_g, self.m, self.v, lr * math.sqrt(c2) / c1, self.b1, self.b2, self.eps,
                     1 - lr * self.wd, n.flat_b16)


class DrrSource:
    """Batches of (network input, normalised pose) rendered on the fly:
    uniform random poses (translations within +-t_range mm, rotations within
    +-r_range deg), proj_forward of every view, then box downsampling and
    standardisation (pn_prepare_images)."""

    def __init__(self, geom, mu, batch, factor, t_range=40.0, r_range=30.0, device="cuda", seed=0):
        self.geom, self.B, self.factor = geom, batch, factor
        self.nvw = geom.views.shape[0]
        self.scale = torch.tensor([t_range] * 3 + [math.radians(r_range)] * 3, device=device)
        self.P = Projector(geom, n_pose=batch, inst_view=np.tile(np.arange(self.nvw), batch),
                           inst_pose=np.repeat(np.arange(batch), self.nvw), ops=PROJ_OP_FORWARD, device=device)
        self.P.set_volume(mu)
        self.proj = torch.empty((batch * self.nvw, geom.nv, geom.nu), device=device)
        self.gen = torch.Generator(device=device).manual_seed(seed)
        self.dev = device

    def render(self, pose, out):
        """Network input for the given poses [B][6] (FP32, physical units)."""
        proj_forward(self.P.plan, pose, self.proj, self.P.ws)
        pn_prepare_images(self.proj, self.B, self.nvw, self.geom.nu, self.geom.nv, self.factor, out)

    def batch(self, out, target):
        """Fill out (BF16 NHWC) and target ([B][6] normalised) with a fresh batch."""
        u = torch.rand((self.B, 6), device=self.dev, generator=self.gen) * 2 - 1
        target.copy_(u)
        self.render((u * self.scale).contiguous(), out)

    def images_for(self, proj_views, out):
        """Network input for given projections [n][n_views][nv][nu] (e.g. the
        target images of a registration)."""
        n = proj_views.shape[0]
        pn_prepare_images(proj_views.reshape(-1).contiguous(), n, self.nvw, self.geom.nu, self.geom.nv, self.factor,
                          out)


def train(net, source, n_samples, lr=1e-3, lr_final=1e-5, log_every=0, log=print):
    """Adam with cosine decay over n_samples DRRs; returns the loss history."""
    opt = AdamW(net, lr=lr)
    target = torch.empty((net.B, 6), device=net.dev)
    steps = max(1, n_samples // net.B)
    hist = []
    t0 = time.perf_counter()
    for s in range(steps):
        source.batch(net.x, target)
        net.forward()
        net.loss_grad(target)
        net.backward()
        k = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * s / steps))
        opt.step(lr=k)
        net.refresh(convert=False)
        hist.append(net.loss.clone())
        if log_every and (s + 1) % log_every == 0:
            log("step %d/%d loss %.5f (%.1f s)" % (s + 1, steps, float(torch.stack(hist[-log_every:]).mean()),
                                                   time.perf_counter() - t0))
    return torch.cat(hist).cpu().numpy()


def propose(net, source, images):
    """Poses [n][6] (physical units) proposed for network inputs [n][hw][hw][views]
    (n <= batch)."""
    n = images.shape[0]
    net.x.zero_()
    net.x[:n].copy_(images)
    out = net.forward()
    return (out[:n, :6] * source.scale).contiguous()


def proposal_vs_multistart(net, source, mu, n_targets=8, n_starts=16, tol=(0.5, 0.5), max_iter=150, seed=5,
                           lr=None, ncc_stop=2.0, dloss_stop=-1.0, lr_refine=None, log=None):
    """Time to a pose within tol = (mm, deg) of the truth (first iteration
    inside the tolerance box), per target pose drawn uniformly from the
    training range, with the same registration settings in both arms (Adam
    with steps lr, default the paper's 10 mm / 2 deg; the loss-based stops
    ncc_stop / dloss_stop, default off):

    * proposal: the network's pose from the target images (input
      preparation + one forward pass), then the NCC registration from that
      single start; with lr_refine also from the same start with those steps;
    * multi-start: n_starts uniform random starts from the same range, each
      registered in turn, until one reaches the tolerance.

    Returns a dict of per-target times (None where no start succeeded) and
    the proposals' errors (max over axes: mm, deg)."""
    from .registration import paper_step_sizes, register
    lr = list(paper_step_sizes() if lr is None else lr)
    geom, dev = source.geom, source.dev
    nvw = source.nvw
    rng = np.random.default_rng(seed)
    scale = source.scale.cpu().numpy().astype(np.float64)
    targets = rng.uniform(-1, 1, (n_targets, 6)) * scale
    mu_h = mu.detach().float().cpu().numpy() if torch.is_tensor(mu) else np.asarray(mu, dtype=np.float32)
    Pt = Projector(geom, n_pose=1, inst_view=np.arange(nvw), inst_pose=np.zeros(nvw, np.int32), ops=PROJ_OP_FORWARD,
                   device=dev)
    Pt.set_volume(torch.as_tensor(mu_h, device=dev))
    x = torch.zeros_like(net.x)
    kw = dict(max_iter=max_iter, ncc_stop=ncc_stop, dloss_stop=dloss_stop, tol=tol, device=dev)
    # one untimed call first: the first use of some library kernels in a process pays one-off set-up costs
    warm = Pt.forward(torch.zeros((1, 6), device=dev)).cpu().numpy()
    register(geom, mu_h, warm, np.zeros((1, 6), np.float32), lr=lr, true_pose=np.zeros(6, np.float32),
             **dict(kw, max_iter=3))
    source.images_for(torch.from_numpy(warm).to(dev).reshape(1, nvw, geom.nv, geom.nu), x[:1])
    propose(net, source, x[:1])
    res = dict(proposal_s=[], proposal_err=[], proposal_small_steps_s=[], multistart_s=[], multistart_starts=[])
    for k in range(n_targets):
        true = targets[k].astype(np.float32)
        img = Pt.forward(torch.from_numpy(true[None]).to(dev)).contiguous()
        img_h = img.cpu().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        source.images_for(img.reshape(1, nvw, geom.nv, geom.nu), x[:1])
        prop = propose(net, source, x[:1]).cpu().numpy()
        t_prop = time.perf_counter() - t0
        d = np.abs(prop[0] - true)
        res["proposal_err"].append((float(d[:3].max()), float(np.degrees(d[3:].max()))))
        r = register(geom, mu_h, img_h, prop, lr=lr, true_pose=true, **kw)
        res["proposal_s"].append(None if r["first_hit_s"] is None else t_prop + r["first_hit_s"])
        if lr_refine is not None:
            r = register(geom, mu_h, img_h, prop, lr=list(lr_refine), true_pose=true, **kw)
            res["proposal_small_steps_s"].append(None if r["first_hit_s"] is None else t_prop + r["first_hit_s"])
        starts = (rng.uniform(-1, 1, (n_starts, 6)) * scale).astype(np.float32)
        spent, hit = 0.0, None
        for c in range(n_starts):
            r = register(geom, mu_h, img_h, starts[c:c + 1], lr=lr, true_pose=true, **kw)
            if r["first_hit_s"] is not None:
                hit = (spent + r["first_hit_s"], c + 1)
                break
            spent += r["seconds"]
        res["multistart_s"].append(hit[0] if hit else None)
        res["multistart_starts"].append(hit[1] if hit else None)
        if log:
            log("target %d: proposal %s s, multistart %s s" % (k, res["proposal_s"][-1], res["multistart_s"][-1]))
    for key in ("proposal_s", "proposal_small_steps_s", "multistart_s"):
        v = [t for t in res[key] if t is not None]
        res[key + "_found"] = len(v)
        res[key + "_median"] = float(np.median(v)) if v else None
    return res

"""FP64 CPU oracle of the pose-proposal network (plain numpy).

TEST INFRASTRUCTURE ONLY, like the rest of this package: only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
it; it shares no code with the CUDA library.

The paper names learned pose initialisation as future work (Sec. V); the
network here is the small regressor the library's tensor-core kernels
serve.  Everything is the textbook definition written out:

* 3x3 convolution with stride 2 and zero padding 1 (cross-correlation, as
  deep-learning layers define it), NHWC activations, weights
  [C_out][3][3][C_in]: y[b,ho,wo,o] = b[o] + sum_{kh,kw,i}
  x[b, 2ho-1+kh, 2wo-1+kw, i] w[o,kh,kw,i], written as nine strided slices
  of the padded input (no im2col, no blocking);
* its gradients by the chain rule on the same nine slices;
* ReLU, fully connected layers y = x W^T + b, mean squared error;
* the input preparation: box average of each DRR over factor x factor
  pixels, then zero mean and unit variance per image.

The network stores its activations and back-propagated gradients in BF16.
``net_forward`` / ``net_backward`` take ``bf16=True`` to round to BF16
(round to nearest even, after rounding to FP32) at exactly those points,
so the same network can be checked tightly (same rounding points) and
loosely (pure FP64); ``bf16_round`` follows the IEEE definition of the
format (8 exponent bits, 7 stored mantissa bits) and is pinned against
torch's own conversion.
"""
from __future__ import annotations

import numpy as np


def conv3x3s2(x, w, b=None):
    """x [B,H,W,Ci], w [Co,3,3,Ci], b [Co] -> [B,(H+1)//2,(W+1)//2,Co]."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    B, H, W, _ = x.shape
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, Ho, Wo, w.shape[0]))
    for kh in range(3):
        for kw in range(3):
            patch = xp[:, kh:kh + 2 * Ho:2, kw:kw + 2 * Wo:2, :]
            y += patch @ w[:, kh, kw, :].T
    if b is not None:
        y += np.asarray(b, dtype=np.float64)
    return y


def conv3x3s2_grad(x, w, dy):
    """Gradients (dx, dw, db) of sum(conv3x3s2(x, w, b) * dy)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    B, H, W, _ = x.shape
    Ho, Wo = dy.shape[1], dy.shape[2]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for kh in range(3):
        for kw in range(3):
            sl = (slice(None), slice(kh, kh + 2 * Ho, 2), slice(kw, kw + 2 * Wo, 2), slice(None))
            dw[:, kh, kw, :] = np.einsum("bhwo,bhwi->oi", dy, xp[sl])
            dxp[sl] += dy @ w[:, kh, kw, :]
    return dxp[:, 1:H + 1, 1:W + 1, :], dw, dy.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(a):
    """Round to FP32, then to BF16 with round-to-nearest-even on the 16
    dropped bits (finite values)."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _keep(x):
    return x


def net_forward(params, x, bf16=False):
    """params: dict(conv=[(w, b), ...], fc=[(W, b), ...]); ReLU after every
    layer but the last fully connected one.  x NHWC.  Returns (out, cache).
    bf16: round every stored activation (not the output) to BF16."""
    rd = bf16_round if bf16 else _keep
    acts = [np.asarray(x, dtype=np.float64)]
    h = acts[0]
    for w, b in params["conv"]:
        h = rd(relu(conv3x3s2(h, w, b)))
        acts.append(h)
    f = h.reshape(h.shape[0], -1)
    fcs = [f]
    for j, (W, b) in enumerate(params["fc"]):
        f = f @ np.asarray(W, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
        if j + 1 < len(params["fc"]):
            f = rd(relu(f))
        fcs.append(f)
    return f, dict(acts=acts, fcs=fcs)


def net_backward(params, cache, dout, bf16=False):
    """Gradients of sum(out * dout) for every parameter, same structure as
    params, plus the input gradient.  bf16: round every back-propagated
    activation gradient (after its ReLU mask) to BF16; dout is used as
    given."""
    rd = bf16_round if bf16 else _keep
    acts, fcs = cache["acts"], cache["fcs"]
    g = np.asarray(dout, dtype=np.float64)
    fc_grads = []
    n_fc = len(params["fc"])
    for j in reversed(range(n_fc)):
        W = np.asarray(params["fc"][j][0], dtype=np.float64)
        if j + 1 < n_fc:
            g = rd(g * (fcs[j + 1] > 0))
        fc_grads.append((g.T @ fcs[j], g.sum(axis=0)))
        g = g @ W
    fc_grads.reverse()
    g = g.reshape(acts[-1].shape)
    conv_grads = []
    for l in reversed(range(len(params["conv"]))):
        g = rd(g * (acts[l + 1] > 0))
        dx, dw, db = conv3x3s2_grad(acts[l], params["conv"][l][0], g)
        conv_grads.append((dw, db))
        g = dx
    conv_grads.reverse()
    return dict(conv=conv_grads, fc=fc_grads, input=g)


def mse(y, t):
    """(mean (y - t)^2, gradient 2 (y - t) / y.size)."""
    y = np.asarray(y, dtype=np.float64)
    d = y - np.asarray(t, dtype=np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def prepare(proj, n_views, factor):
    """proj [n_img*n_views][nv][nu] -> [n_img][nv/f][nu/f][n_views]: box
    average, then per image (x - mean) / std (population std; constant
    images map to zero)."""
    p = np.asarray(proj, dtype=np.float64)
    n, nv, nu = p.shape
    d = p.reshape(n, nv // factor, factor, nu // factor, factor).mean(axis=(2, 4))
    m = d.mean(axis=(1, 2), keepdims=True)
    v = d.var(axis=(1, 2), keepdims=True)
    s = np.where(v > 1e-20, 1.0 / np.sqrt(np.where(v > 1e-20, v, 1.0)), 0.0)
    z = (d - m) * s
    return z.reshape(n // n_views, n_views, nv // factor, nu // factor).transpose(0, 2, 3, 1)

"""GPU parity of the pose-proposal network kernels (tensor-core BF16 GEMM,
im2col / col2im, transposes, column sums, input preparation, loss) against
the FP64 oracle on the same BF16-rounded inputs.

Bars.  FP32 outputs of the GEMM: the only difference from FP64 is FP32
accumulation of K exact BF16 x BF16 products, rel-L2 <= 1e-5 up to K = 8192.
BF16 outputs: one final rounding (relative 2^-9), rel-L2 <= 4e-3.  Layer
gradients that pass through a BF16 intermediate: rel-L2 <= 1e-2."""
import numpy as np
import pytest

from oracle import posenet as on

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()


import paper_2508_13304_b300 as pb  # noqa: E402


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bf16(rng, shape, scale=1.0):
    return (scale * torch.from_numpy(rng.standard_normal(shape).astype(np.float32))).to("cuda").bfloat16()


def f64(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("M,N,K,lda,ldb", [(128, 128, 64, 64, 64), (300, 48, 200, 200, 208), (1000, 256, 576, 576, 576),
                                           (64, 6, 256, 256, 256), (517, 1152, 128, 136, 128), (256, 96, 24, 24, 24)])
def test_gemm_fp32_output(M, N, K, lda, ldb):
    rng = np.random.default_rng(M + N + K)
    A, B = bf16(rng, (M, lda)), bf16(rng, (N, ldb))
    D = torch.full((M, N), float("nan"), device="cuda")
    pb.pn_gemm_bf16(M, N, K, A, lda, B, ldb, D32=D)
    torch.cuda.synchronize()
    assert pb.pn_status() == 0
    ref = f64(A)[:, :K] @ f64(B)[:, :K].T
    assert rel(D.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("M,N,K", [(512, 512, 256), (300, 512, 1000), (517, 1152, 136)])
def test_gemm_pair_tiles_match_single_sm_tiles(M, N, K):
    """The persistent and per-tile 2-SM 256 x 256 tiles (cta_group::2) and
    the 1-SM 128 x 256 tiles give the same products (same K order per
    element) and match FP64."""
    rng = np.random.default_rng(M * 7 + N)
    A, B = bf16(rng, (M, K)), bf16(rng, (N, K))
    outs = {}
    old = pb.pn_gemm_use_pair_tiles(2)
    try:
        for mode in (2, 1, 0):   # persistent 2-SM, 2-SM per tile, 1-SM
            pb.pn_gemm_use_pair_tiles(mode)
            outs[mode] = torch.empty((M, N), device="cuda")
            pb.pn_gemm_bf16(M, N, K, A, K, B, K, D32=outs[mode])
    finally:
        pb.pn_gemm_use_pair_tiles(old)
    torch.cuda.synchronize()
    assert pb.pn_status() == 0
    ref = f64(A) @ f64(B).T
    assert rel(outs[2].cpu().numpy(), ref) <= 1e-5
    assert rel(outs[2].cpu().numpy(), outs[1].cpu().numpy()) <= 1e-6
    assert rel(outs[2].cpu().numpy(), outs[0].cpu().numpy()) <= 1e-6


def test_gemm_split_k_is_deterministic_and_exact():
    rng = np.random.default_rng(9)
    M, N, K = 300, 520, 8192   # 2-SM tiles with a ragged pair and split-K
    A, B = bf16(rng, (M, K)), bf16(rng, (N, K))
    split = 8
    part = torch.empty(split * M * N, device="cuda")
    D1 = torch.empty((M, N), device="cuda")
    D2 = torch.empty((M, N), device="cuda")
    pb.pn_gemm_bf16(M, N, K, A, K, B, K, D32=D1, split_k=split, part=part)
    pb.pn_gemm_bf16(M, N, K, A, K, B, K, D32=D2, split_k=split, part=part)
    torch.cuda.synchronize()
    assert pb.pn_status() == 0
    assert torch.equal(D1, D2)
    assert rel(D1.cpu().numpy(), f64(A) @ f64(B).T) <= 1e-5
    assert 1 <= pb.pn_gemm_split_hint(M, N, K) <= 64


def test_gemm_epilogue_bias_relu_mask_bf16():
    rng = np.random.default_rng(10)
    M, N, K = 700, 64, 288
    A, B = bf16(rng, (M, K)), bf16(rng, (N, K))
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).cuda()
    mask = bf16(rng, (M, N))
    D16 = torch.empty((M, N), device="cuda", dtype=torch.bfloat16)
    D32 = torch.empty((M, N), device="cuda")
    pb.pn_gemm_bf16(M, N, K, A, K, B, K, bias=bias, mask=mask, ldm=N, relu=True, D32=D32, D16=D16)
    torch.cuda.synchronize()
    ref = np.maximum(f64(A) @ f64(B).T + bias.cpu().numpy(), 0.0) * (f64(mask) > 0)
    assert rel(D32.cpu().numpy(), ref) <= 1e-5
    assert rel(f64(D16), ref) <= 4e-3
    assert np.all(f64(D16)[f64(mask) <= 0] == 0)


def test_gemm_bounded_waits_run_out_and_report():
    """Failure path of the tensor-core GEMM, made on purpose without a fault:
    with a 1 ms wait limit and the TMA producer stalled (each stage barrier
    armed for its bytes, no copy issued), the call returns, the bounded
    mbarrier waits report through pn_status, no CTA stores its incomplete
    accumulator, and the next GEMM in the same process is exact."""
    import time
    rng = np.random.default_rng(9)
    M, N, K = 256, 128, 512          # 8 K blocks > 4 stages: the producer also waits for a free stage
    A, B = bf16(rng, (M, K)), bf16(rng, (N, K))
    assert pb.pn_status() == 0
    D = torch.full((M, N), float("nan"), device="cuda")
    pb.pn_gemm_test_hooks(wait_ns=1_000_000, stall_tma=True)
    try:
        t0 = time.perf_counter()
        pb.pn_gemm_bf16(M, N, K, A, K, B, K, D32=D)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
    finally:
        pb.pn_gemm_test_hooks(0, False)
    st = pb.pn_status()
    assert (st & 1) and (st & 4), st
    assert torch.isnan(D).all()
    assert elapsed < 1.0, elapsed
    pb.pn_gemm_bf16(M, N, K, A, K, B, K, D32=D)
    torch.cuda.synchronize()
    assert pb.pn_status() == 0
    assert rel(D.cpu().numpy(), f64(A) @ f64(B).T) <= 1e-5


def test_gemm_rejects_bad_arguments():
    A = torch.zeros((8, 24), device="cuda", dtype=torch.bfloat16)
    D = torch.zeros((8, 8), device="cuda")
    L = pb.lib()
    # lda not a multiple of 8
    assert L.pn_gemm_bf16(8, 8, 20, A.data_ptr(), 20, A.data_ptr(), 24, None, None, 0, 0, D.data_ptr(), None, 8, 1,
                          None, None) == pb.PROJ_E_ARG
    # split-K without a partial-sum buffer
    assert L.pn_gemm_bf16(8, 8, 16, A.data_ptr(), 24, A.data_ptr(), 24, None, None, 0, 0, D.data_ptr(), None, 8, 2,
                          None, None) == pb.PROJ_E_ARG
    # misaligned operand
    assert L.pn_gemm_bf16(8, 8, 16, A.data_ptr() + 2, 24, A.data_ptr(), 24, None, None, 0, 0, D.data_ptr(), None, 8,
                          1, None, None) == pb.PROJ_E_ARG
    assert "16-byte" in pb.proj_last_error()


# ------------------------------------------------------------ conv layer pieces

def conv_case(rng, B, H, W, Ci, Co):
    x = torch.relu(bf16(rng, (B, H, W, Ci)))
    w = bf16(rng, (Co, 3, 3, Ci), scale=(2.0 / (9 * Ci)) ** 0.5)
    return x, w


def kpad(Ci):
    return (9 * Ci + 7) // 8 * 8


def weight_matrix(w, kp):
    Co = w.shape[0]
    Wm = torch.zeros((Co, kp), device="cuda", dtype=torch.bfloat16)
    Wm[:, :w[0].numel()] = w.reshape(Co, -1)
    return Wm


@pytest.mark.parametrize("B,H,W,Ci,Co", [(3, 16, 16, 2, 32), (2, 18, 14, 32, 64), (1, 9, 7, 64, 128)])
def test_conv_forward_im2col_gemm(B, H, W, Ci, Co):
    rng = np.random.default_rng(B * H + Ci)
    x, w = conv_case(rng, B, H, W, Ci, Co)
    b = torch.from_numpy(0.1 * rng.standard_normal(Co).astype(np.float32)).cuda()
    kp = kpad(Ci)
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    M = B * Ho * Wo
    col = torch.empty((M, kp), device="cuda", dtype=torch.bfloat16)
    pb.pn_im2col_3x3s2(x, B, H, W, Ci, kp, col)
    Wm = weight_matrix(w, kp)
    y = torch.empty((M, Co), device="cuda")
    pb.pn_gemm_bf16(M, Co, kp, col, kp, Wm, kp, bias=b, D32=y)
    torch.cuda.synchronize()
    ref = on.conv3x3s2(f64(x), f64(w), b.cpu().numpy())
    assert rel(y.cpu().numpy().reshape(ref.shape), ref) <= 1e-5


@pytest.mark.parametrize("B,H,W,Ci,Co", [(2, 32, 32, 8, 16), (3, 31, 17, 32, 64), (4, 16, 16, 64, 128),
                                        (2, 8, 8, 128, 128), (1, 5, 7, 16, 32), (5, 9, 33, 128, 40)])
def test_conv_implicit_gemm_equals_im2col_gemm(B, H, W, Ci, Co):
    """The implicit-GEMM convolution gathers the 3x3 patches itself: its
    FP32 and BF16 outputs equal im2col + the 1-SM GEMM bit for bit (same
    products, same K order) and match the FP64 convolution.  Odd sizes leave
    ragged last M and N tiles and padding taps on every border."""
    rng = np.random.default_rng(B * H + Ci + Co)
    x, w = conv_case(rng, B, H, W, Ci, Co)
    b = torch.from_numpy(0.1 * rng.standard_normal(Co).astype(np.float32)).cuda()
    kp = kpad(Ci)
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    M = B * Ho * Wo
    col = torch.empty((M, kp), device="cuda", dtype=torch.bfloat16)
    pb.pn_im2col_3x3s2(x, B, H, W, Ci, kp, col)
    Wm = weight_matrix(w, kp)
    y32 = torch.full((M, Co), float("nan"), device="cuda")
    y16 = torch.full((M, Co), float("nan"), device="cuda", dtype=torch.bfloat16)
    pb.pn_gemm_bf16(M, Co, kp, col, kp, Wm, kp, bias=b, relu=True, D32=y32, D16=y16)
    z32 = torch.full((M, Co), float("nan"), device="cuda")
    z16 = torch.full((M, Co), float("nan"), device="cuda", dtype=torch.bfloat16)
    pb.pn_conv3x3s2_bf16(x, B, H, W, Ci, Wm, Co, bias=b, relu=True, y32=z32, y16=z16)
    torch.cuda.synchronize()
    assert pb.pn_status() == 0
    assert torch.equal(z32, y32) and torch.equal(z16, y16)
    ref = np.maximum(on.conv3x3s2(f64(x), f64(w), b.cpu().numpy()), 0.0)
    assert rel(z32.cpu().numpy().reshape(ref.shape), ref) <= 1e-5


def test_conv_implicit_gemm_rejects_bad_arguments():
    x = torch.zeros((1, 8, 8, 12), device="cuda", dtype=torch.bfloat16)
    w = torch.zeros((16, 108), device="cuda", dtype=torch.bfloat16)
    y = torch.empty((1, 4, 4, 16), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(pb.ProjError):                     # C must be a multiple of 8
        pb.pn_conv3x3s2_bf16(x, 1, 8, 8, 12, w, 16, y16=y)


def test_network_forward_implicit_equals_explicit():
    """PoseNet with implicit-GEMM convolutions and with im2col + GEMM give the
    same outputs bit for bit; the gradients of the layers after the first
    input gradient agree bit for bit too, the others within the BF16 bar
    (the implicit input gradient sums the same exact products in another
    FP32 order, and its BF16 result can round the other way)."""
    from paper_2508_13304_b300 import posenet as pn
    rng = np.random.default_rng(21)
    B = 64                                   # layer 2 has 64 x 16 x 16 = 16384 output pixels: implicit GEMM
    nets = [pn.PoseNet(B, in_hw=64, n_views=2, channels=(16, 32, 32, 32), hidden=64, seed=5, implicit=imp)
            for imp in (True, False)]
    x = torch.from_numpy(rng.standard_normal((B, 64, 64, 2)).astype(np.float32)).cuda().bfloat16()
    t = torch.from_numpy(rng.uniform(-1, 1, (B, 6)).astype(np.float32)).cuda()
    outs, grads = [], []
    for net in nets:
        outs.append(net.forward(x).clone())
        net.loss_grad(t)
        net.backward()
        grads.append([g.clone() for g in net.grads])
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])
    n_conv = len(nets[0].layers)
    for k, (g0, g1) in enumerate(zip(*grads)):
        if k >= 2 * (n_conv - 1):        # last convolution and the fully connected layers: no input gradient before
            assert torch.equal(g0, g1)
        else:
            assert rel(g0.cpu().numpy(), g1.cpu().numpy()) <= 1e-2


@pytest.mark.parametrize("B,H,W,Ci,Co", [(3, 16, 16, 2, 32), (2, 18, 14, 32, 64), (2, 8, 8, 128, 128)])
def test_conv_backward_pieces(B, H, W, Ci, Co):
    """dx = col2im(dy . W) with the ReLU mask of x; dW = dy^T . col via
    transposes and split-K; db = column sums of dy."""
    rng = np.random.default_rng(B * W + Co)
    x, w = conv_case(rng, B, H, W, Ci, Co)
    kp = kpad(Ci)
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    M = B * Ho * Wo
    dy = bf16(rng, (M, Co))
    Wm = weight_matrix(w, kp)
    WmT = torch.empty((kp, Co), device="cuda", dtype=torch.bfloat16)
    pb.pn_transpose_bf16(Wm, Co, kp, WmT, Co)
    dcol = torch.empty((M, kp), device="cuda")
    pb.pn_gemm_bf16(M, kp, Co, dy, Co, WmT, Co, D32=dcol)
    dx = torch.empty((B, H, W, Ci), device="cuda")
    pb.pn_col2im_3x3s2(dcol, B, H, W, Ci, kp, mask=x, dx32=dx)
    col = torch.empty((M, kp), device="cuda", dtype=torch.bfloat16)
    pb.pn_im2col_3x3s2(x, B, H, W, Ci, kp, col)
    Mp = (M + 7) // 8 * 8   # TMA needs 16-byte row strides
    dyT = torch.full((Co, Mp), 7.0, device="cuda", dtype=torch.bfloat16)
    colT = torch.full((kp, Mp), 7.0, device="cuda", dtype=torch.bfloat16)
    pb.pn_transpose_bf16(dy, M, Co, dyT, Mp)
    pb.pn_transpose_bf16(col, M, kp, colT, Mp)
    split = pb.pn_gemm_split_hint(Co, kp, Mp)
    part = torch.empty(max(1, split) * Co * kp, device="cuda")
    dW = torch.empty((Co, kp), device="cuda")
    pb.pn_gemm_bf16(Co, kp, Mp, dyT, Mp, colT, Mp, D32=dW, split_k=split, part=part)
    db = torch.empty(Co, device="cuda")
    scratch = torch.empty(pb.pn_colsum_scratch_floats(M, Co), device="cuda")
    pb.pn_colsum_bf16(dy, M, Co, Co, db, scratch)
    torch.cuda.synchronize()
    assert pb.pn_status() == 0
    dx_ref, dw_ref, db_ref = on.conv3x3s2_grad(f64(x), f64(w), f64(dy).reshape(B, Ho, Wo, Co))
    dx_ref = dx_ref * (f64(x) > 0)
    assert rel(dx.cpu().numpy(), dx_ref) <= 1e-5
    assert rel(dW.cpu().numpy()[:, :9 * Ci].reshape(dw_ref.shape), dw_ref) <= 1e-5
    assert np.all(dW.cpu().numpy()[:, 9 * Ci:] == 0)
    assert rel(db.cpu().numpy(), db_ref) <= 1e-6


@pytest.mark.parametrize("B,H,W,Ci,Co", [(2, 18, 14, 32, 64), (3, 17, 9, 16, 32), (2, 8, 8, 128, 128),
                                        (1, 5, 7, 40, 8), (4, 16, 16, 64, 128), (2, 11, 13, 2, 16)])
def test_conv_implicit_dgrad(B, H, W, Ci, Co):
    """The implicit-GEMM input gradient (the kernel gathers, per input pixel
    and tap, the output-gradient row that reads it) matches the FP64 input
    gradient with the ReLU mask, and the GEMM + col2im path (both FP32
    accumulation of exact BF16 products, in different orders).  Odd sizes
    leave ragged M and N tiles and taps without an output pixel on every
    border."""
    rng = np.random.default_rng(B * H * W + Ci + Co)
    x, w = conv_case(rng, B, H, W, Ci, Co)
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    M = B * Ho * Wo
    dy = bf16(rng, (M, Co))
    w9 = w.reshape(Co, 9 * Ci).contiguous()
    wt = torch.full((Ci, 9 * Co), 7.0, device="cuda", dtype=torch.bfloat16)
    pb.pn_conv_dgrad_weights(w9, Co, Ci, wt)
    dx32 = torch.full((B, H, W, Ci), float("nan"), device="cuda")
    dx16 = torch.full((B, H, W, Ci), float("nan"), device="cuda", dtype=torch.bfloat16)
    pb.pn_conv3x3s2_dgrad_bf16(dy, B, H, W, Ci, wt, Co, mask=x, dx32=dx32, dx16=dx16)
    kp = kpad(Ci)
    WmT = torch.empty((kp, Co), device="cuda", dtype=torch.bfloat16)
    pb.pn_transpose_bf16(weight_matrix(w, kp), Co, kp, WmT, Co)
    dcol = torch.empty((M, kp), device="cuda")
    pb.pn_gemm_bf16(M, kp, Co, dy, Co, WmT, Co, D32=dcol)
    dx_col = torch.empty((B, H, W, Ci), device="cuda")
    pb.pn_col2im_3x3s2(dcol, B, H, W, Ci, kp, mask=x, dx32=dx_col)
    torch.cuda.synchronize()
    assert pb.pn_status() == 0
    assert torch.equal(wt.cpu(), w.permute(3, 1, 2, 0).reshape(Ci, 9 * Co).cpu())
    dx_ref, _, _ = on.conv3x3s2_grad(f64(x), f64(w), f64(dy).reshape(B, Ho, Wo, Co))
    dx_ref = dx_ref * (f64(x) > 0)
    got = dx32.cpu().numpy()
    assert rel(got, dx_ref) <= 1e-5
    assert rel(got, dx_col.cpu().numpy()) <= 1e-5
    assert rel(dx16.float().cpu().numpy(), got) <= 4e-3
    assert np.all(got[f64(x) <= 0] == 0)


def test_conv_implicit_dgrad_rejects_bad_arguments():
    dy = torch.zeros((1, 4, 4, 12), device="cuda", dtype=torch.bfloat16)
    wt = torch.zeros((16, 108), device="cuda", dtype=torch.bfloat16)
    dx = torch.empty((1, 8, 8, 16), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(pb.ProjError):                     # cout must be a multiple of 8
        pb.pn_conv3x3s2_dgrad_bf16(dy, 1, 8, 8, 16, wt, 12, dx16=dx)
    dy16 = torch.zeros((1, 4, 4, 16), device="cuda", dtype=torch.bfloat16)
    wt16 = torch.zeros((16, 144), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(pb.ProjError):                     # no output
        pb.pn_conv3x3s2_dgrad_bf16(dy16, 1, 8, 8, 16, wt16, 16)


def test_adam_step_matches_numpy():
    """pn_adam_step: three bias-corrected Adam steps with decoupled weight decay
    on a flat FP32 array (odd length) against numpy in FP64 (FP32 rounding of
    each operation: rel <= 1e-6), and the BF16 copy of the result."""
    rng = np.random.default_rng(31)
    n = 1001
    p0 = rng.standard_normal(n)
    p = torch.from_numpy(p0.astype(np.float32)).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    p16 = torch.empty(n, device="cuda", dtype=torch.bfloat16)
    lr, b1, b2, eps, wd = 1e-2, 0.9, 0.999, 1e-8, 0.01
    P, M, V = p.cpu().numpy().astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 4):
        g = rng.standard_normal(n)
        step = lr * np.sqrt(1 - b2 ** t) / (1 - b1 ** t)
        pb.pn_adam_step(p, torch.from_numpy(g.astype(np.float32)).cuda(), m, v, step, b1, b2, eps, 1 - lr * wd, p16)
        g32 = g.astype(np.float32).astype(np.float64)
        M = b1 * M + (1 - b1) * g32
        V = b2 * V + (1 - b2) * g32 * g32
        P = P * (1 - lr * wd) - step * M / (np.sqrt(V) + eps)
    torch.cuda.synchronize()
    assert rel(p.cpu().numpy(), P) <= 1e-6
    assert rel(m.cpu().numpy(), M) <= 1e-6 and rel(v.cpu().numpy(), V) <= 1e-6
    assert torch.equal(p16, p.bfloat16())


def test_prepare_and_mse():
    rng = np.random.default_rng(12)
    n_img, n_views, nu, nv, f = 5, 2, 96, 72, 3
    proj = torch.from_numpy(rng.uniform(0, 4, (n_img * n_views, nv, nu)).astype(np.float32)).cuda()
    proj[3] = 2.0   # a constant image
    out = torch.empty((n_img, nv // f, nu // f, n_views), device="cuda", dtype=torch.bfloat16)
    pb.pn_prepare_images(proj, n_img, n_views, nu, nv, f, out)
    ref = on.prepare(proj.cpu().numpy(), n_views, f)
    torch.cuda.synchronize()
    assert rel(f64(out), ref) <= 4e-3
    assert np.all(f64(out)[1, :, :, 1] == 0)
    B, n_out, ld = 37, 6, 8
    y = torch.from_numpy(rng.standard_normal((B, ld)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, n_out)).astype(np.float32)).cuda()
    loss = torch.empty(1, device="cuda")
    dy = torch.empty((B, ld), device="cuda", dtype=torch.bfloat16)
    pb.pn_mse_loss(y, B, n_out, ld, t, loss, dy, ld)
    L_ref, g_ref = on.mse(y.cpu().numpy()[:, :n_out], t.cpu().numpy())
    assert loss.item() == pytest.approx(L_ref, rel=1e-6)
    assert rel(f64(dy)[:, :n_out], g_ref) <= 4e-3
    assert np.all(f64(dy)[:, n_out:] == 0)


# ------------------------------------------------------------ whole network

def test_network_step_matches_oracle():
    """One forward / loss / backward step of a small network.

    Tight: against the oracle network rounding to BF16 at the same points
    as the GPU (every stored activation and back-propagated gradient), on
    the same BF16 weights and input.  What remains is FP32 vs FP64
    accumulation, which moves a stored value to the neighbouring BF16 value
    for a small fraction of elements: rel-L2 <= 3e-3.

    Loose: against the plain FP64 network.  BF16 storage alone moves the
    early layers' weight gradients by 1-5 % (measured by emulating the
    rounding in FP64 on random networks of this shape), the outputs by
    < 0.6 %: bars 1e-1 and 2e-2."""
    from paper_2508_13304_b300 import posenet as pn
    rng = np.random.default_rng(21)
    B = 12
    net = pn.PoseNet(B, in_hw=32, n_views=2, channels=(8, 16, 16, 16), hidden=32, seed=3)
    for L in net.layers:
        L["b"].copy_(torch.from_numpy(0.05 * rng.standard_normal(L["cout"]).astype(np.float32)))
    net.fc[0]["b"].copy_(torch.from_numpy(0.05 * rng.standard_normal(32).astype(np.float32)))
    net.fc[1]["b"][:6] = torch.from_numpy(0.05 * rng.standard_normal(6).astype(np.float32))
    net.refresh()
    x = bf16(rng, (B, 32, 32, 2))
    t = torch.from_numpy(rng.uniform(-1, 1, (B, 6)).astype(np.float32)).cuda()
    out = net.forward(x)
    loss = net.loss_grad(t)
    net.backward()
    torch.cuda.synchronize()
    assert pb.pn_status() == 0
    P = net.as_oracle_params()
    got_out = out.cpu().numpy()
    assert np.all(got_out[:, 6:] == 0)
    got = [(L["gw"].cpu().numpy(), L["gb"].cpu().numpy(), L["cin"]) for L in net.layers]
    for L in net.layers:
        assert np.all(L["gw"].cpu().numpy()[:, 9 * L["cin"]:] == 0)
    assert np.all(net.fc[1]["gw"].cpu().numpy()[6:] == 0)
    fc_got = [(net.fc[0]["gw"].cpu().numpy(), net.fc[0]["gb"].cpu().numpy()),
              (net.fc[1]["gw"].cpu().numpy()[:6], net.fc[1]["gb"].cpu().numpy()[:6])]
    for mode, tol_out, tol_g in ((True, 3e-3, 3e-3), (False, 2e-2, 1e-1)):
        out_ref, cache = on.net_forward(P, f64(x), bf16=mode)
        L_ref, dout_ref = on.mse(out_ref, t.cpu().numpy())
        if mode:
            dout_ref = on.bf16_round(dout_ref)
        G = on.net_backward(P, cache, dout_ref, bf16=mode)
        assert rel(got_out[:, :6], out_ref) <= tol_out, mode
        assert loss.item() == pytest.approx(L_ref, rel=tol_out)
        for (gw, gb, cin), (dw, db) in zip(got, G["conv"]):
            assert rel(gw[:, :9 * cin].reshape(dw.shape), dw) <= tol_g, mode
            assert rel(gb, db) <= tol_g, mode
        for (gw, gb), (dw, db) in zip(fc_got, G["fc"]):
            assert rel(gw, dw) <= tol_g, mode
            assert rel(gb, db) <= tol_g, mode


def test_trained_proposals_beat_the_prior():
    """What the network gains: trained for a few seconds on DRRs of a small
    phantom (2 views, 32 x 32 inputs, rotations +-30 deg, translations
    +-10 mm), its proposals for fresh poses have a median error well under
    a quarter of the error of the best constant guess (the range centre,
    median |error| = half the range)."""
    import synth
    from paper_2508_13304_b300 import posenet as pn
    rng = np.random.default_rng(31)
    views = synth.circular_views(2, 300.0, 450.0, 1.5, 1.5, angles=[0.0, np.pi / 2])
    g = synth.Geometry(64, 64, 64, 1.0, 1.0, 1.0, 96, 96, views, 0.5)
    ell = synth.random_ellipsoids(rng, 8, 14.0, (4.0, 16.0), (0.01, 0.03))
    cyl = synth.random_cylinders(rng, 2, 12.0, (2.0, 4.0), (8.0, 20.0), (0.05, 0.08))
    mu = torch.from_numpy(synth.voxelise(g, ell, cyl).astype(np.float32)).cuda()
    B = 128
    net = pn.PoseNet(B, in_hw=32, channels=(16, 32, 32, 32), hidden=64, seed=1)
    src = pn.DrrSource(g, mu, B, factor=3, t_range=10.0, r_range=30.0, seed=2)
    hist = pn.train(net, src, 60000, lr=2e-3)
    assert hist[-20:].mean() < 0.25 * hist[:5].mean()
    test_src = pn.DrrSource(g, mu, B, factor=3, t_range=10.0, r_range=30.0, seed=77)
    x = torch.empty_like(net.x)
    t = torch.empty((B, 6), device="cuda")
    test_src.batch(x, t)
    err = (pn.propose(net, test_src, x) - t * test_src.scale).abs().cpu().numpy()
    torch.cuda.synchronize()
    assert pb.pn_status() == 0
    assert np.median(err[:, :3]) < 0.25 * 5.0, np.median(err[:, :3])                  # mm; prior median 5 mm
    assert np.degrees(np.median(err[:, 3:])) < 0.25 * 15.0, np.degrees(np.median(err[:, 3:]))   # prior 15 deg

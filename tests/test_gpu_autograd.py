"""torch.autograd wrappers and the registration loop (GPU)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import small_geom, smooth_volume

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()


import paper_2508_13304_b300 as pb  # noqa: E402
from paper_2508_13304_b300 import autograd as ag  # noqa: E402
from paper_2508_13304_b300 import registration as reg  # noqa: E402


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case():
    rng = np.random.default_rng(77)
    g = small_geom(n=(32, 30, 34), det=(40, 36), pix=1.6, n_views=3)
    mu = smooth_volume(g, rng, n_blobs=8).astype(np.float32)
    poses = np.array([[1.0, -2.0, 0.5, 0.06, -0.04, 0.08], [-1.5, 0.5, 1.0, -0.05, 0.07, 0.02]], dtype=np.float32)
    iv = np.array([0, 1, 2, 1], dtype=np.int32)
    ip = np.array([0, 0, 1, 1], dtype=np.int32)
    return g, mu, poses, iv, ip, rng


def test_forward_project_gradients_match_the_oracle():
    g, mu, poses, iv, ip, rng = case()
    P = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=ag.FORWARD_OPS)
    w = rng.standard_normal((4, g.nv, g.nu)).astype(np.float32)
    mu_t = torch.tensor(mu, device="cuda", requires_grad=True)
    pose_t = torch.tensor(poses, device="cuda", requires_grad=True)
    proj = ag.forward_project(mu_t, pose_t, P)
    (proj * torch.tensor(w, device="cuda")).sum().backward()
    g_pose_ref, _ = oracle.forward_grad(g, mu.astype(np.float64), poses.astype(np.float64), w.astype(np.float64),
                                        iv, ip)
    g_mu_ref = oracle.forward_adjoint(g, w.astype(np.float64), poses.astype(np.float64), iv, ip)
    gp = pose_t.grad.cpu().numpy()
    for p in range(2):
        for blk in (slice(0, 3), slice(3, 6)):
            assert rel(gp[p, blk], g_pose_ref[p, blk]) <= 1e-3
    assert rel(mu_t.grad.cpu().numpy(), g_mu_ref) <= 1e-4


def test_back_project_gradients_match_the_oracle():
    g, mu, poses, iv, ip, rng = case()
    P = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=ag.BACK_OPS)
    img = (oracle.forward(g, mu.astype(np.float64), np.zeros(6), iv, np.zeros(4, dtype=np.int32))
           + 0.05 * rng.uniform(0, 1, (4, g.nv, g.nu))).astype(np.float32)
    wv = rng.standard_normal(g.vol_shape).astype(np.float32)
    img_t = torch.tensor(img, device="cuda", requires_grad=True)
    pose_t = torch.tensor(poses, device="cuda", requires_grad=True)
    vol = ag.back_project(img_t, pose_t, P, pb.PROJ_W_FDK)
    (vol * torch.tensor(wv, device="cuda")).sum().backward()
    g_pose_ref, _ = oracle.back_grad(g, img.astype(np.float64), poses.astype(np.float64), wv.astype(np.float64), iv,
                                     ip, weight=oracle.W_FDK)
    g_img_ref = oracle.back_adjoint(g, wv.astype(np.float64), poses.astype(np.float64), iv, ip, weight=oracle.W_FDK)
    gp = pose_t.grad.cpu().numpy()
    for p in range(2):
        for blk in (slice(0, 3), slice(3, 6)):
            assert rel(gp[p, blk], g_pose_ref[p, blk]) <= 1e-3
    assert rel(img_t.grad.cpu().numpy(), g_img_ref) <= 1e-4


def test_autograd_pose_gradient_agrees_with_finite_differences():
    """The paper's accuracy metric (Sec. II-D.1): cosine similarity between
    the analytic pose gradient (through autograd, NCC loss in torch) and a
    central finite difference of the loss, here on the GPU in FP32."""
    g, mu, poses, iv, ip, rng = case()
    P = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=ag.FORWARD_OPS)
    target = torch.tensor(oracle.forward(g, mu.astype(np.float64), np.zeros(6), np.arange(3),
                                         np.zeros(3, dtype=np.int32)), device="cuda", dtype=torch.float32)
    mu_t = torch.tensor(mu, device="cuda")

    def loss_of(pz):
        return ag.ncc_loss(ag.forward_project(mu_t, pz, P), target, iv, ip, 2).sum()

    pose_t = torch.tensor(poses, device="cuda", requires_grad=True)
    loss_of(pose_t).backward()
    ga = pose_t.grad.cpu().numpy().astype(np.float64)
    fd = np.zeros_like(ga)
    steps = [0.05] * 3 + [5e-4] * 3
    with torch.no_grad():
        for p in range(2):
            for j in range(6):
                e = torch.zeros((2, 6), device="cuda")
                e[p, j] = steps[j]
                base = torch.tensor(poses, device="cuda")
                fd[p, j] = (loss_of(base + e).item() - loss_of(base - e).item()) / (2 * steps[j])
    for p in range(2):
        assert oracle.cosine(ga[p], fd[p] * np.array([1, 1, 1, 1, 1, 1])) >= 0.99, (ga[p], fd[p])


def test_batched_registration_converges():
    """Small registration: 3 views of an ellipsoid phantom, starts within
    3 deg and 3 mm of the true pose; every candidate's NCC loss decreases,
    the batched and plain loops follow the same trajectories, and the
    median candidate ends within 0.5 deg / 0.5 mm of the true pose."""
    rng = np.random.default_rng(5)
    views = synth.circular_views(3, 300.0, 450.0, 1.2, 1.2, angles=[0.0, 1.2, 2.4])
    g = synth.Geometry(40, 40, 40, 1.0, 1.0, 1.0, 48, 48, views, 0.5)
    ell = synth.random_ellipsoids(rng, 8, 8.0, (3.0, 8.0), (0.01, 0.03))
    mu = synth.voxelise(g, ell, supersample=2).astype(np.float32)
    true = np.array([1.5, -1.0, 0.5, 0.03, -0.02, 0.04], dtype=np.float32)
    target = oracle.forward(g, mu.astype(np.float64), true.astype(np.float64), np.arange(3),
                            np.zeros(3, dtype=np.int32))
    starts = true + np.concatenate([rng.uniform(-3, 3, (6, 3)), np.deg2rad(rng.uniform(-3, 3, (6, 3)))], axis=1)
    lr = [0.5] * 3 + [np.deg2rad(0.5)] * 3
    kw = dict(max_iter=400, lr=lr, ncc_stop=1.0, dloss_stop=1e-8)
    out_b = reg.register(g, mu, target, starts, batched=True, **kw)
    out_p = reg.register(g, mu, target, starts[:2], batched=False, **kw)
    te, re = reg.pose_error(out_b["poses"], true)
    assert np.all(out_b["ncc"] > 0.99), out_b["ncc"]
    assert np.median(te) < 0.5 and np.median(re) < 0.5, (te, re, out_b["ncc"])
    np.testing.assert_allclose(out_p["poses"], out_b["poses"][:2], atol=1e-4)


def test_independent_single_view_registrations_match_separate_runs():
    """register(inst_view=...) advances independent single-view problems
    (pose i against view i) in one launch; each follows the trajectory it
    has when registered alone."""
    rng = np.random.default_rng(6)
    views = synth.circular_views(3, 300.0, 450.0, 1.2, 1.2, angles=[0.2, 1.3, 2.5])
    g = synth.Geometry(40, 40, 40, 1.0, 1.0, 1.0, 48, 48, views, 0.5)
    ell = synth.random_ellipsoids(rng, 8, 8.0, (3.0, 8.0), (0.01, 0.03))
    mu = synth.voxelise(g, ell, supersample=2).astype(np.float32)
    target = oracle.forward(g, mu.astype(np.float64), np.zeros(6), np.arange(3), np.zeros(3, dtype=np.int32))
    starts = np.concatenate([rng.uniform(-2, 2, (3, 3)), np.deg2rad(rng.uniform(-2, 2, (3, 3)))],
                            axis=1).astype(np.float32)
    kw = dict(max_iter=40, lr=[0.5] * 3 + [np.deg2rad(0.5)] * 3, ncc_stop=1.0, dloss_stop=-1.0)
    together = reg.register(g, mu, target, starts, inst_view=[0, 1, 2], **kw)
    for i in range(3):
        alone = reg.register(g, mu, target, starts[i:i + 1], inst_view=[i], **kw)
        np.testing.assert_array_equal(together["poses"][i], alone["poses"][0])
        assert together["ncc"][i] == alone["ncc"][0]
    assert np.all(together["ncc"] > 0.9)

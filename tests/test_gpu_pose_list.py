"""The per-call pose list of the fused pose gradient
(proj_forward_pose_grad_list) and the multi-start registration built on it
(registration.register_waves): listed poses give the oracle's gradients and
exactly the plan-wide call's values, unlisted rows stay untouched, bad
indices raise a status bit, and starts run in refilled waves follow the
trajectories they have alone."""
import numpy as np
import pytest

import oracle
import synth
from helpers import small_geom, smooth_volume

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()


import paper_2508_13304_b300 as pb  # noqa: E402
from paper_2508_13304_b300 import registration as reg  # noqa: E402


def grad_rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1, 6)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 6)
    worst = 0.0
    for p in range(b.shape[0]):
        for blk in (slice(0, 3), slice(3, 6)):
            worst = max(worst, np.linalg.norm(a[p, blk] - b[p, blk]) / np.linalg.norm(b[p, blk]))
    return worst


def case(n_pose=4):
    rng = np.random.default_rng(77)
    g = small_geom(n=(37, 42, 33), vox=(1.1, 0.9, 1.0), det=(41, 46), pix=1.5, n_views=3, off=(0.8, -1.2, 0.5))
    mu = smooth_volume(g, rng, n_blobs=8).astype(np.float32)
    poses = np.concatenate([rng.uniform(-3, 3, (n_pose, 3)), rng.uniform(-0.12, 0.12, (n_pose, 3))],
                           axis=1).astype(np.float32)
    # uneven instance counts per pose: pose 0 sees 3 views, pose 1 one, the others 2
    iv = np.array([0, 1, 2, 1, 0, 2, 1, 2][:2 * n_pose], dtype=np.int32)
    ip = np.array([0, 0, 0, 1, 2, 2, 3, 3][:2 * n_pose], dtype=np.int32)
    target = rng.uniform(0, 1, (3, g.nv, g.nu)).astype(np.float32)
    return g, mu, poses, iv, ip, target


@pytest.mark.parametrize("loss", [pb.PROJ_LOSS_L2, pb.PROJ_LOSS_NCC])
def test_listed_poses_match_the_full_call_and_the_oracle(loss):
    g, mu, poses, iv, ip, target = case()
    dev = torch.device("cuda", torch.cuda.current_device())
    P = pb.Projector(g, n_pose=4, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(torch.from_numpy(mu).to(dev))
    pose_d = torch.from_numpy(poses).to(dev)
    tgt = torch.from_numpy(target).to(dev)
    full_g, full_l, full_p = P.forward_pose_grad(pose_d, loss, tgt, want_proj=True)
    lst = torch.tensor([2, -1, 0, 3, 2], dtype=torch.int32, device=dev)   # an empty slot and a duplicate
    grad = torch.full((4, 6), float("nan"), device=dev)
    lossv = torch.full((4,), float("nan"), device=dev)
    proj = torch.full_like(full_p, float("nan"))
    pb.proj_forward_pose_grad_list(P.plan, pose_d, lst, loss, tgt, grad, lossv, proj, P.ws)
    assert P.check() == 0
    g_np, l_np, p_np = grad.cpu().numpy(), lossv.cpu().numpy(), proj.cpu().numpy()
    for q in (0, 2, 3):
        np.testing.assert_array_equal(g_np[q], full_g.cpu().numpy()[q])
        assert l_np[q] == full_l.cpu().numpy()[q]
    assert np.isnan(g_np[1]).all() and np.isnan(l_np[1])
    for i in range(len(iv)):
        if ip[i] == 1:
            assert np.isnan(p_np[i]).all()
        else:
            np.testing.assert_array_equal(p_np[i], full_p.cpu().numpy()[i])
    proj_ref = oracle.forward(g, mu, poses, iv, ip)
    _, w = oracle.pose_loss_weights("l2" if loss == pb.PROJ_LOSS_L2 else "ncc", proj_ref, target, iv, ip, 4)
    gth, _ = oracle.forward_grad(g, mu, poses, w, iv, ip, mode=oracle.GRAD_ANALYTIC)
    assert grad_rel(g_np[[0, 2, 3]], np.asarray(gth)[[0, 2, 3]]) <= TOL_GRAD


def test_out_of_range_entries_set_a_status_bit():
    g, mu, poses, iv, ip, target = case()
    dev = torch.device("cuda", torch.cuda.current_device())
    P = pb.Projector(g, n_pose=4, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(torch.from_numpy(mu).to(dev))
    pose_d = torch.from_numpy(poses).to(dev)
    tgt = torch.from_numpy(target).to(dev)
    full_g, _ = P.forward_pose_grad(pose_d, pb.PROJ_LOSS_L2, tgt)
    assert P.check() == 0
    grad = torch.full((4, 6), float("nan"), device=dev)
    lst = torch.tensor([7, 1, -5], dtype=torch.int32, device=dev)
    pb.proj_forward_pose_grad_list(P.plan, pose_d, lst, pb.PROJ_LOSS_L2, tgt, grad, None, None, P.ws)
    assert P.check() == pb.PROJ_STATUS_BAD_INDEX
    np.testing.assert_array_equal(grad.cpu().numpy()[1], full_g.cpu().numpy()[1])
    assert np.isnan(grad.cpu().numpy()[[0, 2, 3]]).all()
    with pytest.raises(pb.ProjError):      # n_list must be >= 1
        pb.proj_forward_pose_grad_list(P.plan, pose_d, torch.zeros(0, dtype=torch.int32, device=dev),
                                       pb.PROJ_LOSS_L2, tgt, grad, None, None, P.ws)


def test_waves_follow_the_trajectories_of_single_starts():
    """register_waves with 2 slots over 5 starts (stops on, so starts leave
    and new ones join mid-run): every start ends exactly where it ends when
    registered alone, after the same number of updates."""
    rng = np.random.default_rng(8)
    views = synth.circular_views(2, 300.0, 450.0, 1.2, 1.2, angles=[0.0, np.pi / 2])
    g = synth.Geometry(40, 40, 40, 1.0, 1.0, 1.0, 48, 48, views, 0.5)
    ell = synth.random_ellipsoids(rng, 8, 8.0, (3.0, 8.0), (0.01, 0.03))
    mu = synth.voxelise(g, ell, supersample=2).astype(np.float32)
    true = np.array([1.0, -0.5, 0.5, 0.02, -0.03, 0.01], dtype=np.float32)
    target = oracle.forward(g, mu.astype(np.float64), true.astype(np.float64), np.arange(2),
                            np.zeros(2, dtype=np.int32))
    starts = true + np.concatenate([rng.uniform(-3, 3, (5, 3)), np.deg2rad(rng.uniform(-3, 3, (5, 3)))], axis=1)
    kw = dict(max_iter=60, lr=[0.5] * 3 + [np.deg2rad(0.5)] * 3, ncc_stop=0.9999, dloss_stop=1e-7)
    w = reg.register(g, mu, target, starts, wave=2, **kw)
    assert w["started"] == 5
    for i in range(5):
        alone = reg.register(g, mu, target, starts[i:i + 1], batched=True, **kw)
        np.testing.assert_array_equal(w["poses"][i], alone["poses"][0])
        assert w["iters"][i] == alone["iters"][0]
    assert len(set(w["iters"].tolist())) > 1      # starts stopped at different iterations

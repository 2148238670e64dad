"""GPU parity at full sizes, in the launch configurations the benchmark times,
on outputs the FP64 oracle can compute one by one (sampled candidates, views,
pixels and voxels).  Bars as in test_gpu_parity: images rel-L2 <= 1e-4, pose
gradients rel <= 1e-3 per pose on each block."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_IMG = 1e-4
TOL_GRAD = 1e-3


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


def grad_rel(g_gpu, g_ref):
    worst = 0.0
    for blk in (slice(0, 3), slice(3, 6)):
        worst = max(worst, rel(g_gpu[blk], g_ref[blk]))
    return worst


def f32(a):
    return np.asarray(a, dtype=np.float32)


def test_registration_batch_full_size():
    """256^3, 2 views of 384^2, 64 candidates in one launch, NCC fused;
    candidates 0, 31 and 63 checked against the oracle."""
    w = synth.workload_registration(n_cand=64)
    g = w["geom"]
    mu = f32(w["mu"])
    poses = f32(w["poses"])
    iv2, ip2 = np.arange(2), np.zeros(2, dtype=np.int32)
    target = f32(oracle.forward(g, mu.astype(np.float64), f32(w["pose_true"]).astype(np.float64), iv2, ip2))
    iv = np.tile(np.arange(2, dtype=np.int32), 64)
    ip = np.repeat(np.arange(64, dtype=np.int32), 2)
    P = pb.Projector(g, n_pose=64, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(mu)
    grad, loss, proj = P.forward_pose_grad(poses, pb.PROJ_LOSS_NCC, target, want_proj=True)
    grad, loss, proj = grad.cpu().numpy(), loss.cpu().numpy(), proj.cpu().numpy()
    for c in (0, 31, 63):
        pose = poses[c].astype(np.float64)
        pr = oracle.forward(g, mu.astype(np.float64), pose, iv2, ip2)
        L, wts = oracle.pose_loss_weights("ncc", pr, target, iv2, ip2, 1)
        gref, _ = oracle.forward_grad(g, mu.astype(np.float64), pose, wts, iv2, ip2)
        assert rel(proj[2 * c:2 * c + 2], pr) <= TOL_IMG
        assert grad_rel(grad[c], gref[0]) <= TOL_GRAD, (c, grad[c], gref[0])
        assert abs(loss[c] - L[0]) <= 1e-4 * abs(L[0])


def test_moco_back_projection_full_size():
    """256^3, 360 views of 512^2 at 0.6 mm, per-view smooth motion, FDK
    weight: back-projection at 3000 sampled voxels and the pose gradient of
    6 sampled views, from one full-size launch each."""
    rng = np.random.default_rng(1003)
    g = synth.Geometry(256, 256, 256, 0.8, 0.8, 0.8, 512, 512,
                       synth.circular_views(360, synth.SAD, synth.SDD, 0.6, 0.6), 0.4)
    motion = f32(synth.smooth_motion(rng, 360, 2.0, 3.0))
    img = f32(rng.uniform(0.0, 1.0, (360, 512, 512)))
    wvol = f32(rng.standard_normal((256, 256, 256)))
    P = pb.Projector(g, n_pose=360, inst_view=np.arange(360), inst_pose=np.arange(360),
                     ops=pb.PROJ_OP_BACK | pb.PROJ_OP_BACK_GRAD)
    vol = P.back(img, motion, pb.PROJ_W_FDK).cpu().numpy()
    grad = P.back_pose_grad(img, motion, wvol, pb.PROJ_W_FDK).cpu().numpy()
    vox = np.stack([rng.integers(0, 256, 3000), rng.integers(0, 256, 3000), rng.integers(0, 256, 3000)], axis=1)
    ref = oracle.back_voxels(g, img, motion.astype(np.float64), vox, np.arange(360), np.arange(360),
                             weight=oracle.W_FDK)
    assert rel(vol[vox[:, 2], vox[:, 1], vox[:, 0]], ref) <= TOL_IMG
    views = np.array([0, 77, 151, 200, 299, 359])
    gref, _ = oracle.back_grad(g, img[views], motion[views].astype(np.float64), wvol.astype(np.float64),
                               inst_view=views, inst_pose=np.arange(len(views)), weight=oracle.W_FDK)
    for i, v in enumerate(views):
        assert grad_rel(grad[v], gref[i]) <= TOL_GRAD, (v, grad[v], gref[i])


def test_calibration_forward_full_size():
    """512^3 at 0.5 mm, 720 views of 768^2 at 0.556 mm, per-view pose
    noise: forward projection of 2000 sampled pixels and the residual
    pose gradient of one view, from full-size launches."""
    rng = np.random.default_rng(1004)
    base = synth.workload_registration(seed=1004, n_cand=1, nvox=256, ndet=8, vox=1.0)["mu"]
    mu = f32(np.repeat(np.repeat(np.repeat(base, 2, 0), 2, 1), 2, 2))
    g = synth.Geometry(512, 512, 512, 0.5, 0.5, 0.5, 768, 768,
                       synth.circular_views(720, synth.SAD, synth.SDD, 0.556, 0.556), 0.25)
    poses = np.zeros((720, 6))
    poses[:, :3] = rng.normal(0.0, 1.0, (720, 3))
    poses[:, 3:] = np.deg2rad(rng.normal(0.0, 0.5, (720, 3)))
    poses = f32(poses)
    P = pb.Projector(g, n_pose=720, inst_view=np.arange(720), inst_pose=np.arange(720),
                     ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(mu)
    proj = P.forward(poses).cpu().numpy()
    pix = np.stack([rng.integers(0, 720, 2000), rng.integers(0, 768, 2000), rng.integers(0, 768, 2000)], axis=1)
    ref = oracle.forward_pixels(g, mu.astype(np.float64), poses.astype(np.float64), pix, np.arange(720),
                                np.arange(720))
    assert rel(proj[pix[:, 0], pix[:, 2], pix[:, 1]], ref) <= TOL_IMG
    del proj
    resid = rng.standard_normal((720, 768, 768), dtype=np.float32)
    grad, _ = P.forward_pose_grad(poses, pb.PROJ_LOSS_RESIDUAL, resid)
    grad = grad.cpu().numpy()
    v = 123
    gref, _ = oracle.forward_grad(g, mu.astype(np.float64), poses[v].astype(np.float64),
                                  resid[v:v + 1].astype(np.float64), inst_view=[v], inst_pose=[0])
    assert grad_rel(grad[v], gref[0]) <= TOL_GRAD, (grad[v], gref[0])


def test_pose_proposal_drr_batch_full_size():
    """The network's training batch in the benchmark's configuration: 256
    poses (rot +-30 deg, trans +-40 mm) x 2 views of 384^2 from 256^3 at
    0.8 mm, down-sampled 3x to 128^2 BF16 inputs.  2000 sampled DRR pixels
    against the FP64 march, and the prepared inputs of three poses against
    the oracle's box average and standardisation of the same projections
    (BF16 storage: <= 4e-3 rel-L2)."""
    from oracle import posenet as on
    from paper_2508_13304_b300 import posenet as pn
    w = synth.workload_registration(seed=1002, n_cand=1)
    g = w["geom"]
    mu = torch.from_numpy(w["mu"]).cuda()
    B = 256
    src = pn.DrrSource(g, mu, B, factor=3, seed=7)
    x = torch.empty((B, 128, 128, 2), device="cuda", dtype=torch.bfloat16)
    t = torch.empty((B, 6), device="cuda")
    src.batch(x, t)
    torch.cuda.synchronize()
    assert float(t.abs().max()) <= 1.0
    pose = (t * src.scale).cpu().numpy()      # the poses the batch was rendered at
    proj = src.proj.cpu().numpy()
    rng = np.random.default_rng(55)
    inst = rng.integers(0, 2 * B, 2000)
    pix = np.stack([inst, rng.integers(0, 384, 2000), rng.integers(0, 384, 2000)], axis=1)
    ref = oracle.forward_pixels(g, w["mu"].astype(np.float64), pose.astype(np.float64), pix,
                                np.tile([0, 1], B), np.repeat(np.arange(B), 2))
    assert rel(proj[pix[:, 0], pix[:, 2], pix[:, 1]], ref) <= TOL_IMG
    xs = x.float().cpu().numpy()
    for b in (0, 101, 255):
        prep = on.prepare(proj[2 * b:2 * b + 2], 2, 3)[0]
        assert rel(xs[b], prep) <= 4e-3, b


def test_uneven_batch_full_size():
    """The uneven calibration batch in one persistent launch: 512^3 with 720
    per-view poses on 768^2 detectors plus 24 single-view problems (volumes
    128..320^3, detectors 256..512^2), L2 loss.  Every problem's gradients
    and losses equal those of its own proj_forward_pose_grad call; two views
    of the large problem and three of the small ones against the oracle."""
    rng = np.random.default_rng(1004)
    gen = torch.Generator(device="cuda").manual_seed(1004)
    items, host = [], []
    for q in synth.workload_uneven(with_large=True):
        g = q["geom"]
        nvw = g.n_views
        mu = rng.random((g.nz, g.ny, g.nx), dtype=np.float32)
        P = pb.Projector(g, n_pose=nvw, inst_view=np.arange(nvw), inst_pose=np.arange(nvw),
                         ops=pb.PROJ_OP_FORWARD_GRAD)
        P.set_volume(mu)
        items.append(dict(plan=P.plan, loss=pb.PROJ_LOSS_L2, pose=torch.from_numpy(f32(q["poses"])).cuda(),
                          ref=torch.rand((nvw, g.nv, g.nu), device="cuda", generator=gen), grad=torch.zeros((nvw, 6), device="cuda"),
                          loss_out=torch.zeros(nvw, device="cuda"), ws=P.ws))
        host.append((g, mu, f32(q["poses"]), P))
    b = pb.proj_batch_create(items)
    pb.proj_batch_run(b)
    torch.cuda.synchronize()
    got = [(it["grad"].cpu().numpy(), it["loss_out"].cpu().numpy()) for it in items]
    for k, (it, (g, mu, pose, P)) in enumerate(zip(items, host)):
        gs, ls = P.forward_pose_grad(it["pose"], pb.PROJ_LOSS_L2, it["ref"])
        assert rel(got[k][0], gs.cpu().numpy()) <= 1e-6, k
        np.testing.assert_allclose(got[k][1], ls.cpu().numpy(), rtol=1e-6)
    order = np.argsort([h[0].nx * h[0].nu ** 2 for h in host[1:]]) + 1
    for k, v in [(0, 0), (0, 437)] + [(int(k), 0) for k in (order[0], order[12], order[-1])]:
        g, mu, pose, _ = host[k]
        ref = items[k]["ref"][v:v + 1].cpu().numpy().astype(np.float64)
        pr = oracle.forward(g, mu.astype(np.float64), pose[v].astype(np.float64), [v], [0])
        L, w = oracle.pose_loss_weights("l2", pr, ref, [0], [0], 1)
        gref, _ = oracle.forward_grad(g, mu.astype(np.float64), pose[v].astype(np.float64), w, [v], [0])
        assert grad_rel(got[k][0][v], gref[0]) <= TOL_GRAD, (k, v, got[k][0][v], gref[0])
        assert abs(got[k][1][v] - L[0]) <= 1e-4 * abs(L[0]), (k, v)


def test_odd_sizes_records_and_transposes():
    """Large odd sizes for the cell-record layouts: a 257 x 300 x 259 volume
    (odd slice count, anisotropic voxels) and 513 x 385 detectors, 6 views
    with their own poses.  Forward projection at 1500 sampled pixels and
    back-projection at 1500 sampled voxels against the oracle; both
    transposes through the adjoint identities <A x, y> = <x, A^T y> against
    the GPU's own forward and back-projection."""
    rng = np.random.default_rng(77)
    views = synth.circular_views(6, synth.SAD, synth.SDD, 0.7, 0.65)
    g = synth.Geometry(257, 300, 259, 0.8, 0.75, 0.7, 513, 385, views, 0.375, (1.0, -2.0, 0.5))
    mu = f32(rng.random((259, 300, 257), dtype=np.float32))
    poses = np.zeros((6, 6))
    poses[:, :3] = rng.normal(0.0, 2.0, (6, 3))
    poses[:, 3:] = np.deg2rad(rng.normal(0.0, 3.0, (6, 3)))
    poses = f32(poses)
    iv = np.arange(6, dtype=np.int32)
    P = pb.Projector(g, n_pose=6, inst_view=iv, inst_pose=iv,
                     ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_ADJOINT | pb.PROJ_OP_BACK)
    P.set_volume(mu)
    proj = P.forward(poses).cpu().numpy()
    pix = np.stack([rng.integers(0, 6, 1500), rng.integers(0, 513, 1500), rng.integers(0, 385, 1500)], axis=1)
    ref = oracle.forward_pixels(g, mu.astype(np.float64), poses.astype(np.float64), pix, iv, iv)
    assert rel(proj[pix[:, 0], pix[:, 2], pix[:, 1]], ref) <= TOL_IMG
    img = f32(rng.random((6, 385, 513), dtype=np.float32))
    vol = P.back(img, poses, pb.PROJ_W_FDK).cpu().numpy()
    vox = np.stack([rng.integers(0, 257, 1500), rng.integers(0, 300, 1500), rng.integers(0, 259, 1500)], axis=1)
    refb = oracle.back_voxels(g, img.astype(np.float64), poses.astype(np.float64), vox, iv, iv, weight=oracle.W_FDK)
    assert rel(vol[vox[:, 2], vox[:, 1], vox[:, 0]], refb) <= TOL_IMG
    # <A mu, img> = <mu, A^T img>, <B img, x> = <img, B^T x>
    at = P.forward_adjoint(img, poses).cpu().numpy()
    lhs, rhs = np.vdot(proj.astype(np.float64), img), np.vdot(mu.astype(np.float64), at)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    x = f32(rng.standard_normal((259, 300, 257), dtype=np.float32))
    bt = P.back_adjoint(x, poses, pb.PROJ_W_FDK).cpu().numpy()
    lhs, rhs = np.vdot(vol.astype(np.float64), x), np.vdot(img, bt.astype(np.float64))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(vol) * np.linalg.norm(x)

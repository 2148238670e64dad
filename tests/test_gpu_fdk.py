"""FDK filtering, sharpness loss and the motion-compensated FDK loop (GPU)."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()


import paper_2508_13304_b300 as pb  # noqa: E402
from paper_2508_13304_b300 import moco  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_fdk_filter_matches_the_oracle():
    rng = np.random.default_rng(61)
    views = synth.circular_views(5, 300.0, 450.0, 0.9, 1.1)
    views[2, 3:6] += np.array([2.0, 1.0, -3.0])          # shifted detector centre (principal point off-centre)
    g = synth.Geometry(8, 8, 8, 1.0, 1.0, 1.0, 77, 51, views, 0.5)
    proj = rng.uniform(0, 1, (5, 51, 77)).astype(np.float32)
    P = pb.Projector(g, n_pose=5, inst_view=np.arange(5), inst_pose=np.arange(5), ops=pb.PROJ_OP_BACK)
    got = P.fdk_filter(proj, 0.3).cpu().numpy()
    ref = oracle.fdk_filter(g, proj, np.arange(5), 0.3)
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("shape", [(20, 18, 22), (64, 64, 64)])
def test_sharpness_matches_the_oracle(shape):
    rng = np.random.default_rng(62)
    g = synth.Geometry(shape[2], shape[1], shape[0], 0.9, 1.0, 1.1, 8, 8, synth.circular_views(1, 100, 150, 1, 1), 0.5)
    mu = rng.uniform(0, 1, shape).astype(np.float32)
    mu[mu < 0.3] = 0.0                                       # flat regions: |grad mu| = 0 voxels
    P = pb.Projector(g, n_pose=1, inst_view=[0], inst_pose=[0], ops=pb.PROJ_OP_SHARPNESS)
    loss, grad = P.sharpness(mu)
    vox = (0.9, 1.0, 1.1)
    assert abs(loss.item() - oracle.sharpness(mu, vox)) <= 1e-5 * abs(oracle.sharpness(mu, vox))
    assert rel(grad.cpu().numpy(), oracle.sharpness_grad(mu, vox)) <= 1e-4


def test_motion_compensated_fdk_loop():
    """60 views of an ellipsoid phantom with smooth zero-mean per-view motion
    (rot <= 2 deg, trans <= 3 mm): the loss prefers the true motion to no
    motion, its descent direction at zero motion points towards the true
    translations, and the loop lowers it.  (With independent 6-DOF poses per
    view this loss also has sharper, streaky minima beyond the true motion,
    so the loop's end point is not asserted to be the true motion.)"""
    rng = np.random.default_rng(63)
    n_views = 60
    views = synth.circular_views(n_views, 300.0, 450.0, 1.6, 1.6)
    g = synth.Geometry(48, 48, 48, 1.5, 1.5, 1.5, 80, 80, views, 0.75)
    ell = synth.random_ellipsoids(rng, 10, 12.0, (3.0, 10.0), (0.01, 0.03))
    mu = synth.voxelise(g, ell, supersample=2).astype(np.float32)
    motion = synth.smooth_motion(rng, n_views, 2.0, 3.0).astype(np.float32)
    motion -= motion.mean(axis=0)
    P = pb.Projector(g, n_pose=n_views, inst_view=np.arange(n_views), inst_pose=np.arange(n_views),
                     ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_BACK | pb.PROJ_OP_BACK_GRAD | pb.PROJ_OP_SHARPNESS)
    P.set_volume(mu)
    proj = P.forward(motion)
    q = P.fdk_filter(proj, math.pi / n_views)
    zero = np.zeros_like(motion)
    s_zero, d_zero = P.sharpness(P.back(q, zero, pb.PROJ_W_FDK))
    s_true = P.sharpness(P.back(q, motion, pb.PROJ_W_FDK), want_grad=False)
    assert s_true.item() < s_zero.item()
    gz = P.back_pose_grad(q, zero, d_zero, pb.PROJ_W_FDK).cpu().numpy()
    cos_t = float(np.sum(-gz[:, :3] * motion[:, :3]) / np.linalg.norm(gz[:, :3]) / np.linalg.norm(motion[:, :3]))
    assert cos_t > 0.3, cos_t
    out = moco.moco_fdk(g, proj.cpu().numpy(), n_iter=20,
                        lr=[0.02] * 3 + [math.radians(0.02)] * 3)
    s = out["sharpness"]
    assert s[-1] < s[0], s


def test_spline_motion_recovers_the_reconstruction():
    """Motion-compensated FDK with the motion as a centred 24-node cubic
    B-spline over the views (translations only): on the 60-view phantom of
    the test above, the reconstruction's distance to the motion-free one
    falls by more than half (to the level that the true motion gives), and
    the translation error drops."""
    rng = np.random.default_rng(63)
    n_views = 60
    views = synth.circular_views(n_views, 300.0, 450.0, 1.6, 1.6)
    g = synth.Geometry(48, 48, 48, 1.5, 1.5, 1.5, 80, 80, views, 0.75)
    ell = synth.random_ellipsoids(rng, 10, 12.0, (3.0, 10.0), (0.01, 0.03))
    mu = synth.voxelise(g, ell, supersample=2).astype(np.float32)
    motion = synth.smooth_motion(rng, n_views, 2.0, 3.0).astype(np.float32)
    motion -= motion.mean(axis=0)
    F = pb.Projector(g, n_pose=n_views, inst_view=np.arange(n_views), inst_pose=np.arange(n_views),
                     ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_BACK)
    F.set_volume(mu)
    proj = F.forward(motion)
    zero = np.zeros((n_views, 6), np.float32)
    ref = F.back(F.fdk_filter(F.forward(zero), math.pi / n_views), zero, pb.PROJ_W_FDK).cpu().numpy()
    out = moco.moco_fdk(g, proj.cpu().numpy(), n_iter=80, lr=[0.05] * 3 + [0.0] * 3, spline_nodes=24)
    e0, e1 = rel(out["fdk0"], ref), rel(out["fdk"], ref)
    assert e1 < 0.5 * e0, (e0, e1)
    d = out["poses"] - motion
    assert np.sqrt((d[:, :3] ** 2).mean()) < np.sqrt((motion[:, :3] ** 2).mean())
    assert out["sharpness"][-1] < out["sharpness"][0]

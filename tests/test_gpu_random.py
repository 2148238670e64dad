"""Randomised GPU parity: small geometries drawn at random (odd and even
sizes from 1 voxel / 1 pixel up, anisotropic voxels, volume offsets, views of
a circular orbit turned by a random rotation so that neither detector axis
lies along a grid axis, poses with large rotations), every call against the
FP64 oracle at the parity bars, and both transposes through their adjoint
identities.  Exercises the layout choices of the kernels (cell records, slice
pairs, the copy with rows along y, band-major tile order) away from the
benchmark geometries."""
import numpy as np
import pytest

import oracle
import synth
from helpers import smooth_volume

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def grad_ok(g_gpu, g_ref):
    for blk in (slice(0, 3), slice(3, 6)):
        nb = np.linalg.norm(g_ref[blk])
        if nb > 1e-12 and np.linalg.norm(g_gpu[blk] - g_ref[blk]) > TOL_GRAD * nb:
            return False
    return True


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def random_case(seed):
    rng = np.random.default_rng(seed)
    n = rng.integers(1, 42, 3)
    vox = rng.uniform(0.6, 1.8, 3)
    ext = float(np.linalg.norm(n * vox))
    nu, nv = rng.integers(1, 52, 2)
    n_views = int(rng.integers(1, 4))
    sad = ext * rng.uniform(1.5, 4.0)
    sdd = sad * rng.uniform(1.2, 2.0)
    pix = 1.3 * ext * sdd / sad / max(nu, nv, 8)
    views = synth.circular_views(n_views, sad, sdd, pix, pix * rng.uniform(0.8, 1.25),
                                 angles=rng.uniform(0, 2 * np.pi, n_views))
    R = rotation(rng)
    for k in range(4):
        views[:, 3 * k:3 * k + 3] = views[:, 3 * k:3 * k + 3] @ R.T
    off = tuple(rng.uniform(-0.2, 0.2, 3) * n * vox)
    g = synth.Geometry(int(n[0]), int(n[1]), int(n[2]), *vox, int(nu), int(nv), views,
                       float(0.5 * vox.min()), off)
    mu = f32(smooth_volume(g, rng, n_blobs=5, sigma=(0.15 * ext, 0.3 * ext)))
    n_pose = int(rng.integers(1, 4))
    poses = f32(np.concatenate([rng.normal(0, 0.1 * ext, (n_pose, 3)),
                                rng.normal(0, 0.4, (n_pose, 3))], axis=1))
    iv = np.tile(np.arange(n_views), n_pose).astype(np.int32)
    ip = np.repeat(np.arange(n_pose), n_views).astype(np.int32)
    return g, mu, poses, iv, ip, rng


@pytest.mark.parametrize("seed", range(48))
def test_random_geometry_against_the_oracle(seed):
    g, mu, poses, iv, ip, rng = random_case(seed)
    P = pb.Projector(g, n_pose=len(poses), inst_view=iv, inst_pose=ip)
    P.set_volume(mu)
    ni = len(iv)
    # forward projection
    ref = oracle.forward(g, mu, poses, iv, ip)
    proj = P.forward(poses).cpu().numpy()
    if np.linalg.norm(ref) > 0:
        assert rel(proj, ref) <= TOL_IMG
    else:
        assert np.all(proj == 0)
    # fused pose gradient of a residual
    w = f32(rng.standard_normal((ni, g.nv, g.nu)))
    gth, _ = oracle.forward_grad(g, mu, poses, w, iv, ip, mode=oracle.GRAD_ANALYTIC)
    grad = P.forward_pose_grad(poses, pb.PROJ_LOSS_RESIDUAL, w)[0].cpu().numpy()
    for p in range(len(poses)):
        assert grad_ok(grad[p], gth[p]), (seed, p, grad[p], gth[p])
    # FDK-weighted back-projection and its pose gradient
    img = f32(rng.uniform(0, 1, (ni, g.nv, g.nu)))
    vref = oracle.back(g, img, poses, iv, ip, weight=oracle.W_FDK)
    vol = P.back(img, poses, pb.PROJ_W_FDK).cpu().numpy()
    if np.linalg.norm(vref) > 0:
        assert rel(vol, vref) <= TOL_IMG
    wv = f32(rng.standard_normal(g.vol_shape))
    gb, _ = oracle.back_grad(g, img, poses, wv, iv, ip, weight=oracle.W_NONE, mode=oracle.GRAD_ANALYTIC)
    gbg = P.back_pose_grad(img, poses, wv, pb.PROJ_W_NONE).cpu().numpy()
    for p in range(len(poses)):
        assert grad_ok(gbg[p], gb[p]), (seed, p, gbg[p], gb[p])
    # both transposes: <A mu, y> = <mu, A^T y>, <B img, x> = <img, B^T x>
    at = P.forward_adjoint(w, poses).cpu().numpy()
    assert abs(np.vdot(proj, w) - np.vdot(mu, at)) <= 1e-5 * np.linalg.norm(proj) * np.linalg.norm(w) + 1e-12
    bt = P.back_adjoint(wv, poses, pb.PROJ_W_FDK).cpu().numpy()
    assert abs(np.vdot(vol, wv) - np.vdot(img, bt)) <= 1e-5 * np.linalg.norm(vol) * np.linalg.norm(wv) + 1e-12

"""The allocation-free forward pose gradient.

Some callers cannot allocate device memory at all (a plug-in whose host
application owns every allocation, a real-time loop with memory frozen
after start-up, a caller whose allocator is not CUDA's).  For them the
library has proj_forward_pose_grad_static: no plan, no workspace, its
scratch in one static device array.  These tests check that it gives the
same gradient as the plan-based entry point on two calls in a row, and that
sizes beyond its static limit are refused with a clear message.  This file
is collected last on purpose."""
import numpy as np
import pytest

import paper_2508_13304_b300 as pb
from helpers import small_geom, smooth_volume

TOL_GRAD = 1e-3


def case():
    rng = np.random.default_rng(404)
    g = small_geom(n=(40, 36, 44), vox=(1.0, 1.1, 0.9), det=(50, 37), pix=1.6, n_views=3,
                   off=(1.5, -0.7, 0.4), step=0.5)
    mu = smooth_volume(g, rng, n_blobs=8).astype(np.float32)
    poses = np.concatenate([rng.uniform(-3, 3, (2, 3)), rng.uniform(-0.15, 0.15, (2, 3))], axis=1).astype(np.float32)
    inst_view = np.array([0, 1, 2, 0, 2], dtype=np.int32)
    inst_pose = np.array([0, 0, 0, 1, 1], dtype=np.int32)
    target = rng.uniform(0, 1, (3, g.nv, g.nu)).astype(np.float32)
    return g, mu, poses, inst_view, inst_pose, target


def grad_rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1, 6)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 6)
    worst = 0.0
    for p in range(b.shape[0]):
        for blk in (slice(0, 3), slice(3, 6)):
            worst = max(worst, np.linalg.norm(a[p, blk] - b[p, blk]) / np.linalg.norm(b[p, blk]))
    return worst


@pytest.mark.gpu
@pytest.mark.parametrize("loss", [pb.PROJ_LOSS_L2, pb.PROJ_LOSS_NCC])
def test_static_entry_point_matches_the_plan_based_one(loss):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()
    g, mu, poses, iv, ip, target = case()
    dev = torch.device("cuda", torch.cuda.current_device())
    mu_d = torch.from_numpy(mu).to(dev)
    pose_d = torch.from_numpy(poses).to(dev)
    target_d = torch.from_numpy(target).to(dev)

    P = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(mu_d)
    ref_grad, ref_loss = P.forward_pose_grad(pose_d, loss, target_d)
    ref_grad = ref_grad.cpu().numpy()

    for _ in range(2):                      # two calls in a row share the static scratch
        grad = torch.full((2, 6), float("nan"), device=dev)
        lossv = torch.full((2,), float("nan"), device=dev)
        pb.proj_forward_pose_grad_static(g, 2, iv, ip, mu_d, pose_d, loss, target_d, grad, lossv)
        torch.cuda.synchronize()
        assert grad_rel(grad.cpu().numpy(), ref_grad) <= TOL_GRAD
        np.testing.assert_allclose(lossv.cpu().numpy(), ref_loss.cpu().numpy(), rtol=1e-5)


@pytest.mark.gpu
def test_static_entry_point_at_its_size_limits():
    """A 64^3 volume (pitched (mu, grad mu) volume of exactly 74 x 70 x 68),
    64 views, 64 poses and 64 instances on a 128^2 detector (64 x 64 = 4096
    ray tiles): every region of the static scratch is used up to its end."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()
    rng = np.random.default_rng(405)
    g = small_geom(n=(64, 64, 64), vox=(1.0, 1.0, 1.0), det=(128, 128), pix=1.0, n_views=64, step=0.5,
                   sad=300.0, sdd=450.0)
    mu = smooth_volume(g, rng, n_blobs=10).astype(np.float32)
    n = 64
    poses = np.concatenate([rng.uniform(-4, 4, (n, 3)), rng.uniform(-0.2, 0.2, (n, 3))], axis=1).astype(np.float32)
    iv = np.arange(n, dtype=np.int32)
    ip = rng.permutation(n).astype(np.int32)
    target = rng.uniform(0, 1, (n, g.nv, g.nu)).astype(np.float32)
    dev = torch.device("cuda", torch.cuda.current_device())
    mu_d, pose_d, target_d = (torch.from_numpy(a).to(dev) for a in (mu, poses, target))
    P = pb.Projector(g, n_pose=n, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(mu_d)
    ref_grad, ref_loss = P.forward_pose_grad(pose_d, pb.PROJ_LOSS_L2, target_d)
    for _ in range(2):
        grad = torch.full((n, 6), float("nan"), device=dev)
        lossv = torch.full((n,), float("nan"), device=dev)
        pb.proj_forward_pose_grad_static(g, n, iv, ip, mu_d, pose_d, pb.PROJ_LOSS_L2, target_d, grad, lossv)
        torch.cuda.synchronize()
        assert grad_rel(grad.cpu().numpy(), ref_grad.cpu().numpy()) <= TOL_GRAD
        np.testing.assert_allclose(lossv.cpu().numpy(), ref_loss.cpu().numpy(), rtol=1e-5)


@pytest.mark.gpu
def test_static_entry_point_refuses_a_capturing_stream():
    """Its host tables are copied from memory that lives only for the call,
    so capturing it into a CUDA graph is refused before anything is
    enqueued; the next uncaptured call works."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()
    g, mu, poses, iv, ip, target = case()
    dev = torch.device("cuda", torch.cuda.current_device())
    mu_d, pose_d, target_d = (torch.from_numpy(a).to(dev) for a in (mu, poses, target))
    grad = torch.zeros((2, 6), device=dev)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        with pytest.raises(pb.ProjError) as info:
            pb.proj_forward_pose_grad_static(g, 2, iv, ip, mu_d, pose_d, pb.PROJ_LOSS_L2, target_d, grad)
    assert info.value.code == pb.PROJ_E_ARG and "capturing" in str(info.value)
    pb.proj_forward_pose_grad_static(g, 2, iv, ip, mu_d, pose_d, pb.PROJ_LOSS_L2, target_d, grad)
    torch.cuda.synchronize()
    assert torch.isfinite(grad).all() and grad.abs().sum() > 0


def test_sizes_beyond_the_static_limit_are_refused():
    from paper_2508_13304_b300 import build
    build.build()
    g = small_geom(n=(70, 70, 70), det=(16, 16), n_views=2)
    ctype, views = pb.make_geometry(g)
    iv = np.array([0, 1], dtype=np.int32)
    ip = np.array([0, 0], dtype=np.int32)
    import ctypes
    one = ctypes.c_void_p(256)              # never dereferenced: the size check comes first
    rc = pb.lib().proj_forward_pose_grad_static(
        ctypes.byref(ctype), 1, 2, iv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        ip.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), one, one, pb.PROJ_LOSS_L2, one, one, None, None)
    assert rc == pb.PROJ_E_ARG
    assert "static scratch limit" in pb.proj_last_error()
    g2 = small_geom(n=(20, 20, 20), det=(16, 16), n_views=2)
    ctype2, views2 = pb.make_geometry(g2)
    iv2 = np.zeros(65, dtype=np.int32)
    ip2 = np.zeros(65, dtype=np.int32)
    rc = pb.lib().proj_forward_pose_grad_static(
        ctypes.byref(ctype2), 1, 65, iv2.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        ip2.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), one, one, pb.PROJ_LOSS_L2, one, one, None, None)
    assert rc == pb.PROJ_E_ARG and "n_inst 65 exceeds the static scratch limit of 64" in pb.proj_last_error()

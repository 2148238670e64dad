"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded
inputs.  Bars: projections and back-projections rel-L2 <= 1e-4; pose
gradients rel <= 1e-3 per pose, on the translation and rotation blocks
separately (the units differ: 1/mm and 1/rad)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import small_geom, smooth_volume

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


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def grad_rel(g_gpu, g_ref):
    """Worst relative error over poses and over the two blocks."""
    g_gpu = np.asarray(g_gpu, dtype=np.float64).reshape(-1, 6)
    g_ref = np.asarray(g_ref, dtype=np.float64).reshape(-1, 6)
    worst = 0.0
    for p in range(g_ref.shape[0]):
        for blk in (slice(0, 3), slice(3, 6)):
            worst = max(worst, rel_l2(g_gpu[p, blk], g_ref[p, blk]))
    return worst


def np32(t):
    return t.detach().cpu().numpy().astype(np.float64)


def f32(a):
    """Round an input to FP32 once so both sides see the same numbers."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


# --------------------------------------------------------------- small ragged

# two ragged grids: even and odd slice counts (the volume copies store z slices
# in pairs), detector sizes that are not multiples of the 16-pixel tile
RAGGED = {"even_z": ((40, 36, 44), (50, 37)), "odd_z": ((37, 42, 33), (41, 46))}


def ragged_case(seed=101, shape="even_z"):
    rng = np.random.default_rng(seed)
    n, det = RAGGED[shape]
    g = small_geom(n=n, vox=(1.0, 1.1, 0.9), det=det, pix=1.6, n_views=3,
                   off=(1.5, -0.7, 0.4), step=0.5)
    mu = f32(smooth_volume(g, rng, n_blobs=8) + 0.3 * (rng.uniform(0, 1, g.vol_shape) > 0.97))
    poses = f32(np.concatenate([rng.uniform(-3, 3, (2, 3)), rng.uniform(-0.15, 0.15, (2, 3))], axis=1))
    inst_view = np.array([0, 1, 2, 0, 2], dtype=np.int32)
    inst_pose = np.array([0, 0, 0, 1, 1], dtype=np.int32)
    return g, mu, poses, inst_view, inst_pose, rng


@pytest.fixture(scope="module", params=sorted(RAGGED))
def ragged(request):
    g, mu, poses, iv, ip, rng = ragged_case(shape=request.param)
    P = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip)
    P.set_volume(mu)
    return dict(g=g, mu=mu, poses=poses, iv=iv, ip=ip, rng=rng, P=P)


def test_forward_ragged(ragged):
    d = ragged
    ref, ns = oracle.forward(d["g"], d["mu"], d["poses"], d["iv"], d["ip"], return_samples=True)
    got = np32(d["P"].forward(d["poses"]))
    assert rel_l2(got, ref) <= TOL_IMG
    cnt = np32(d["P"].count_samples(d["poses"]))
    np.testing.assert_allclose(cnt, ns, rtol=5e-3)


@pytest.mark.parametrize("loss", ["residual", "l2", "ncc"])
def test_forward_pose_grad_ragged(ragged, loss):
    d = ragged
    g, mu, poses, iv, ip = d["g"], d["mu"], d["poses"], d["iv"], d["ip"]
    rng = np.random.default_rng(7)
    proj_ref = oracle.forward(g, mu, poses, iv, ip)
    if loss == "residual":
        w = f32(rng.standard_normal(proj_ref.shape))
        ref_in, mode = w, pb.PROJ_LOSS_RESIDUAL
        L_ref = np.zeros(2)
    else:
        target = f32(oracle.forward(g, mu, f32([[1.0, -1.0, 0.5, 0.05, -0.02, 0.03]]), inst_view=[0, 1, 2],
                                    inst_pose=[0, 0, 0]))
        ref_in = target
        mode = pb.PROJ_LOSS_L2 if loss == "l2" else pb.PROJ_LOSS_NCC
        L_ref, w = oracle.pose_loss_weights(loss, proj_ref, target, iv, ip, 2)
    gth, _ = oracle.forward_grad(g, mu, poses, w, iv, ip, mode=oracle.GRAD_ANALYTIC)
    grad, L, proj = d["P"].forward_pose_grad(poses, mode, ref_in, want_proj=True)
    assert rel_l2(np32(proj), proj_ref) <= TOL_IMG
    assert grad_rel(np32(grad), gth) <= TOL_GRAD, (np32(grad), gth)
    if loss != "residual":
        np.testing.assert_allclose(np32(L), L_ref, rtol=1e-4)


@pytest.mark.parametrize("width", [2, 8, 16])
def test_forward_pose_grad_warp_shapes(ragged, width):
    """Every ray-tile shape of the fused march meets the parity bars and
    agrees with the default shape to FP32 rounding of the tile sums."""
    d = ragged
    g, mu, poses, iv, ip = d["g"], d["mu"], d["poses"], d["iv"], d["ip"]
    target = f32(oracle.forward(g, mu, f32([[1.0, -1.0, 0.5, 0.05, -0.02, 0.03]]), inst_view=[0, 1, 2],
                                inst_pose=[0, 0, 0]))
    proj_ref = oracle.forward(g, mu, poses, iv, ip)
    L_ref, w = oracle.pose_loss_weights("ncc", proj_ref, target, iv, ip, 2)
    gth, _ = oracle.forward_grad(g, mu, poses, w, iv, ip, mode=oracle.GRAD_ANALYTIC)
    P = d["P"]
    base, _ = P.forward_pose_grad(poses, pb.PROJ_LOSS_NCC, target)
    pb.proj_set_warp_shape(P.plan, width)
    try:
        assert pb.proj_get_warp_shape(P.plan) == width
        grad, L = P.forward_pose_grad(poses, pb.PROJ_LOSS_NCC, target)
    finally:
        pb.proj_set_warp_shape(P.plan, 4)
    assert grad_rel(np32(grad), gth) <= TOL_GRAD
    assert grad_rel(np32(grad), np32(base)) <= 1e-5
    np.testing.assert_allclose(np32(L), L_ref, rtol=1e-4)
    with pytest.raises(pb.ProjError):
        pb.proj_set_warp_shape(P.plan, 3)


def test_autotune_picks_a_shape_and_keeps_results(ragged):
    d = ragged
    P = pb.Projector(d["g"], n_pose=2, inst_view=d["iv"], inst_pose=d["ip"], ops=pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(d["mu"])
    target = f32(oracle.forward(d["g"], d["mu"], np.zeros(6), inst_view=[0, 1, 2], inst_pose=[0, 0, 0]))
    base, _ = P.forward_pose_grad(d["poses"], pb.PROJ_LOSS_L2, target)
    width, times = P.autotune(d["poses"], pb.PROJ_LOSS_L2, target, reps=2)
    assert width in pb.WARP_WIDTHS and pb.proj_get_warp_shape(P.plan) == width
    assert all(t > 0 for t in times.values()) and times[width] == min(times.values())
    grad, _ = P.forward_pose_grad(d["poses"], pb.PROJ_LOSS_L2, target)
    assert grad_rel(np32(grad), np32(base)) <= 1e-5


@pytest.mark.parametrize("shape", range(len(pb.BRICK_SHAPES)))
def test_back_pose_grad_brick_shapes(ragged, shape):
    d = ragged
    g = d["g"]
    rng = np.random.default_rng(16)
    img = f32(oracle.forward(g, d["mu"], np.zeros(6), d["iv"], np.zeros(5, dtype=np.int32))
              + 0.05 * rng.uniform(0, 1, (5, g.nv, g.nu)))
    wvol = f32(rng.standard_normal(g.vol_shape))
    gth, _ = oracle.back_grad(g, img, d["poses"], wvol, d["iv"], d["ip"], weight=pb.PROJ_W_FDK,
                              mode=oracle.GRAD_ANALYTIC)
    P = pb.Projector(g, n_pose=2, inst_view=d["iv"], inst_pose=d["ip"], ops=pb.PROJ_OP_BACK_GRAD)
    pb.proj_set_brick_shape(P.plan, shape)
    assert pb.proj_get_brick_shape(P.plan) == shape
    got = np32(P.back_pose_grad(img, d["poses"], wvol, pb.PROJ_W_FDK))
    assert grad_rel(got, gth) <= TOL_GRAD, (shape, got, gth)


def test_brick_autotune_picks_a_shape_and_keeps_results(ragged):
    d = ragged
    g = d["g"]
    rng = np.random.default_rng(17)
    img = f32(rng.uniform(0, 1, (5, g.nv, g.nu)))
    wvol = f32(rng.standard_normal(g.vol_shape))
    P = pb.Projector(g, n_pose=2, inst_view=d["iv"], inst_pose=d["ip"], ops=pb.PROJ_OP_BACK_GRAD)
    base = np32(P.back_pose_grad(img, d["poses"], wvol, pb.PROJ_W_FDK))
    shape, times = P.autotune_back(img, d["poses"], wvol, pb.PROJ_W_FDK, reps=2)
    assert shape in range(len(pb.BRICK_SHAPES)) and pb.proj_get_brick_shape(P.plan) == shape
    assert all(t > 0 for t in times.values()) and times[shape] == min(times.values())
    got = np32(P.back_pose_grad(img, d["poses"], wvol, pb.PROJ_W_FDK))
    assert grad_rel(got, base) <= 1e-5
    with pytest.raises(pb.ProjError):
        pb.proj_set_brick_shape(P.plan, len(pb.BRICK_SHAPES))


def test_forward_pose_grad_is_deterministic(ragged):
    d = ragged
    w = f32(np.random.default_rng(3).standard_normal((5, d["g"].nv, d["g"].nu)))
    a = np32(d["P"].forward_pose_grad(d["poses"], pb.PROJ_LOSS_RESIDUAL, w)[0])
    b = np32(d["P"].forward_pose_grad(d["poses"], pb.PROJ_LOSS_RESIDUAL, w)[0])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("weight", [pb.PROJ_W_NONE, pb.PROJ_W_FDK])
def test_back_ragged(ragged, weight):
    d = ragged
    rng = np.random.default_rng(5)
    img = f32(rng.uniform(0, 1, (5, d["g"].nv, d["g"].nu)))
    ref = oracle.back(d["g"], img, d["poses"], d["iv"], d["ip"], weight=weight)
    got = np32(d["P"].back(img, d["poses"], weight))
    assert rel_l2(got, ref) <= TOL_IMG


@pytest.mark.parametrize("weight", [pb.PROJ_W_NONE, pb.PROJ_W_FDK, pb.PROJ_W_FDK_CONST])
def test_back_pose_grad_ragged(ragged, weight):
    d = ragged
    g = d["g"]
    rng = np.random.default_rng(6)
    img = f32(oracle.forward(g, d["mu"], np.zeros(6), d["iv"], np.zeros(5, dtype=np.int32))
              + 0.05 * rng.uniform(0, 1, (5, g.nv, g.nu)))
    wvol = f32(rng.standard_normal(g.vol_shape))
    gth, _ = oracle.back_grad(g, img, d["poses"], wvol, d["iv"], d["ip"], weight=weight,
                              mode=oracle.GRAD_ANALYTIC)
    got = np32(d["P"].back_pose_grad(img, d["poses"], wvol, weight))
    assert grad_rel(got, gth) <= TOL_GRAD, (got, gth)


def test_forward_adjoint_ragged(ragged):
    d = ragged
    g = d["g"]
    y = f32(np.random.default_rng(8).standard_normal((5, g.nv, g.nu)))
    ref = oracle.forward_adjoint(g, y, d["poses"], d["iv"], d["ip"])
    got = np32(d["P"].forward_adjoint(y, d["poses"]))
    assert rel_l2(got, ref) <= TOL_IMG
    # adjoint identity on the GPU pair itself
    x = f32(np.random.default_rng(9).standard_normal(g.vol_shape))
    P2 = pb.Projector(g, n_pose=2, inst_view=d["iv"], inst_pose=d["ip"])
    P2.set_volume(x)
    ax = np32(P2.forward(d["poses"]))
    assert abs(np.sum(ax * y) - np.sum(x * got)) <= 1e-4 * np.linalg.norm(ax) * np.linalg.norm(y)


@pytest.mark.parametrize("weight", [pb.PROJ_W_NONE, pb.PROJ_W_FDK])
def test_back_adjoint_ragged(ragged, weight):
    d = ragged
    g = d["g"]
    x = f32(np.random.default_rng(10).standard_normal(g.vol_shape))
    ref = oracle.back_adjoint(g, x, d["poses"], d["iv"], d["ip"], weight=weight)
    got = np32(d["P"].back_adjoint(x, d["poses"], weight))
    assert rel_l2(got, ref) <= TOL_IMG


# --------------------------------------------------------------- edge cases

def test_non_finite_pose_sets_status_and_zero_gradient(ragged):
    d = ragged
    poses = d["poses"].copy()
    poses[1, 4] = np.nan
    w = np.ones((5, d["g"].nv, d["g"].nu))
    grad = np32(d["P"].forward_pose_grad(poses, pb.PROJ_LOSS_RESIDUAL, w)[0])
    assert d["P"].check() == pb.PROJ_STATUS_BAD_POSE
    assert np.all(grad[1] == 0) and np.all(np.isfinite(grad[0])) and np.any(grad[0] != 0)
    assert d["P"].check() == 0
    proj = np32(d["P"].forward(poses))
    assert np.all(proj[3:] == 0) and np.all(np.isfinite(proj))
    d["P"].check()


def test_rays_that_miss_give_zero(ragged):
    d = ragged
    far = np.array([[500.0, 0, 0, 0, 0, 0], [0, 0, 900.0, 0, 0, 0]])
    proj = np32(d["P"].forward(far))
    assert np.all(proj == 0)
    grad = np32(d["P"].forward_pose_grad(far, pb.PROJ_LOSS_RESIDUAL, np.ones((5, d["g"].nv, d["g"].nu)))[0])
    assert np.all(grad == 0)


def test_single_voxel_single_pixel():
    mu = np.zeros((1, 1, 1))
    mu[0, 0, 0] = 2.0
    view = np.array([[-300.0, 0.1, -0.2, 200.0, 0.1, -0.2, 0, 1.0, 0, 0, 0, 1.0]])
    g = synth.Geometry(1, 1, 1, 1.0, 1.0, 1.0, 1, 1, view, 0.25)
    P = pb.Projector(g)
    P.set_volume(mu)
    pose = np.array([[0.05, 0.0, 0.0, 0.0, 0.01, 0.0]])
    ref = oracle.forward(g, mu, pose)
    assert rel_l2(np32(P.forward(pose)), ref) <= TOL_IMG
    img = np.full((1, 1, 1), 3.0)
    assert rel_l2(np32(P.back(img, pose)), oracle.back(g, img, pose)) <= TOL_IMG


def test_source_inside_the_volume():
    """A degenerate geometry: the source sits inside the volume (10 mm from
    the isocentre of a 40 mm grid).  Rays start at the source (sample k = 0);
    voxels behind the source (w' <= 0) receive nothing from the
    back-projector.  Every call against the oracle."""
    rng = np.random.default_rng(21)
    g = small_geom(n=(40, 38, 36), vox=(1.0, 1.0, 1.0), det=(45, 40), pix=2.5, n_views=2, sad=10.0, sdd=60.0)
    mu = f32(smooth_volume(g, rng, n_blobs=6))
    poses = f32([[0.5, -0.3, 0.2, 0.02, -0.03, 0.01]])
    P = pb.Projector(g)
    P.set_volume(mu)
    ref = oracle.forward(g, mu, poses)
    assert rel_l2(np32(P.forward(poses)), ref) <= TOL_IMG
    w = f32(rng.standard_normal(ref.shape))
    gth, _ = oracle.forward_grad(g, mu, poses, w, mode=oracle.GRAD_ANALYTIC)
    assert grad_rel(np32(P.forward_pose_grad(poses, pb.PROJ_LOSS_RESIDUAL, w)[0]), gth) <= TOL_GRAD
    img = f32(rng.uniform(0, 1, ref.shape))
    for weight in (pb.PROJ_W_NONE, pb.PROJ_W_FDK):
        vref = oracle.back(g, img, poses, weight=weight)
        assert np.any(vref == 0) and np.any(vref != 0)       # some voxels lie behind the source
        assert rel_l2(np32(P.back(img, poses, weight)), vref) <= TOL_IMG
    wv = f32(rng.standard_normal(g.vol_shape))
    gb, _ = oracle.back_grad(g, img, poses, wv, weight=pb.PROJ_W_NONE, mode=oracle.GRAD_ANALYTIC)
    assert grad_rel(np32(P.back_pose_grad(img, poses, wv, pb.PROJ_W_NONE)), gb) <= TOL_GRAD


# --------------------------------------------------------------- C1 (64^3) full

@pytest.fixture(scope="module")
def tiny():
    w = synth.workload_tiny()
    w["mu"] = f32(w["mu"])
    w["pose"] = f32(w["pose"])
    w["pose_true"] = f32(w["pose_true"])
    P = pb.Projector(w["geom"])
    P.set_volume(w["mu"])
    w["P"] = P
    return w


def test_tiny_forward_and_l2_gradient(tiny):
    g, mu = tiny["geom"], tiny["mu"]
    target = f32(oracle.forward(g, mu, tiny["pose_true"]))
    proj_ref = oracle.forward(g, mu, tiny["pose"])
    assert rel_l2(np32(tiny["P"].forward(tiny["pose"])), proj_ref) <= TOL_IMG
    L_ref, w = oracle.pose_loss_weights("l2", proj_ref, target, np.arange(8), np.zeros(8, dtype=int), 1)
    gth, _ = oracle.forward_grad(g, mu, tiny["pose"], w)
    grad, L = tiny["P"].forward_pose_grad(tiny["pose"], pb.PROJ_LOSS_L2, target)
    assert grad_rel(np32(grad), gth) <= TOL_GRAD
    np.testing.assert_allclose(np32(L), L_ref, rtol=1e-4)


def test_tiny_back_and_gradient(tiny):
    g = tiny["geom"]
    img = f32(tiny["det_image"])
    ref = oracle.back(g, img, tiny["pose"])
    assert rel_l2(np32(tiny["P"].back(img, tiny["pose"])), ref) <= TOL_IMG
    target = oracle.back(g, img, np.zeros(6))
    _, wvol = oracle.l2_loss(ref, target)
    wvol = f32(wvol)
    gth, _ = oracle.back_grad(g, img, tiny["pose"], wvol)
    got = np32(tiny["P"].back_pose_grad(img, tiny["pose"], wvol))
    assert grad_rel(got, gth) <= TOL_GRAD


def test_yfast_volume_copy_gives_identical_results():
    """Instances whose detector u axis is closer to y than to x march the
    copy of the (mu, grad mu) volume with y fastest; the values and the
    arithmetic are the same, so the results equal those of the static entry
    point, which marches the x-fast volume for every instance, bit for bit.
    Views at 0, 45+1 and 90 deg cover both layouts."""
    rng = np.random.default_rng(17)
    views = synth.circular_views(3, 200.0, 320.0, 1.6, 1.6, angles=[0.0, np.radians(46.0), np.pi / 2])
    g = synth.Geometry(40, 36, 44, 1.0, 1.1, 0.9, 50, 37, views, 0.5, (1.5, -0.7, 0.4))
    mu = f32(smooth_volume(g, rng, n_blobs=8))
    poses = f32(np.concatenate([rng.uniform(-3, 3, (2, 3)), rng.uniform(-0.15, 0.15, (2, 3))], axis=1))
    iv = np.array([0, 1, 2, 0, 2], dtype=np.int32)
    ip = np.array([0, 0, 0, 1, 1], dtype=np.int32)
    target = torch.from_numpy(rng.uniform(0, 1, (3, g.nv, g.nu)).astype(np.float32)).cuda()
    mu_d = torch.from_numpy(mu.astype(np.float32)).cuda()
    pose_d = torch.from_numpy(poses.astype(np.float32)).cuda()
    P = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(mu_d)
    for loss in (pb.PROJ_LOSS_L2, pb.PROJ_LOSS_NCC):
        grad, L = P.forward_pose_grad(pose_d, loss, target)
        g2 = torch.empty((2, 6), device="cuda")
        L2 = torch.empty((2,), device="cuda")
        pb.proj_forward_pose_grad_static(g, 2, iv, ip, mu_d, pose_d, loss, target, g2, L2)
        torch.cuda.synchronize()
        assert torch.equal(grad, g2), (grad, g2)
        assert torch.equal(L, L2)


def test_one_copy_plan_gives_identical_results(ragged):
    """PROJ_FLAG_ONE_COPY keeps only the rows-along-x copies of the prepared
    volume: a smaller workspace and the same projections and pose gradients
    bit for bit (the instances whose u axis runs along y march the x copy)."""
    d = ragged
    g, mu, poses, iv, ip = d["g"], d["mu"], d["poses"], d["iv"], d["ip"]
    target = f32(oracle.forward(g, mu, f32([[1.0, -1.0, 0.5, 0.05, -0.02, 0.03]]), inst_view=[0, 1, 2],
                                inst_pose=[0, 0, 0]))
    ops = pb.PROJ_OP_FORWARD | pb.PROJ_OP_FORWARD_GRAD
    P2 = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=ops)
    P1 = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=ops | pb.PROJ_FLAG_ONE_COPY)
    assert pb.proj_workspace_size(P1.plan) < pb.proj_workspace_size(P2.plan)
    for P in (P1, P2):
        P.set_volume(mu)
    for loss in (pb.PROJ_LOSS_L2, pb.PROJ_LOSS_NCC):
        g1, l1 = P1.forward_pose_grad(poses, loss, target)
        g2, l2 = P2.forward_pose_grad(poses, loss, target)
        np.testing.assert_array_equal(np32(g1), np32(g2))
        np.testing.assert_array_equal(np32(l1), np32(l2))
    np.testing.assert_array_equal(np32(P1.forward(poses)), np32(P2.forward(poses)))
    assert rel_l2(np32(P1.forward(poses)), oracle.forward(g, mu, poses, iv, ip)) <= TOL_IMG


@pytest.mark.parametrize("edge", [0, 8])
def test_bricked_plan_gives_identical_results(ragged, edge):
    """PROJ_FLAG_BRICKS marches a copy of the prepared volume stored in 4^3-cell
    bricks with a one-element apron: the same corner values and fractions in
    the same order, so pose gradients, losses, projections and pose-list calls
    equal the row-layout plan's bit for bit, with and without skipping, and
    the gradients stay within the oracle bars."""
    d = ragged
    g, mu, poses, iv, ip = d["g"], d["mu"], d["poses"], d["iv"], d["ip"]
    target = f32(oracle.forward(g, mu, f32([[1.0, -1.0, 0.5, 0.05, -0.02, 0.03]]), inst_view=[0, 1, 2],
                                inst_pose=[0, 0, 0]))
    ops = pb.PROJ_OP_FORWARD | pb.PROJ_OP_FORWARD_GRAD
    P2 = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=ops)
    PB = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=ops | pb.PROJ_FLAG_BRICKS)
    for P in (PB, P2):
        pb.proj_set_skip_brick(P.plan, edge)
        P.set_volume(mu)
    resid = f32(np.random.default_rng(7).standard_normal((len(iv), g.nv, g.nu)))
    for loss, ref in ((pb.PROJ_LOSS_L2, target), (pb.PROJ_LOSS_NCC, target), (pb.PROJ_LOSS_RESIDUAL, resid)):
        gb, lb, pr_b = PB.forward_pose_grad(poses, loss, ref, want_proj=True)
        g2, l2, pr_2 = P2.forward_pose_grad(poses, loss, ref, want_proj=True)
        np.testing.assert_array_equal(np32(gb), np32(g2))
        np.testing.assert_array_equal(np32(lb), np32(l2))
        np.testing.assert_array_equal(np32(pr_b), np32(pr_2))
    # a pose list (second pose only) on the bricked plan
    pose_d = torch.from_numpy(np.asarray(poses, dtype=np.float32)).cuda()
    tgt = torch.from_numpy(np.asarray(target, dtype=np.float32)).cuda()
    gl = torch.zeros((2, 6), device="cuda")
    ll = torch.zeros((2,), device="cuda")
    pb.proj_forward_pose_grad_list(PB.plan, pose_d, torch.tensor([1], dtype=torch.int32, device="cuda"),
                                   pb.PROJ_LOSS_L2, tgt, gl, ll, None, PB.ws)
    g2, _ = P2.forward_pose_grad(poses, pb.PROJ_LOSS_L2, target)
    assert torch.equal(gl[1], g2[1].cuda())
    _, w = oracle.pose_loss_weights("l2", oracle.forward(g, mu, poses, iv, ip), target, iv, ip, 2)
    gref, _ = oracle.forward_grad(g, mu, poses, w, iv, ip, mode=oracle.GRAD_ANALYTIC)
    gb, _ = PB.forward_pose_grad(poses, pb.PROJ_LOSS_L2, target)
    for p in range(2):
        for blk in (slice(0, 3), slice(3, 6)):
            assert rel_l2(np32(gb)[p, blk], gref[p, blk]) <= TOL_GRAD

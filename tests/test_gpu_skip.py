"""Empty-space skipping of the forward marches (proj_set_skip_brick,
proj_set_skip_cells): each ray keeps only its samples around the occupied
bricks it crosses, and the fused march leaves out the samples whose cell has
no non-zero corner.  A sample left out reads eight zero corners, so
projections, losses and pose gradients must be bit-identical with skipping
off, with 8^3 and with 16^3 bricks, each with and without the cell test.  The
volumes here are sparse on purpose: small ellipsoids in air, single voxels
at the corners and faces of the grid (rays that graze a brick boundary),
one-voxel lines, random geometries turned off the grid axes."""
import numpy as np
import pytest

import oracle
import synth
from helpers import small_geom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()


import paper_2508_13304_b300 as pb  # noqa: E402

EDGES = (0, 8, 16)
MODES = [(e, c) for e in EDGES for c in (0, 1)] + [(8, 2)]   # (brick edge, cell test off / on / automatic)


def sparse_volume(g, rng, n_ell=3, n_dots=12):
    """A few small ellipsoids plus isolated voxels (corners, faces, random)
    and a one-voxel line: exact zeros everywhere else."""
    ext = np.array([g.nx * g.vx, g.ny * g.vy, g.nz * g.vz])
    ell = synth.random_ellipsoids(rng, n_ell, 0.15 * float(ext.min()),
                                  (0.04 * float(ext.min()), 0.12 * float(ext.min())), (0.01, 0.03))
    mu = synth.voxelise(g, ell).astype(np.float32)
    nx, ny, nz = g.nx, g.ny, g.nz
    for (i, j, k) in [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny - 1, nz // 2), (nx // 2, 0, nz - 1)]:
        mu[k, j, i] = 0.05
    for _ in range(n_dots):
        mu[rng.integers(nz), rng.integers(ny), rng.integers(nx)] = rng.uniform(0.01, 0.08)
    mu[rng.integers(nz), rng.integers(ny), :] += 0.02                       # a line along x
    return mu


def all_calls(P, g, poses, target, resid):
    out = {}
    out["proj"] = P.forward(poses).cpu().numpy()
    for name, loss, ref in (("l2", pb.PROJ_LOSS_L2, target), ("ncc", pb.PROJ_LOSS_NCC, target),
                            ("res", pb.PROJ_LOSS_RESIDUAL, resid)):
        gr, lo, pr = P.forward_pose_grad(poses, loss, ref, want_proj=True)
        out[name] = (gr.cpu().numpy(), lo.cpu().numpy(), pr.cpu().numpy())
    return out


def same(a, b):
    if isinstance(a, tuple):
        return all(same(x, y) for x, y in zip(a, b))
    return np.array_equal(a, b)


def check_exact(g, mu, poses, iv, ip, rng):
    target = rng.uniform(0, 0.2, (g.n_views, g.nv, g.nu)).astype(np.float32)
    resid = rng.standard_normal((len(iv), g.nv, g.nu)).astype(np.float32)
    P = pb.Projector(g, n_pose=len(poses), inst_view=iv, inst_pose=ip,
                     ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(mu)
    res, counts = {}, {}
    for e, c in MODES:
        pb.proj_set_skip_brick(P.plan, e)
        pb.proj_set_skip_cells(P.plan, c)
        assert pb.proj_get_skip_brick(P.plan) == e and pb.proj_get_skip_cells(P.plan) == c
        res[e, c] = all_calls(P, g, poses, target, resid)
        counts[e, c] = int(P.count_marched_samples(poses).sum().item())
    pb.proj_set_skip_brick(P.plan, 8)
    pb.proj_set_skip_cells(P.plan, pb.SKIP_CELLS_AUTO)
    base = (0, 0)
    for m in MODES[1:]:
        for k in res[base]:
            assert same(res[m][k], res[base][k]), (m, k)
    assert counts[8, 0] <= counts[16, 0] <= counts[0, 0]
    # the brick ranges hold every sample whose cell has a non-zero corner: the cell test counts the same
    assert counts[0, 1] == counts[8, 1] == counts[16, 1] <= counts[8, 0]
    assert counts[8, 2] in (counts[8, 0], counts[8, 1])
    out = {e: counts[e, 0] for e in EDGES} | {("cells", e): counts[e, 1] for e in EDGES}
    out["auto"] = counts[8, 2]
    res[base]["target"] = target
    return res[base], out


def test_sparse_phantom_exact_and_against_the_oracle():
    rng = np.random.default_rng(31)
    g = small_geom(n=(48, 40, 44), vox=(1.0, 1.1, 0.9), det=(52, 47), pix=1.4, n_views=3, off=(1.0, -0.5, 0.8))
    mu = sparse_volume(g, rng)
    poses = np.concatenate([rng.uniform(-3, 3, (2, 3)), rng.uniform(-0.3, 0.3, (2, 3))], axis=1).astype(np.float32)
    iv = np.array([0, 1, 2, 0, 2], dtype=np.int32)
    ip = np.array([0, 0, 0, 1, 1], dtype=np.int32)
    res, counts = check_exact(g, mu, poses, iv, ip, rng)
    assert counts[8] < 0.8 * counts[0]                 # the phantom leaves most samples in air
    ref = oracle.forward(g, mu.astype(np.float64), poses.astype(np.float64), iv, ip)
    assert np.linalg.norm(res["proj"] - ref) <= 1e-4 * np.linalg.norm(ref)
    # the pose gradients (equal in every skipping mode) against the oracle's analytic gradient
    target = res["target"].astype(np.float64)
    for kind in ("l2", "ncc"):
        _, w = oracle.pose_loss_weights(kind, ref, target, iv, ip, 2)
        gth, _ = oracle.forward_grad(g, mu.astype(np.float64), poses.astype(np.float64), w, iv, ip,
                                     mode=oracle.GRAD_ANALYTIC)
        got = res[kind][0].astype(np.float64)
        for p in range(2):
            for blk in (slice(0, 3), slice(3, 6)):
                assert np.linalg.norm(got[p, blk] - gth[p, blk]) <= 1e-3 * np.linalg.norm(gth[p, blk]), (kind, p)


@pytest.mark.parametrize("seed", range(16))
def test_random_sparse_geometries_exact(seed):
    rng = np.random.default_rng(500 + seed)
    n = rng.integers(8, 40, 3)
    vox = rng.uniform(0.6, 1.6, 3)
    ext = float(np.linalg.norm(n * vox))
    nu, nv = rng.integers(8, 48, 2)
    n_views = int(rng.integers(1, 4))
    sad = ext * rng.uniform(1.5, 4.0)
    sdd = sad * rng.uniform(1.2, 2.0)
    pix = 1.3 * ext * sdd / sad / max(nu, nv, 8)
    views = synth.circular_views(n_views, sad, sdd, pix, pix, angles=rng.uniform(0, 2 * np.pi, n_views))
    q = rng.standard_normal((3, 3))
    R, _ = np.linalg.qr(q)
    R *= np.sign(np.linalg.det(R))
    for k in range(4):
        views[:, 3 * k:3 * k + 3] = views[:, 3 * k:3 * k + 3] @ R.T
    g = synth.Geometry(int(n[0]), int(n[1]), int(n[2]), *vox, int(nu), int(nv), views, float(0.5 * vox.min()),
                       tuple(rng.uniform(-0.2, 0.2, 3) * n * vox))
    mu = sparse_volume(g, rng, n_ell=int(rng.integers(0, 3)), n_dots=int(rng.integers(1, 10)))
    n_pose = int(rng.integers(1, 4))
    poses = np.concatenate([rng.normal(0, 0.1 * ext, (n_pose, 3)), rng.normal(0, 0.4, (n_pose, 3))],
                           axis=1).astype(np.float32)
    iv = np.tile(np.arange(n_views), n_pose).astype(np.int32)
    ip = np.repeat(np.arange(n_pose), n_views).astype(np.int32)
    check_exact(g, mu, poses, iv, ip, rng)


def test_automatic_cell_test_follows_the_volume():
    """SKIP_CELLS_AUTO turns the cell test on for a volume with much empty
    space inside the occupied bricks and off for a nearly full one (an empty
    slab of 8 slices in a filled volume); results stay bit-identical."""
    rng = np.random.default_rng(17)
    g = small_geom(n=(40, 36, 44), det=(40, 38), n_views=2)
    poses = np.array([[1.0, -0.5, 0.3, 0.05, -0.04, 0.08]], dtype=np.float32)
    iv = np.arange(2, dtype=np.int32)
    ip = np.zeros(2, dtype=np.int32)
    _, sparse = check_exact(g, sparse_volume(g, rng), poses, iv, ip, rng)
    assert sparse["auto"] == sparse["cells", 8] < sparse[8]
    full = rng.uniform(0.01, 0.03, g.vol_shape).astype(np.float32)
    full[18:26] = 0.0
    _, dense = check_exact(g, full, poses, iv, ip, rng)
    assert dense["cells", 8] < dense[8]            # the slab's inner cells are empty ...
    assert dense["auto"] == dense[8]               # ... but too few for the automatic test


def test_skip_settings_reject_invalid_values():
    g = small_geom(n=(12, 10, 14), det=(16, 12), n_views=1)
    P = pb.Projector(g, n_pose=1, inst_view=np.zeros(1, np.int32), inst_pose=np.zeros(1, np.int32),
                     ops=pb.PROJ_OP_FORWARD_GRAD)
    L = pb.lib()
    for bad in (-1, 4, 9, 32):
        assert L.proj_set_skip_brick(P.plan.handle, bad) == pb.PROJ_E_ARG
    for bad in (-1, 3):
        assert L.proj_set_skip_cells(P.plan.handle, bad) == pb.PROJ_E_ARG
    assert pb.proj_get_skip_brick(P.plan) == 8 and pb.proj_get_skip_cells(P.plan) == pb.SKIP_CELLS_AUTO


def test_empty_volume_marches_nothing():
    rng = np.random.default_rng(3)
    g = small_geom(n=(20, 18, 22), det=(24, 20), n_views=2)
    mu = np.zeros(g.vol_shape, dtype=np.float32)
    poses = np.zeros((1, 6), dtype=np.float32)
    iv = np.arange(2, dtype=np.int32)
    ip = np.zeros(2, dtype=np.int32)
    res, counts = check_exact(g, mu, poses, iv, ip, rng)
    assert counts[8] == 0 and counts[16] == 0 and counts[0] > 0 and counts["cells", 0] == 0
    assert np.all(res["proj"] == 0) and np.all(res["res"][0] == 0)


def test_autotune_march_and_batch_with_skipping():
    """proj_autotune_march keeps a valid (brick edge, cell test, warp shape)
    with the same results; a persistent batch of sparse problems equals the
    per-plan calls and the unskipped march bit for bit."""
    rng = np.random.default_rng(41)
    probs = []
    for n, det in (((40, 36, 30), (44, 40)), ((28, 33, 25), (30, 26)), ((36, 36, 36), (38, 38))):
        g = small_geom(n=n, det=det, pix=1.5, n_views=2)
        mu = sparse_volume(g, rng)
        poses = np.concatenate([rng.uniform(-2, 2, (2, 3)), rng.uniform(-0.2, 0.2, (2, 3))], axis=1).astype(np.float32)
        iv = np.tile(np.arange(2), 2).astype(np.int32)
        ip = np.repeat(np.arange(2), 2).astype(np.int32)
        P = pb.Projector(g, n_pose=2, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD_GRAD)
        P.set_volume(mu)
        tgt = torch.from_numpy(rng.uniform(0, 0.2, (2, g.nv, g.nu)).astype(np.float32)).cuda()
        pose_d = torch.from_numpy(poses).cuda()
        probs.append((P, pose_d, tgt))
    P, pose_d, tgt = probs[0]
    base, _ = P.forward_pose_grad(pose_d, pb.PROJ_LOSS_NCC, tgt)
    w, e, c, times = pb.proj_autotune_march(P.plan, pose_d, pb.PROJ_LOSS_NCC, tgt, P.ws, reps=1)
    assert w in pb.WARP_WIDTHS and e in pb.SKIP_BRICK_EDGES and len(times) == 24
    assert all(t > 0 for t in times.values())
    assert pb.proj_get_skip_brick(P.plan) == e and pb.proj_get_warp_shape(P.plan) == w
    assert pb.proj_get_skip_cells(P.plan) == c
    pb.proj_set_warp_shape(P.plan, 4)
    for edge, cells in ((0, False), (16, True), (8, False), (8, True)):
        pb.proj_set_skip_brick(P.plan, edge)
        pb.proj_set_skip_cells(P.plan, cells)
        g2, _ = P.forward_pose_grad(pose_d, pb.PROJ_LOSS_NCC, tgt)
        assert torch.equal(g2, base)
    singles = [Q.forward_pose_grad(pq, pb.PROJ_LOSS_L2, tq)[0] for Q, pq, tq in probs]
    grads = [torch.empty((2, 6), device="cuda") for _ in probs]
    batch = pb.proj_batch_create([dict(plan=Q.plan, loss=pb.PROJ_LOSS_L2, pose=pq, ref=tq, grad=gr, ws=Q.ws)
                                  for (Q, pq, tq), gr in zip(probs, grads)])
    pb.proj_batch_run(batch)
    torch.cuda.synchronize()
    for a, b in zip(grads, singles):
        assert torch.equal(a, b)
    for Q, _, _ in probs:
        pb.proj_set_skip_brick(Q.plan, 0)
        pb.proj_set_skip_cells(Q.plan, pb.SKIP_CELLS_OFF)
    unskipped = [Q.forward_pose_grad(pq, pb.PROJ_LOSS_L2, tq)[0] for Q, pq, tq in probs]
    for a, b in zip(grads, unskipped):
        assert torch.equal(a, b)

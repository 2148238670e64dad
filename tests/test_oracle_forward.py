"""Pins of the oracle's ray-driven forward projector (Eq. forward,
Sec. II-C.1) and of its rigid-pose gradient (Eqs. for_grad, final_forward,
for_int, dis_forward) against results that do not come from the oracle:
analytic chord lengths, Gaussian line integrals, exact invariances, a
hand-derived single-voxel case, finite differences and the adjoint
identity."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import central_fd, euler_from_matrix, small_geom, smooth_volume

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def chord_length(o, d, centre, axes, semi):
    """Length of the chord of the line o + s d (|d| = 1) inside the
    ellipsoid {|diag(1/semi) axes^T (x - centre)| <= 1}: roots of a
    quadratic in s."""
    ot = (axes.T @ (o - centre)) / semi
    dt = (axes.T @ d) / semi
    A, B, C = dt @ dt, 2 * ot @ dt, ot @ ot - 1
    disc = B * B - 4 * A * C
    return np.sqrt(disc) / A if disc > 0 else 0.0


def pixel_rays(geom, vi):
    """Source and unit directions of every pixel ray of view vi."""
    vw = geom.views[vi]
    iu, iv = np.meshgrid(np.arange(geom.nu), np.arange(geom.nv))
    q = vw[3:6] + (iu[..., None] - (geom.nu - 1) / 2) * vw[6:9] \
        + (iv[..., None] - (geom.nv - 1) / 2) * vw[9:12]
    d = q - vw[0:3]
    return vw[0:3], d / np.linalg.norm(d, axis=-1, keepdims=True)


@pytest.mark.parametrize("supersample", [1])
def test_chord_lengths_of_moved_ellipsoids(supersample):
    """l = sum_e mu_e chord_e through the moved ellipsoids; the voxelisation
    error of an indicator is O(h): a few percent rel-L2 at 64^3 and about
    halved at 128^3."""
    rng = np.random.default_rng(7)
    ell = synth.random_ellipsoids(rng, 10, 10.0, (5.0, 18.0), (0.01, 0.03))
    pose = np.array([2.0, -3.0, 1.5, np.deg2rad(4), np.deg2rad(-3), np.deg2rad(2)])
    R, _ = oracle.rotation(pose)
    errs = []
    nd = 40
    views = synth.circular_views(3, 800.0, 1200.0, 3.5, 3.5)
    for n, v in [(64, 1.0), (128, 0.5)]:
        g = synth.Geometry(n, n, n, v, v, v, nd, nd, views, 0.5 * v)
        mu = synth.voxelise(g, ell, supersample=supersample)
        p = oracle.forward(g, mu, pose)
        ref = np.zeros_like(p)
        for vi in range(g.n_views):
            s, dirs = pixel_rays(g, vi)
            for iv in range(nd):
                for iu in range(nd):
                    ref[vi, iv, iu] = sum(
                        e.mu * chord_length(s, dirs[iv, iu], R @ e.centre + pose[:3],
                                            R @ e.axes, e.semi) for e in ell)
        errs.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
    assert errs[0] <= 3e-2, errs
    assert errs[0] / errs[1] >= 1.7, errs


def gaussian_line_integral(s, d, amp, c, sigma):
    """Integral of amp exp(-|x-c|^2/(2 sigma^2)) along the full line s + t d
    (|d| = 1): amp sigma sqrt(2 pi) exp(-dist^2 / (2 sigma^2))."""
    w = c - s
    along = w @ d
    dist2 = w @ w - along * along
    return amp * sigma * np.sqrt(2 * np.pi) * np.exp(-dist2 / (2 * sigma ** 2))


def blob_setup(n, v):
    views = synth.circular_views(3, 300.0, 450.0, 1.6, 1.6, angles=[0.3, 1.4, 2.6])
    g = synth.Geometry(n, n, n, v, v, v, 24, 24, views, 0.5 * v)
    blobs = [(1.0, np.array([3.0, -2.0, 1.0]), 7.0), (0.6, np.array([-6.0, 5.0, -4.0]), 6.0)]
    return g, blobs, synth.gaussian_blobs(g, blobs)


def test_gaussian_line_integrals_converge_quadratically():
    pose = np.array([1.5, -1.0, 2.0, 0.05, -0.08, 0.1])
    R, _ = oracle.rotation(pose)
    errs = []
    for n, v in [(48, 1.6), (96, 0.8)]:
        g, blobs, mu = blob_setup(n, v)
        p = oracle.forward(g, mu, pose)
        ref = np.zeros_like(p)
        for vi in range(g.n_views):
            s, dirs = pixel_rays(g, vi)
            for iv in range(g.nv):
                for iu in range(g.nu):
                    ref[vi, iv, iu] = sum(gaussian_line_integral(
                        s, dirs[iv, iu], a, R @ c + pose[:3], sg) for a, c, sg in blobs)
        errs.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
    assert errs[0] < 1e-2, errs
    assert errs[0] / errs[1] > 3.3, errs          # O(h^2): ideal ratio 4


def test_gaussian_pose_gradient_converges_to_closed_form():
    """For L = sum_i l_i the continuous gradient is the sum over rays of the
    derivative of the closed-form line integral as the blob centre moves to
    R c + t.  Both gradient modes approach it at O(h^2)."""
    pose = np.array([1.5, -1.0, 2.0, 0.05, -0.08, 0.1])
    R, dR = oracle.rotation(pose)
    errs = {0: [], 1: []}
    for n, v in [(48, 1.6), (96, 0.8)]:
        g, blobs, mu = blob_setup(n, v)
        ref = np.zeros(6)
        for vi in range(g.n_views):
            s, dirs = pixel_rays(g, vi)
            for iv in range(g.nv):
                for iu in range(g.nu):
                    d = dirs[iv, iu]
                    for a, c, sg in blobs:
                        cw = R @ c + pose[:3]
                        li = gaussian_line_integral(s, d, a, cw, sg)
                        w = cw - s
                        perp = w - (w @ d) * d
                        dl_dc = -li * perp / sg ** 2
                        ref[:3] += dl_dc
                        for j in range(3):
                            ref[3 + j] += dl_dc @ (dR[j] @ c)
        w = np.ones((g.n_views, g.nv, g.nu))
        for mode in (oracle.GRAD_ANALYTIC, oracle.GRAD_EXACT):
            gth, _ = oracle.forward_grad(g, mu, pose, w, mode=mode)
            errs[mode].append(np.linalg.norm(gth[0] - ref) / np.linalg.norm(ref))
    for mode in errs:
        assert errs[mode][0] < 2e-2, errs
        assert errs[mode][0] / errs[mode][1] > 3.0, errs


def test_single_voxel_tent_integrals():
    """One unit voxel at the centre of a 3^3 grid (1 mm voxels); single rays
    along +x at lateral offsets (dy, dz).  The trilinear interpolant is a
    tensor-product hat, and the step-0.5 Riemann sum of a unit hat is exactly
    its integral for any phase, so l = 1 mm * (1-|dy|)(1-|dz|)."""
    mu = np.zeros((3, 3, 3))
    mu[1, 1, 1] = 1.0
    for dy, dz, phase in [(0.0, 0.0, 0.0), (0.3, -0.2, 0.37), (-0.75, 0.5, 0.11), (0.0, 0.99, 0.25)]:
        view = np.array([-800.0 - phase, dy, dz, 400.0, dy, dz, 0, 1.0, 0, 0, 0, 1.0])
        g = synth.Geometry(3, 3, 3, 1.0, 1.0, 1.0, 1, 1, view[None, :], 0.5)
        p = oracle.forward(g, mu, np.zeros(6))
        assert abs(p[0, 0, 0] - (1 - abs(dy)) * (1 - abs(dz))) < 1e-12


def test_integer_voxel_translation_equals_shifted_array():
    rng = np.random.default_rng(11)
    g = small_geom()
    mu = np.zeros(g.vol_shape)
    mu[4:-4, 4:-4, 4:-4] = rng.uniform(0, 1, (g.nz - 8, g.ny - 8, g.nx - 8))
    shift = np.array([2, -1, 3])            # voxels along x, y, z
    t = shift * np.array([g.vx, g.vy, g.vz])
    moved = oracle.forward(g, mu, np.concatenate([t, np.zeros(3)]))
    shifted = np.roll(mu, (shift[2], shift[1], shift[0]), axis=(0, 1, 2))
    static = oracle.forward(g, shifted, np.zeros(6))
    np.testing.assert_allclose(moved, static, rtol=0, atol=1e-10 * np.abs(static).max())


def test_quarter_turn_about_z_equals_permuted_array():
    rng = np.random.default_rng(12)
    g = small_geom(n=(16, 16, 14), vox=(1.0, 1.0, 1.2))
    mu = np.zeros(g.vol_shape)
    mu[3:-3, 3:-3, 3:-3] = rng.uniform(0, 1, (g.nz - 6, g.ny - 6, g.nx - 6))
    moved = oracle.forward(g, mu, np.array([0, 0, 0, 0, 0, np.pi / 2]))
    # object point (x, y) goes to world (-y, x): static[k, j, i] = mu[k, n-1-i, j]
    n = g.nx
    k, j, i = np.meshgrid(np.arange(g.nz), np.arange(n), np.arange(n), indexing="ij")
    static_mu = mu[k, n - 1 - i, j]
    static = oracle.forward(g, static_mu, np.zeros(6))
    np.testing.assert_allclose(moved, static, rtol=0, atol=1e-10 * np.abs(static).max())


def test_rigid_move_of_scanner_and_object_leaves_projections_unchanged():
    rng = np.random.default_rng(13)
    g = small_geom()
    mu = smooth_volume(g, rng)
    pose = np.array([1.0, -2.0, 0.5, 0.1, -0.2, 0.15])
    base = oracle.forward(g, mu, pose)
    # move the whole scanner by (Q, d) and the object pose by the same motion
    Q, _ = oracle.rotation([0, 0, 0, 0.3, -0.4, 0.7])
    d = np.array([5.0, -7.0, 3.0])
    views = g.views.copy()
    for vi in range(g.n_views):
        views[vi, 0:3] = Q @ g.views[vi, 0:3] + d
        views[vi, 3:6] = Q @ g.views[vi, 3:6] + d
        views[vi, 6:9] = Q @ g.views[vi, 6:9]
        views[vi, 9:12] = Q @ g.views[vi, 9:12]
    g2 = synth.Geometry(g.nx, g.ny, g.nz, g.vx, g.vy, g.vz, g.nu, g.nv, views, g.step, g.off)
    R, _ = oracle.rotation(pose)
    R2 = Q @ R
    pose2 = np.concatenate([Q @ pose[:3] + d, euler_from_matrix(R2)])
    np.testing.assert_allclose(oracle.rotation(pose2)[0], R2, atol=1e-13)
    moved = oracle.forward(g2, mu, pose2)
    np.testing.assert_allclose(moved, base, rtol=0, atol=1e-9 * np.abs(base).max())


def test_volume_offset_equals_translation():
    """A volume centred at off in the object frame projects like the
    centred volume translated by R off (here R = I)."""
    rng = np.random.default_rng(14)
    g = small_geom(off=(3.0, -2.0, 1.5))
    mu = smooth_volume(g, rng)
    g0 = small_geom()
    a = oracle.forward(g, mu, np.zeros(6))
    b = oracle.forward(g0, mu, np.array([3.0, -2.0, 1.5, 0, 0, 0]))
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-10 * np.abs(b).max())


def test_adjoint_identity_forward():
    rng = np.random.default_rng(15)
    g = small_geom(n=(11, 9, 13), det=(14, 12), n_views=2)
    poses = np.array([[1.0, -0.5, 0.3, 0.1, 0.2, -0.3], [0.0, 1.0, 0.0, -0.2, 0.0, 0.4]])
    x = rng.standard_normal(g.vol_shape)
    y = rng.standard_normal((2, g.nv, g.nu))
    ax = oracle.forward(g, x, poses, inst_view=[0, 1], inst_pose=[0, 1])
    aty = oracle.forward_adjoint(g, y, poses, inst_view=[0, 1], inst_pose=[0, 1])
    lhs, rhs = np.sum(ax * y), np.sum(x * aty)
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(ax * ax) * np.sum(y * y))


def _loss_fd(g, mu, w, pose, inst_view=None):
    def f(th):
        return float(np.sum(w * oracle.forward(g, mu, th, inst_view=inst_view)))
    return f


def test_exact_mode_gradient_equals_finite_differences():
    """Exact-discrete gradient == central FD of the discrete forward model.
    Steps are tiny so that trilinear kinks are crossed rarely."""
    rng = np.random.default_rng(16)
    g = small_geom(n=(18, 16, 20), det=(16, 14), n_views=2)
    mu = smooth_volume(g, rng) + 0.2 * rng.uniform(0, 1, g.vol_shape)
    for trial in range(3):
        pose = np.concatenate([rng.uniform(-3, 3, 3), rng.uniform(-0.3, 0.3, 3)])
        w = rng.standard_normal((g.n_views, g.nv, g.nu))
        gth, _ = oracle.forward_grad(g, mu, pose, w, mode=oracle.GRAD_EXACT)
        fd = central_fd(_loss_fd(g, mu, w, pose), pose, [1e-6] * 3 + [1e-7] * 3)
        for blk in (slice(0, 3), slice(3, 6)):
            rel = np.linalg.norm(gth[0, blk] - fd[blk]) / np.linalg.norm(fd[blk])
            assert rel < 1e-7, (trial, blk, rel, gth, fd)


def _paper_bars():
    with open(os.path.join(GOLDEN, "paper_gradient_cosine.json")) as f:
        return json.load(f)


def test_paper_analytic_gradient_cosine_similarity():
    """Paper-analytic gradient (central-difference grad mu interpolated at
    each sample) vs the true derivative of the discrete model, by cosine
    similarity (Sec. II-D.1).  L2 loss against a target at another pose,
    8 views over 0-90 deg.  Mean bar = the paper's RD figure (Sec. III-A)."""
    bars = _paper_bars()
    rng = np.random.default_rng(17)
    views = synth.circular_views(8, 200.0, 320.0, 2.0, 2.0,
                                 angles=np.linspace(0, np.pi / 2, 8))
    g = synth.Geometry(24, 24, 24, 1.5, 1.5, 1.5, 20, 20, views, 0.75)
    mu = smooth_volume(g, rng, n_blobs=8, sigma=(3.0, 6.0))
    target = oracle.forward(g, mu, np.zeros(6))
    cos = []
    for _ in range(12):
        pose = np.concatenate([rng.normal(0, 3.0, 3), np.deg2rad(rng.normal(0, 5.0, 3))])
        proj = oracle.forward(g, mu, pose)
        _, w = oracle.l2_loss(proj, target)
        ga, _ = oracle.forward_grad(g, mu, pose, w, mode=oracle.GRAD_ANALYTIC)
        ge, _ = oracle.forward_grad(g, mu, pose, w, mode=oracle.GRAD_EXACT)
        cos.append(oracle.cosine(ga, ge))
    assert np.mean(cos) >= bars["forward_rd_mean"], cos


def test_golden_forward_regression():
    """Stored oracle output of a tiny fixed case (written by
    tests/golden/make_golden.py, which calls only the oracle)."""
    path = os.path.join(GOLDEN, "forward_tiny.npz")
    data = np.load(path)
    g = synth.Geometry(*[int(x) for x in data["dims"]], *data["vox"],
                       int(data["det"][0]), int(data["det"][1]), data["views"],
                       float(data["step"]), tuple(data["off"]))
    p = oracle.forward(g, data["mu"], data["poses"], inst_view=data["inst_view"],
                       inst_pose=data["inst_pose"])
    np.testing.assert_allclose(p, data["proj"], rtol=1e-12, atol=1e-14)


def test_analytic_gradient_is_continuous_across_the_box_face():
    """The interpolated central-difference volume gradient lives on
    (-2, n+1)^3: a ray moving across the face of the volume's box changes
    the analytic forward gradient continuously."""
    mu = np.ones((3, 3, 3))
    view = np.array([-800.0, 0.0, 0.0, 400.0, 0.0, 0.0, 0, 1.0, 0, 0, 0, 1.0])
    g = synth.Geometry(3, 3, 3, 1.0, 1.0, 1.0, 1, 1, view[None, :], 0.5)
    w = np.ones((1, 1, 1))
    vals = []
    for ty in (1.999, 2.001):      # the ray passes at index y = 1 - ty, near the face y = -1
        gth, _ = oracle.forward_grad(g, mu, np.array([0, ty, 0, 0, 0, 0.0]), w, mode=oracle.GRAD_ANALYTIC)
        vals.append(gth[0])
    assert abs(vals[0][1]) > 0.1
    assert np.linalg.norm(vals[0] - vals[1]) < 1e-2 * np.linalg.norm(vals[0])


def test_voxel_centre_recipe_differs_at_second_order():
    """The paper's three-step recipe read literally (form G = grad mu (x)
    (r - t) at voxel centres, then interpolate it like mu) and the graded
    reading (interpolate grad mu, multiply by the exact r - t of each
    integration point) differ only by the interpolation error of a product:
    on the same continuous phantom, halving the voxel size divides the
    difference by about 4, and it is small next to the gradient itself."""
    pose = np.array([1.5, -1.0, 2.0, 0.05, -0.08, 0.1])
    rng = np.random.default_rng(8)
    w = rng.standard_normal((3, 24, 24))
    diffs = []
    for n, v in [(48, 1.6), (96, 0.8)]:
        g, _, mu = blob_setup(n, v)
        ga, gMa = oracle.forward_grad(g, mu, pose, w, mode=oracle.GRAD_ANALYTIC)
        gc, gMc = oracle.forward_grad(g, mu, pose, w, mode=oracle.GRAD_VOXEL_CENTRE)
        diffs.append(np.linalg.norm(gMc - gMa) / np.linalg.norm(gMa))
    assert 0 < diffs[1] < diffs[0] < 2e-2, diffs
    assert 2.8 < diffs[0] / diffs[1] < 6.0, diffs            # O(h^2): ideal ratio 4

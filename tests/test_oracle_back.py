"""Pins of the oracle's voxel-driven back-projector (Eq. back, Sec.
II-C.2) and of its rigid-pose gradient (Eqs. back_derive, final_back,
back_int, dis_back) against results that do not come from the oracle:
detector coordinates by ray-plane intersection, images that bilinear
interpolation reproduces exactly, finite differences and the adjoint
identity."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import central_fd, detector_coords, hat_support, small_geom, smooth_volume

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def moved_voxels(g, pose):
    """World positions R r' + t of all voxel centres, [N, 3] in memory order."""
    X, Y, Z = synth.voxel_centres(g)
    rp = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    R, _ = oracle.rotation(pose)
    return rp @ R.T + pose[:3]


def fdk_weight_independent(view, r):
    """(SAD / depth)^2 with depth measured along the detector normal from the
    source and SAD the same depth of the world origin."""
    s, U, V = view[0:3], view[6:9], view[9:12]
    n = np.cross(U, V)
    n = n / np.linalg.norm(n)
    n = n if np.dot(view[3:6] - s, n) > 0 else -n
    return (np.dot(-s, n) / ((r - s) @ n)) ** 2


@pytest.mark.parametrize("weight", [oracle.W_NONE, oracle.W_FDK])
def test_constant_image_back_projects_to_weight_sum(weight):
    """l = 1 on every detector: mu_j = sum_v W_v(r_j) h(u_j) h(v_j), where h
    is the bilinear interpolant of an all-ones row with zero padding."""
    rng = np.random.default_rng(21)
    g = small_geom(det=(14, 11), pix=1.4, n_views=3)
    poses = np.concatenate([rng.uniform(-2, 2, (3, 3)), rng.uniform(-0.2, 0.2, (3, 3))], axis=1)
    proj = np.ones((3, g.nv, g.nu))
    vol = oracle.back(g, proj, poses, inst_view=[0, 1, 2], inst_pose=[0, 1, 2], weight=weight)
    expect = np.zeros(g.vol_shape).ravel()
    for n in range(3):
        r = moved_voxels(g, poses[n])
        u, v, _ = detector_coords(g.views[n], g.nu, g.nv, r)
        W = fdk_weight_independent(g.views[n], r) if weight == oracle.W_FDK else 1.0
        expect += W * hat_support(u, g.nu) * hat_support(v, g.nv)
    np.testing.assert_allclose(vol.ravel(), expect, rtol=1e-11, atol=1e-12)
    assert np.count_nonzero(expect == 0) > 0 and np.count_nonzero(expect) > 0


def linear_image_case(weight, pose):
    g = small_geom(n=(12, 10, 9), det=(90, 80), pix=1.0, n_views=2)
    coef = [(0.013, -0.021, 0.7), (-0.008, 0.017, 1.1)]
    proj = np.zeros((2, g.nv, g.nu))
    iu, iv = np.meshgrid(np.arange(g.nu), np.arange(g.nv))
    for n, (a, b, c) in enumerate(coef):
        proj[n] = a * iu + b * iv + c

    def closed_form(th):
        out = np.zeros(g.nx * g.ny * g.nz)
        for n, (a, b, c) in enumerate(coef):
            r = moved_voxels(g, th)
            u, v, _ = detector_coords(g.views[n], g.nu, g.nv, r)
            assert u.min() > 2 and u.max() < g.nu - 3 and v.min() > 2 and v.max() < g.nv - 3
            W = fdk_weight_independent(g.views[n], r) if weight != oracle.W_NONE else 1.0
            out += W * (a * u + b * v + c)
        return out.reshape(g.vol_shape)
    return g, proj, closed_form


@pytest.mark.parametrize("weight", [oracle.W_NONE, oracle.W_FDK])
def test_linear_image_back_projects_exactly(weight):
    pose = np.array([1.0, -0.5, 0.8, 0.05, -0.1, 0.2])
    g, proj, closed = linear_image_case(weight, pose)
    vol = oracle.back(g, proj, pose, inst_view=[0, 1], inst_pose=[0, 0], weight=weight)
    np.testing.assert_allclose(vol, closed(pose), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("weight", [oracle.W_NONE, oracle.W_FDK])
def test_linear_image_gradient_matches_closed_form(weight):
    """For a linear image whose support covers every projected voxel, the
    central-difference detector gradient equals the true one, so both
    gradient modes must equal the FD of the closed-form back-projection
    (which uses no projection matrix, no Jacobian and no weight derivative
    from the oracle)."""
    pose = np.array([1.0, -0.5, 0.8, 0.05, -0.1, 0.2])
    g, proj, closed = linear_image_case(weight, pose)
    rng = np.random.default_rng(22)
    wvol = rng.standard_normal(g.vol_shape)
    fd = central_fd(lambda th: float(np.sum(wvol * closed(th))), pose, [1e-5] * 3 + [1e-6] * 3)
    for mode in (oracle.GRAD_ANALYTIC, oracle.GRAD_EXACT):
        gth, _ = oracle.back_grad(g, proj, pose, wvol, inst_view=[0, 1], inst_pose=[0, 0],
                                  weight=weight, mode=mode)
        for blk in (slice(0, 3), slice(3, 6)):
            rel = np.linalg.norm(gth[0, blk] - fd[blk]) / np.linalg.norm(fd[blk])
            assert rel < 1e-7, (mode, blk, rel)


@pytest.mark.parametrize("weight", [oracle.W_NONE, oracle.W_FDK])
def test_adjoint_identity_back(weight):
    rng = np.random.default_rng(23)
    g = small_geom(n=(10, 12, 9), det=(15, 13), n_views=2)
    poses = np.array([[0.5, -0.5, 0.3, 0.1, 0.2, -0.3], [0.0, 1.0, 0.0, -0.2, 0.0, 0.4]])
    y = rng.standard_normal((2, g.nv, g.nu))
    x = rng.standard_normal(g.vol_shape)
    by = oracle.back(g, y, poses, inst_view=[0, 1], inst_pose=[0, 1], weight=weight)
    btx = oracle.back_adjoint(g, x, poses, inst_view=[0, 1], inst_pose=[0, 1], weight=weight)
    lhs, rhs = np.sum(by * x), np.sum(y * btx)
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(by * by) * np.sum(x * x))


def smooth_projections(g, rng, n_inst):
    """Smooth detector images: projections of a blob volume."""
    mu = smooth_volume(g, rng)
    return oracle.forward(g, mu, np.zeros(6), inst_view=np.arange(n_inst) % g.n_views,
                          inst_pose=np.zeros(n_inst, dtype=int))


@pytest.mark.parametrize("weight", [oracle.W_NONE, oracle.W_FDK])
def test_exact_mode_gradient_equals_finite_differences(weight):
    rng = np.random.default_rng(24)
    g = small_geom(n=(14, 12, 16), det=(22, 20), n_views=2)
    proj = smooth_projections(g, rng, 2) + 0.1 * rng.uniform(0, 1, (2, g.nv, g.nu))
    for trial in range(2):
        pose = np.concatenate([rng.uniform(-3, 3, 3), rng.uniform(-0.3, 0.3, 3)])
        wvol = rng.standard_normal(g.vol_shape)

        def loss(th):
            return float(np.sum(wvol * oracle.back(g, proj, th, inst_view=[0, 1],
                                                   inst_pose=[0, 0], weight=weight)))
        gth, _ = oracle.back_grad(g, proj, pose, wvol, inst_view=[0, 1], inst_pose=[0, 0],
                                  weight=weight, mode=oracle.GRAD_EXACT)
        fd = central_fd(loss, pose, [1e-6] * 3 + [1e-7] * 3)
        for blk in (slice(0, 3), slice(3, 6)):
            rel = np.linalg.norm(gth[0, blk] - fd[blk]) / np.linalg.norm(fd[blk])
            assert rel < 1e-7, (trial, blk, rel)


def test_constant_weight_variant_drops_the_weight_derivative():
    """The paper-literal variant (no l * grad W term) is not the derivative
    of the FDK-weighted back-projection; the full variant is."""
    rng = np.random.default_rng(25)
    g = small_geom(n=(14, 12, 16), det=(22, 20), n_views=2)
    proj = smooth_projections(g, rng, 2) + 1.0
    pose = np.array([1.0, 2.0, -1.0, 0.1, 0.05, -0.1])
    wvol = rng.uniform(0.5, 1.0, g.vol_shape)
    full, _ = oracle.back_grad(g, proj, pose, wvol, inst_view=[0, 1], inst_pose=[0, 0],
                               weight=oracle.W_FDK, mode=oracle.GRAD_EXACT)
    const, _ = oracle.back_grad(g, proj, pose, wvol, inst_view=[0, 1], inst_pose=[0, 0],
                                weight=oracle.W_FDK_CONST, mode=oracle.GRAD_EXACT)
    assert np.linalg.norm(full - const) > 1e-3 * np.linalg.norm(full)


def test_paper_analytic_gradient_cosine_similarity():
    """Paper-analytic BP gradient (central-difference detector gradient
    interpolated at each projected voxel) vs the true derivative of the
    discrete back-projector, L2 image loss (Eq. back_loss).  Mean bar = the
    paper's VD figure (Sec. III-A)."""
    with open(os.path.join(GOLDEN, "paper_gradient_cosine.json")) as f:
        bars = json.load(f)
    rng = np.random.default_rng(26)
    views = synth.circular_views(8, 200.0, 320.0, 1.5, 1.5,
                                 angles=np.linspace(0, np.pi / 2, 8))
    g = synth.Geometry(20, 20, 20, 1.5, 1.5, 1.5, 32, 32, views, 0.75)
    mu_true = smooth_volume(g, rng, n_blobs=8, sigma=(3.0, 6.0))
    proj = oracle.forward(g, mu_true, np.zeros(6))
    target = oracle.back(g, proj, np.zeros(6))
    cos = []
    for _ in range(10):
        pose = np.concatenate([rng.normal(0, 3.0, 3), np.deg2rad(rng.normal(0, 5.0, 3))])
        vol = oracle.back(g, proj, pose)
        _, wvol = oracle.l2_loss(vol, target)
        ga, _ = oracle.back_grad(g, proj, pose, wvol, mode=oracle.GRAD_ANALYTIC)
        ge, _ = oracle.back_grad(g, proj, pose, wvol, mode=oracle.GRAD_EXACT)
        cos.append(oracle.cosine(ga, ge))
    assert np.mean(cos) >= bars["back_vd_mean"], cos


def test_voxels_behind_the_source_receive_nothing():
    """A source inside the volume: voxels with w' <= 0 get no contribution."""
    view = np.array([0.0, 0.0, 0.0, -50.0, 0.0, 0.0, 0.0, 5.0, 0.0, 0.0, 0.0, 5.0])
    g = synth.Geometry(9, 3, 3, 2.0, 2.0, 2.0, 40, 40, view[None, :], 1.0)
    vol = oracle.back(g, np.ones((1, 40, 40)), np.zeros(6))
    X, _, _ = synth.voxel_centres(g)
    assert np.all(vol[X > 0] == 0) and np.all(vol[X < -1] > 0)


def test_analytic_gradient_is_continuous_across_the_image_edge():
    """The interpolated central-difference detector gradient lives on
    (-2, nu+1): moving a voxel's projection across u = -1 changes the
    analytic BP gradient continuously (no jump of order l[0])."""
    view = np.array([400.0, 0.0, 0.0, -400.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0])
    g = synth.Geometry(1, 1, 1, 1.0, 1.0, 1.0, 8, 8, view[None, :], 1.0)
    img = np.full((1, 8, 8), 3.0)
    wvol = np.ones((1, 1, 1))
    # the voxel at the origin projects to u = 3.5 + 2 ty (magnification 2,
    # 1 mm pixels): u = -1 at ty = -2.25
    vals = []
    for ty in (-2.249, -2.251):
        gth, _ = oracle.back_grad(g, img, np.array([0, ty, 0, 0, 0, 0.0]), wvol, weight=oracle.W_NONE)
        vals.append(gth[0])
    assert abs(vals[0][1]) > 0.1
    assert np.linalg.norm(vals[0] - vals[1]) < 1e-2 * np.linalg.norm(vals[0])

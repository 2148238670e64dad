"""Pins of the oracle's pose and projection-matrix construction (Table I,
Eq. projmatrix) against geometric facts that do not come from the oracle."""
import numpy as np
import pytest

import oracle
from helpers import axis_angle_matrix, detector_coords, euler_from_matrix


def rot(gx=0.0, gy=0.0, gz=0.0):
    return oracle.rotation([0, 0, 0, gx, gy, gz])


@pytest.mark.parametrize("axis,src,dst", [(0, 1, 2), (1, 2, 0), (2, 0, 1)])
def test_quarter_turns_are_right_handed(axis, src, dst):
    g = [0.0, 0.0, 0.0]
    g[axis] = np.pi / 2
    R, _ = rot(*g)
    e = np.zeros(3)
    e[src] = 1.0
    expect = np.zeros(3)
    expect[dst] = 1.0
    np.testing.assert_allclose(R @ e, expect, atol=1e-15)


def test_single_axis_matches_rodrigues():
    rng = np.random.default_rng(0)
    for axis in range(3):
        for ang in rng.uniform(-3, 3, 5):
            g = [0.0, 0.0, 0.0]
            g[axis] = ang
            R, _ = rot(*g)
            np.testing.assert_allclose(R, axis_angle_matrix(np.eye(3)[axis], ang),
                                       atol=1e-14)


def test_composition_order_is_z_y_x():
    rng = np.random.default_rng(1)
    for _ in range(5):
        gx, gy, gz = rng.uniform(-1.2, 1.2, 3)
        R, _ = rot(gx, gy, gz)
        expect = axis_angle_matrix([0, 0, 1], gz) @ axis_angle_matrix([0, 1, 0], gy) \
            @ axis_angle_matrix([1, 0, 0], gx)
        np.testing.assert_allclose(R, expect, atol=1e-14)
        np.testing.assert_allclose(euler_from_matrix(R), [gx, gy, gz], atol=1e-12)


def test_rotation_derivatives_match_finite_differences():
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(5):
        th = np.concatenate([rng.uniform(-5, 5, 3), rng.uniform(-1, 1, 3)])
        _, dR = oracle.rotation(th)
        for j in range(3):
            e = np.zeros(6)
            e[3 + j] = h
            fd = (oracle.rotation(th + e)[0] - oracle.rotation(th - e)[0]) / (2 * h)
            np.testing.assert_allclose(dR[j], fd, atol=1e-9)


def random_view(rng):
    s = rng.uniform(-50, 50, 3) + np.array([700.0, 0, 0])
    c = rng.uniform(-20, 20, 3) + np.array([-400.0, 0, 0])
    U = np.array([0.0, 1.0, 0.0]) * 1.3 + rng.uniform(-0.2, 0.2, 3)
    V = np.array([0.0, 0.0, 1.0]) * 0.9 + rng.uniform(-0.2, 0.2, 3)
    return np.concatenate([s, c, U, V])


def test_projection_matrix_matches_ray_plane_intersection():
    rng = np.random.default_rng(3)
    nu, nv = 37, 23
    for _ in range(5):
        view = random_view(rng)
        P = oracle.projection_matrix(view, nu, nv)
        pts = rng.uniform(-60, 60, (50, 3))
        h = pts @ P[:, :3].T + P[:, 3]
        u, v, lam = detector_coords(view, nu, nv, pts)
        np.testing.assert_allclose(h[:, 0] / h[:, 2], u, rtol=0, atol=1e-9)
        np.testing.assert_allclose(h[:, 1] / h[:, 2], v, rtol=0, atol=1e-9)
        # w' is the distance ratio |r - s| / |q - s| along the ray
        np.testing.assert_allclose(h[:, 2], lam, rtol=1e-12)


def test_pixel_centres_project_to_their_indices():
    rng = np.random.default_rng(4)
    nu, nv = 9, 6
    view = random_view(rng)
    P = oracle.projection_matrix(view, nu, nv)
    s, c, U, V = view[0:3], view[3:6], view[6:9], view[9:12]
    for iu in range(nu):
        for iv in range(nv):
            q = c + (iu - (nu - 1) / 2) * U + (iv - (nv - 1) / 2) * V
            for lam in (0.3, 0.7, 1.0):
                r = s + lam * (q - s)
                h = P[:, :3] @ r + P[:, 3]
                assert abs(h[0] / h[2] - iu) < 1e-9 and abs(h[1] / h[2] - iv) < 1e-9
                assert abs(h[2] - lam) < 1e-12

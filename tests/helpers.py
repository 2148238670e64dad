"""Small independent helpers for the tests (no projector arithmetic of the
oracle or of the CUDA path is reused here)."""
import numpy as np

import synth


def euler_from_matrix(R):
    """Angles (gx, gy, gz) with R = Rz(gz) Ry(gy) Rx(gx), away from gimbal
    lock (|gy| < 90 deg).  Standard decomposition: R[2,0] = -sin gy,
    R[2,1] = cos gy sin gx, R[2,2] = cos gy cos gx, R[1,0] = sin gz cos gy,
    R[0,0] = cos gz cos gy."""
    gy = -np.arcsin(np.clip(R[2, 0], -1.0, 1.0))
    gx = np.arctan2(R[2, 1], R[2, 2])
    gz = np.arctan2(R[1, 0], R[0, 0])
    return np.array([gx, gy, gz])


def axis_angle_matrix(axis, angle):
    """Rodrigues' formula, independent of the Euler construction."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def detector_coords(view, nu, nv, r):
    """(u, v, depth-ratio) of world points r [N,3] by ray-plane intersection:
    the ray from s through r meets the detector plane at q; solve
    q - q00 = u U + v V.  Returns u, v and lam = |r - s| / |q - s|."""
    s, c, U, V = view[0:3], view[3:6], view[6:9], view[9:12]
    n = np.cross(U, V)
    q00 = c - 0.5 * (nu - 1) * U - 0.5 * (nv - 1) * V
    r = np.atleast_2d(r)
    d = r - s
    lam_q = np.dot(c - s, n) / (d @ n)          # q = s + lam_q d
    q = s + lam_q[:, None] * d
    A = np.stack([U, V], axis=1)               # 3x2
    uv, *_ = np.linalg.lstsq(A, (q - q00).T, rcond=None)
    return uv[0], uv[1], 1.0 / lam_q


def hat_support(x, n):
    """Bilinear interpolant (one axis) of an all-ones image of n pixels with
    zero padding, evaluated at x."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    out = np.where(x < 0, np.clip(1 + x, 0, 1), out)
    out = np.where(x > n - 1, np.clip(n - x, 0, 1), out)
    return out


def central_fd(fun, theta, steps):
    """Central finite differences of a scalar function of a pose vector."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros_like(theta)
    for j in range(theta.size):
        e = np.zeros_like(theta)
        e.flat[j] = steps[j % 6]
        g.flat[j] = (fun(theta + e) - fun(theta - e)) / (2 * steps[j % 6])
    return g


def small_geom(n=(20, 18, 22), vox=(1.0, 1.1, 0.9), det=(24, 20), pix=2.0,
               n_views=3, step=0.5, off=(0.0, 0.0, 0.0), sad=200.0, sdd=320.0):
    views = synth.circular_views(n_views, sad, sdd, pix, pix)
    return synth.Geometry(n[0], n[1], n[2], vox[0], vox[1], vox[2], det[0],
                          det[1], views, step, off)


def smooth_volume(geom, rng, n_blobs=6, sigma=(2.5, 5.0)):
    """Random sum of Gaussian blobs inside the grid."""
    ext = np.array([geom.nx * geom.vx, geom.ny * geom.vy, geom.nz * geom.vz])
    blobs = []
    for _ in range(n_blobs):
        c = rng.uniform(-0.25, 0.25, 3) * ext + np.asarray(geom.off)
        blobs.append((rng.uniform(0.5, 1.5), c, rng.uniform(*sigma)))
    return synth.gaussian_blobs(geom, blobs)

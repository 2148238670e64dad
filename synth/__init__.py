"""Seeded synthetic inputs shared by the tests and the benchmark.

Everything here is input generation only: phantoms voxelised at voxel
centres, circular cone-beam view vectors, random poses and random detector
images.  No projection, interpolation or gradient arithmetic of the method
lives in this module, so both the FP64 oracle and the CUDA path can be fed
the same bytes without sharing any of the method's code.

Conventions (the paper leaves them open, Sec. II-A):
  * world frame in mm, origin = isocentre;
  * view vectors per view: source s, detector centre c, pixel-pitch vectors
    U (along increasing column index iu) and V (along increasing row iv);
    pixel (iu, iv) centre = c + (iu-(nu-1)/2) U + (iv-(nv-1)/2) V;
  * circular orbit at angle b: s = SAD (cos b, sin b, 0),
    c = -(SDD-SAD) (cos b, sin b, 0), U = du (-sin b, cos b, 0),
    V = dv (0, 0, 1);
  * volume memory order [nz][ny][nx]; voxel (i, j, k) centre in the object
    frame = off + ((i-(nx-1)/2) vx, (j-(ny-1)/2) vy, (k-(nz-1)/2) vz);
  * pose theta = (tx, ty, tz, gx, gy, gz) in mm and rad (Table I).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Geometry:
    """Plain description of a cone-beam scan (host data only)."""
    nx: int
    ny: int
    nz: int
    vx: float
    vy: float
    vz: float
    nu: int
    nv: int
    views: np.ndarray            # [n_views][12] float64: s, c, U, V
    step: float                  # ray step (mm) along the world ray
    off: tuple = (0.0, 0.0, 0.0)  # object-frame volume centre (mm)

    @property
    def n_views(self) -> int:
        return int(self.views.shape[0])

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)


def circular_views(n_views, sad, sdd, du, dv, angles=None):
    """View vectors of a circular orbit; angles default to 2*pi*k/n_views."""
    if angles is None:
        angles = 2.0 * np.pi * np.arange(n_views) / n_views
    angles = np.asarray(angles, dtype=np.float64)
    out = np.zeros((len(angles), 12), dtype=np.float64)
    cb, sb = np.cos(angles), np.sin(angles)
    out[:, 0] = sad * cb
    out[:, 1] = sad * sb
    out[:, 3] = -(sdd - sad) * cb
    out[:, 4] = -(sdd - sad) * sb
    out[:, 6] = -du * sb
    out[:, 7] = du * cb
    out[:, 11] = dv
    return out


def voxel_centres(geom: Geometry):
    """Object-frame voxel-centre coordinates as three [nz][ny][nx] arrays."""
    x = (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.vx + geom.off[0]
    y = (np.arange(geom.ny) - (geom.ny - 1) / 2.0) * geom.vy + geom.off[1]
    z = (np.arange(geom.nz) - (geom.nz - 1) / 2.0) * geom.vz + geom.off[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def random_rotation(rng):
    """Uniformly random 3x3 rotation (QR of a Gaussian matrix)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@dataclasses.dataclass
class Ellipsoid:
    centre: np.ndarray   # (3,) mm, object frame
    axes: np.ndarray     # (3,3) columns = unit axis directions
    semi: np.ndarray     # (3,) semi-axis lengths, mm
    mu: float            # attenuation, 1/mm


@dataclasses.dataclass
class Cylinder:
    centre: np.ndarray
    axis: np.ndarray     # (3,) unit
    radius: float
    half_len: float
    mu: float


def random_ellipsoids(rng, n, centre_range, semi_range, mu_range):
    out = []
    for _ in range(n):
        out.append(Ellipsoid(
            centre=rng.uniform(-centre_range, centre_range, 3),
            axes=random_rotation(rng),
            semi=rng.uniform(semi_range[0], semi_range[1], 3),
            mu=float(rng.uniform(mu_range[0], mu_range[1]))))
    return out


def random_cylinders(rng, n, centre_range, radius_range, half_len_range,
                     mu_range):
    out = []
    for _ in range(n):
        a = rng.standard_normal(3)
        out.append(Cylinder(
            centre=rng.uniform(-centre_range, centre_range, 3),
            axis=a / np.linalg.norm(a),
            radius=float(rng.uniform(*radius_range)),
            half_len=float(rng.uniform(*half_len_range)),
            mu=float(rng.uniform(*mu_range))))
    return out


def voxelise(geom: Geometry, ellipsoids=(), cylinders=(), supersample=1):
    """Sum of shapes (overlaps add), point-sampled at voxel centres or at
    supersample^3 sub-voxel points averaged.  Returns float64 [nz][ny][nx]."""
    vol = np.zeros(geom.vol_shape, dtype=np.float64)
    ss = int(supersample)
    subs = (np.arange(ss) + 0.5) / ss - 0.5
    x0 = (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.vx + geom.off[0]
    y0 = (np.arange(geom.ny) - (geom.ny - 1) / 2.0) * geom.vy + geom.off[1]
    z0 = (np.arange(geom.nz) - (geom.nz - 1) / 2.0) * geom.vz + geom.off[2]
    for dz in subs:
        for dy in subs:
            for dx in subs:
                Z = (z0 + dz * geom.vz)[:, None, None]
                Y = (y0 + dy * geom.vy)[None, :, None]
                X = (x0 + dx * geom.vx)[None, None, :]
                for e in ellipsoids:
                    px, py, pz = X - e.centre[0], Y - e.centre[1], Z - e.centre[2]
                    acc = 0.0
                    for a in range(3):
                        q = (px * e.axes[0, a] + py * e.axes[1, a]
                             + pz * e.axes[2, a]) / e.semi[a]
                        acc = acc + q * q
                    vol += np.where(acc <= 1.0, e.mu, 0.0)
                for c in cylinders:
                    px, py, pz = X - c.centre[0], Y - c.centre[1], Z - c.centre[2]
                    along = px * c.axis[0] + py * c.axis[1] + pz * c.axis[2]
                    r2 = px * px + py * py + pz * pz - along * along
                    inside = (r2 <= c.radius ** 2) & (np.abs(along) <= c.half_len)
                    vol += np.where(inside, c.mu, 0.0)
    return vol / float(ss ** 3)


def gaussian_blobs(geom: Geometry, blobs):
    """Sum of isotropic Gaussians A exp(-|r'-c|^2 / (2 s^2)) sampled at voxel
    centres; blobs = [(A, centre(3,), sigma)]."""
    x0 = (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.vx + geom.off[0]
    y0 = (np.arange(geom.ny) - (geom.ny - 1) / 2.0) * geom.vy + geom.off[1]
    z0 = (np.arange(geom.nz) - (geom.nz - 1) / 2.0) * geom.vz + geom.off[2]
    Z, Y, X = z0[:, None, None], y0[None, :, None], x0[None, None, :]
    vol = np.zeros(geom.vol_shape, dtype=np.float64)
    for amp, c, s in blobs:
        r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
        vol += amp * np.exp(-r2 / (2.0 * s * s))
    return vol


def random_poses(rng, n, rot_deg, trans_mm):
    """[n][6] poses, translations U(-trans, trans) mm, rotations
    U(-rot, rot) degrees (returned in rad)."""
    p = np.zeros((n, 6), dtype=np.float64)
    p[:, :3] = rng.uniform(-trans_mm, trans_mm, (n, 3))
    p[:, 3:] = np.deg2rad(rng.uniform(-rot_deg, rot_deg, (n, 3)))
    return p


def smooth_motion(rng, n_views, rot_deg, trans_mm, n_terms=3):
    """Per-view smooth rigid motion: each parameter is a sum of n_terms
    seeded low-frequency sinusoids over the view index, scaled to peak at
    most (trans_mm, rot_deg)."""
    k = np.arange(n_views) / max(n_views, 1)
    out = np.zeros((n_views, 6), dtype=np.float64)
    for p in range(6):
        sig = np.zeros(n_views)
        for _ in range(n_terms):
            f = rng.integers(1, 4)
            ph = rng.uniform(0, 2 * np.pi)
            amp = rng.uniform(0.2, 1.0)
            sig += amp * np.sin(2 * np.pi * f * k + ph)
        sig /= max(np.max(np.abs(sig)), 1e-12)
        lim = trans_mm if p < 3 else np.deg2rad(rot_deg)
        out[:, p] = sig * lim * rng.uniform(0.5, 1.0)
    return out


# ---------------------------------------------------------------------------
# Workloads with the shapes of the five paper-derived configurations.  The
# paper's CQ500 head and real phantom scans are not available; these seeded
# phantoms stand in for them (sum of ellipsoids, plus cylinders for the
# high-contrast case).
# ---------------------------------------------------------------------------

SAD, SDD = 800.0, 1200.0


def workload_tiny(seed=1001):
    """64^3 at 1 mm, 10 ellipsoids; 8 views over 360 deg on a 128^2 detector
    at 1.5 mm; one pose (rot +-5 deg, trans +-5 mm); a target rendered at a
    second pose; a U(0,1) detector image for back-projection."""
    rng = np.random.default_rng(seed)
    geom = Geometry(64, 64, 64, 1.0, 1.0, 1.0, 128, 128,
                    circular_views(8, SAD, SDD, 1.5, 1.5), step=0.5)
    ell = random_ellipsoids(rng, 10, 20.0, (5.0, 25.0), (0.01, 0.03))
    mu = voxelise(geom, ell)
    pose = random_poses(rng, 1, 5.0, 5.0)
    pose_true = random_poses(rng, 1, 5.0, 5.0)
    det = rng.uniform(0.0, 1.0, (geom.n_views, geom.nv, geom.nu))
    return dict(geom=geom, mu=mu, pose=pose, pose_true=pose_true,
                det_image=det, ellipsoids=ell)


def workload_registration(seed=1002, n_cand=64, nvox=256, ndet=384,
                          vox=0.8, pix=0.8):
    """256^3 at 0.8 mm, ellipsoids plus two high-contrast cylinders; two
    views 90 deg apart on 384^2 detectors at 0.8 mm; n_cand candidate poses
    (rot +-15 deg, trans +-20 mm) and a true pose for the target."""
    rng = np.random.default_rng(seed)
    geom = Geometry(nvox, nvox, nvox, vox, vox, vox, ndet, ndet,
                    circular_views(2, SAD, SDD, pix, pix,
                                   angles=[0.0, np.pi / 2]), step=0.5 * vox)
    fov = nvox * vox
    ell = random_ellipsoids(rng, 10, 0.2 * fov, (0.05 * fov, 0.25 * fov),
                            (0.01, 0.03))
    cyl = random_cylinders(rng, 2, 0.2 * fov, (3.0, 8.0),
                           (0.1 * fov, 0.3 * fov), (0.05, 0.08))
    mu = voxelise(geom, ell, cyl)
    cand = random_poses(rng, n_cand, 15.0, 20.0)
    pose_true = random_poses(rng, 1, 15.0, 20.0)
    return dict(geom=geom, mu=mu, poses=cand, pose_true=pose_true,
                ellipsoids=ell, cylinders=cyl)


def workload_moco(seed=1003, n_views=360, nvox=256, ndet=512, vox=0.8,
                  pix=0.6):
    """Motion-compensated FDK-style back-projection: 360 views over 360 deg,
    512^2 detector at 0.6 mm, 256^3 at 0.8 mm, smooth per-view motion
    (rot <= 2 deg, trans <= 3 mm)."""
    rng = np.random.default_rng(seed)
    geom = Geometry(nvox, nvox, nvox, vox, vox, vox, ndet, ndet,
                    circular_views(n_views, SAD, SDD, pix, pix),
                    step=0.5 * vox)
    fov = nvox * vox
    ell = random_ellipsoids(rng, 10, 0.2 * fov, (0.05 * fov, 0.25 * fov),
                            (0.01, 0.03))
    mu = voxelise(geom, ell)
    motion = smooth_motion(rng, n_views, 2.0, 3.0)
    return dict(geom=geom, mu=mu, poses=motion, ellipsoids=ell)


def workload_uneven(seed=1004, n_extra=24, with_large=True, vox=0.5):
    """Uneven batch of independent problems (the calibration-style per-view
    registration scaled up): a 512^3 volume at 0.5 mm seen in 720 views over
    360 deg on 768^2 detectors at 0.556 mm, each view with its own pose
    (translations N(0, 1 mm), rotations N(0, 0.5 deg)); plus n_extra
    problems, each one view (random angle) of its own cubic volume with edge
    U{128..320} at 0.5 mm on a square detector with edge U{256..512} whose
    pitch makes the field of view 1.1x the volume diagonal.  Geometry and
    poses only; the volumes and reference images are drawn by the caller
    (their values do not change the work)."""
    rng = np.random.default_rng(seed)
    probs = []
    if with_large:
        g = Geometry(512, 512, 512, vox, vox, vox, 768, 768,
                     circular_views(720, SAD, SDD, 0.556, 0.556), step=0.5 * vox)
        pose = np.zeros((720, 6))
        pose[:, :3] = rng.normal(0.0, 1.0, (720, 3))
        pose[:, 3:] = np.deg2rad(rng.normal(0.0, 0.5, (720, 3)))
        probs.append(dict(geom=g, poses=pose))
    for _ in range(n_extra):
        n = int(rng.integers(128, 321))
        nd = int(rng.integers(256, 513))
        pitch = 1.1 * n * vox * math.sqrt(3.0) * (SDD / SAD) / nd
        g = Geometry(n, n, n, vox, vox, vox, nd, nd,
                     circular_views(1, SAD, SDD, pitch, pitch,
                                    angles=[rng.uniform(0, 2 * np.pi)]),
                     step=0.5 * vox)
        pose = np.zeros((1, 6))
        pose[:, :3] = rng.normal(0.0, 1.0, (1, 3))
        pose[:, 3:] = np.deg2rad(rng.normal(0.0, 0.5, (1, 3)))
        probs.append(dict(geom=g, poses=pose))
    return probs


def random_image(rng, shape, lo=0.0, hi=1.0):
    return rng.uniform(lo, hi, shape)


def deg(x):
    return math.radians(x)

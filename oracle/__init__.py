"""FP64 CPU oracle for the projector pair and its rigid-pose gradients.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  The CUDA library
never calls it and it never calls the CUDA library; the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over rays or
voxel slabs with a fixed-order final sum); this module only marshals numpy
arrays and adds the loss functions, which are a few lines of numpy:

* L2 projection loss, Eq. forward_loss:  L = sum_i (l_i - b_i)^2.
* NCC (Pearson correlation) of each view instance with its target, the
  registration loss of Sec. II-D.3; the per-pose loss is minus the mean
  over that pose's instances.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

GRAD_ANALYTIC, GRAD_EXACT, GRAD_VOXEL_CENTRE = 0, 1, 2
W_NONE, W_FDK, W_FDK_CONST = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (-O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC",
                               "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("vx", ctypes.c_double), ("vy", ctypes.c_double),
                ("vz", ctypes.c_double), ("off", ctypes.c_double * 3),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int),
                ("n_views", ctypes.c_int),
                ("views", ctypes.POINTER(ctypes.c_double)),
                ("step", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.or_projection_matrix.restype = ctypes.c_int
        _lib.or_max_threads.restype = ctypes.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Call:
    """Keeps the numpy buffers alive while a C call runs."""

    def __init__(self, geom, poses, inst_view=None, inst_pose=None):
        self.views = _f64(geom.views)
        self.g = _Geom(geom.nx, geom.ny, geom.nz, geom.vx, geom.vy, geom.vz,
                       (ctypes.c_double * 3)(*geom.off), geom.nu, geom.nv,
                       self.views.shape[0], _dp(self.views), geom.step)
        self.poses = _f64(np.reshape(poses, (-1, 6)))
        n_pose = self.poses.shape[0]
        if inst_view is None:
            inst_view = np.arange(geom.n_views)
        if inst_pose is None:
            inst_pose = np.zeros(len(inst_view), dtype=np.int32) if n_pose == 1 \
                else np.arange(len(inst_view))
        self.iv = np.ascontiguousarray(inst_view, dtype=np.int32)
        self.ip = np.ascontiguousarray(inst_pose, dtype=np.int32)
        assert self.iv.shape == self.ip.shape
        assert self.iv.min(initial=0) >= 0 and self.iv.max(initial=0) < geom.n_views
        assert self.ip.min(initial=0) >= 0 and self.ip.max(initial=0) < n_pose
        self.n_inst = int(self.iv.shape[0])
        self.n_pose = n_pose


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def max_threads() -> int:
    return int(_load().or_max_threads())


def rotation(theta):
    """R = Rz Ry Rx and dR/dgamma_j (j = x, y, z) for one pose."""
    th = _f64(theta).reshape(6)
    R = np.zeros(9)
    dR = np.zeros(27)
    _load().or_rotation(_dp(th), _dp(R), _dp(dR))
    return R.reshape(3, 3), dR.reshape(3, 3, 3)


def projection_matrix(view, nu, nv):
    """3x4 projection matrix of one view (Eq. projmatrix)."""
    v = _f64(view).reshape(12)
    P = np.zeros(12)
    rc = _load().or_projection_matrix(_dp(v), int(nu), int(nv), _dp(P))
    if rc != 0:
        raise ValueError("singular detector basis")
    return P.reshape(3, 4)


def forward(geom, mu, poses, inst_view=None, inst_pose=None,
            return_samples=False):
    """Forward projections [n_inst][nv][nu] (Eq. forward, ray-driven)."""
    c = _Call(geom, poses, inst_view, inst_pose)
    mu = _f64(mu)
    assert mu.shape == geom.vol_shape
    out = np.zeros((c.n_inst, geom.nv, geom.nu))
    ns = np.zeros(c.n_inst, dtype=np.int64)
    _load().or_forward(ctypes.byref(c.g), _dp(mu), _dp(c.poses), c.n_inst,
                       _ip(c.iv), _ip(c.ip), _dp(out),
                       ns.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return (out, ns) if return_samples else out


def forward_grad(geom, mu, poses, w, inst_view=None, inst_pose=None,
                 mode=GRAD_ANALYTIC):
    """dL/dtheta [n_pose][6] and dL/dM [n_pose][3][4] given w = dL/dl
    ([n_inst][nv][nu]) (Eqs. for_grad, final_forward, dis_forward)."""
    c = _Call(geom, poses, inst_view, inst_pose)
    mu = _f64(mu)
    w = _f64(w)
    assert w.shape == (c.n_inst, geom.nv, geom.nu)
    gM = np.zeros((c.n_pose, 12))
    gth = np.zeros((c.n_pose, 6))
    _load().or_forward_grad(ctypes.byref(c.g), _dp(mu), _dp(c.poses), c.n_pose,
                            c.n_inst, _ip(c.iv), _ip(c.ip), _dp(w), int(mode),
                            _dp(gM), _dp(gth))
    return gth, gM.reshape(c.n_pose, 3, 4)


def forward_adjoint(geom, y, poses, inst_view=None, inst_pose=None):
    """Exact transpose of ``forward`` applied to y ([n_inst][nv][nu])."""
    c = _Call(geom, poses, inst_view, inst_pose)
    y = _f64(y)
    vol = np.zeros(geom.vol_shape)
    _load().or_forward_adjoint(ctypes.byref(c.g), _dp(y), _dp(c.poses), c.n_inst,
                               _ip(c.iv), _ip(c.ip), _dp(vol))
    return vol


def back(geom, proj, poses, inst_view=None, inst_pose=None, weight=W_NONE):
    """Voxel-driven back-projection of proj ([n_inst][nv][nu]) (Eq. back)."""
    c = _Call(geom, poses, inst_view, inst_pose)
    proj = _f64(proj)
    assert proj.shape == (c.n_inst, geom.nv, geom.nu)
    vol = np.zeros(geom.vol_shape)
    _load().or_back(ctypes.byref(c.g), _dp(proj), _dp(c.poses), c.n_inst,
                    _ip(c.iv), _ip(c.ip), int(weight), _dp(vol))
    return vol


def back_adjoint(geom, y, poses, inst_view=None, inst_pose=None,
                 weight=W_NONE):
    """Exact transpose of ``back`` applied to a volume y."""
    c = _Call(geom, poses, inst_view, inst_pose)
    y = _f64(y)
    out = np.zeros((c.n_inst, geom.nv, geom.nu))
    _load().or_back_adjoint(ctypes.byref(c.g), _dp(y), _dp(c.poses), c.n_inst,
                            _ip(c.iv), _ip(c.ip), int(weight), _dp(out))
    return out


def back_grad(geom, proj, poses, wvol, inst_view=None, inst_pose=None,
              weight=W_NONE, mode=GRAD_ANALYTIC):
    """dL/dtheta [n_pose][6] and dL/dM [n_pose][3][4] of an image-domain loss
    given wvol = dL/dmu (Eqs. back_derive, final_back, dis_back)."""
    c = _Call(geom, poses, inst_view, inst_pose)
    proj = _f64(proj)
    wvol = _f64(wvol)
    gM = np.zeros((c.n_pose, 12))
    gth = np.zeros((c.n_pose, 6))
    _load().or_back_grad(ctypes.byref(c.g), _dp(proj), _dp(c.poses), c.n_pose,
                         c.n_inst, _ip(c.iv), _ip(c.ip), int(weight), int(mode),
                         _dp(wvol), _dp(gM), _dp(gth))
    return gth, gM.reshape(c.n_pose, 3, 4)


def forward_pixels(geom, mu, poses, pix, inst_view=None, inst_pose=None):
    """Forward projection of selected rays only; pix = [m][3] (instance,
    iu, iv).  Same definition as ``forward``."""
    c = _Call(geom, poses, inst_view, inst_pose)
    mu = _f64(mu)
    pix = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(pix.shape[0])
    _load().or_forward_pixels(ctypes.byref(c.g), _dp(mu), _dp(c.poses), _ip(c.iv), _ip(c.ip),
                              int(pix.shape[0]), _ip(pix), _dp(out))
    return out


def back_voxels(geom, proj, poses, vox, inst_view=None, inst_pose=None, weight=W_NONE):
    """Back-projection at selected voxels only; vox = [m][3] (i, j, k).
    Same definition as ``back``."""
    c = _Call(geom, poses, inst_view, inst_pose)
    proj = _f64(proj)
    assert proj.shape == (c.n_inst, geom.nv, geom.nu)
    vox = np.ascontiguousarray(vox, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(vox.shape[0])
    _load().or_back_voxels(ctypes.byref(c.g), _dp(proj), _dp(c.poses), c.n_inst, _ip(c.iv), _ip(c.ip),
                           int(weight), int(vox.shape[0]), _ip(vox), _dp(out))
    return out


# ------------------------------------------------------- FDK and sharpness

def ramlak_taps(n):
    """Ram-Lak ramp kernel h[k], k = -(n-1)..(n-1), in units of 1/du^2:
    1/4 at 0, -1/(pi k)^2 at odd k, 0 at even k != 0."""
    k = np.arange(-(n - 1), n)
    h = np.zeros(k.shape)
    h[k == 0] = 0.25
    odd = (k % 2) != 0
    h[odd] = -1.0 / (np.pi * k[odd]) ** 2
    return k, h


def fdk_constants(view, nu, nv):
    """SAD (source to the isocentre plane parallel to the detector), pixel
    pitches on that plane and the principal point in pixel indices."""
    s, c, U, V = view[0:3], view[3:6], view[6:9], view[9:12]
    n = np.cross(U, V)
    n = n / np.linalg.norm(n)
    if np.dot(c - s, n) < 0:
        n = -n
    sdd = np.dot(c - s, n)
    sad = np.dot(-s, n)
    P = projection_matrix(view, nu, nv)
    h = P[:, :3] @ (s + n) + P[:, 3]
    return sad, np.linalg.norm(U) * sad / sdd, np.linalg.norm(V) * sad / sdd, h[0] / h[2], h[1] / h[2]


def fdk_filter(geom, proj, inst_view, scale):
    """Cosine pre-weight and Ram-Lak filtering along detector rows (the
    Ramp(l) of Sec. II-D.3's motion-compensated reconstruction): per
    instance, x = l * SAD / sqrt(SAD^2 + a^2 + b^2), q = scale * du * (x conv h),
    h in units of 1/du^2 (du the pitch on the isocentre plane)."""
    proj = np.asarray(proj, dtype=np.float64)
    out = np.zeros_like(proj)
    nu, nv = geom.nu, geom.nv
    _, h = ramlak_taps(nu)
    idx = np.arange(nu)
    T = h[(idx[:, None] - idx[None, :]) + (nu - 1)]      # T[u, k] = h[u - k]
    for n, vi in enumerate(inst_view):
        sad, du, dv, pu, pv = fdk_constants(geom.views[vi], nu, nv)
        a = (idx - pu) * du
        b = (np.arange(nv) - pv) * dv
        w = sad / np.sqrt(sad ** 2 + a[None, :] ** 2 + b[:, None] ** 2)
        x = proj[n] * w
        out[n] = scale * du * (x @ T.T) / du ** 2
    return out


def _central(mu, vox):
    m = np.pad(np.asarray(mu, dtype=np.float64), 1)
    gz = (m[2:, 1:-1, 1:-1] - m[:-2, 1:-1, 1:-1]) / (2 * vox[2])
    gy = (m[1:-1, 2:, 1:-1] - m[1:-1, :-2, 1:-1]) / (2 * vox[1])
    gx = (m[1:-1, 1:-1, 2:] - m[1:-1, 1:-1, :-2]) / (2 * vox[0])
    return gx, gy, gz


def sharpness(mu, vox):
    """S = -Var(|grad mu|) with central differences of the zero-padded
    volume (per mm) and the population variance over all voxels."""
    gx, gy, gz = _central(mu, vox)
    m = np.sqrt(gx * gx + gy * gy + gz * gz)
    return float(-(np.mean(m * m) - np.mean(m) ** 2))


def sharpness_grad(mu, vox):
    """dS/dmu by the chain rule through m_i = |g(i)| and the central
    differences; voxels with m_i < 1e-12 contribute no direction."""
    gx, gy, gz = _central(mu, vox)
    m = np.sqrt(gx * gx + gy * gy + gz * gz)
    N = m.size
    safe = np.where(m >= 1e-12, m, 1.0)
    coef = np.where(m >= 1e-12, (m - m.mean()) / safe, 0.0) * (-2.0 / N)
    grad = np.zeros(m.shape)
    for g_a, axis, h in ((gx, 2, vox[0]), (gy, 1, vox[1]), (gz, 0, vox[2])):
        c = np.pad(coef * g_a / (2 * h), 1)          # dS/dg_a(i) / (2 v_a), zero outside
        sl_minus = [slice(1, -1)] * 3
        sl_plus = [slice(1, -1)] * 3
        sl_minus[axis] = slice(0, -2)                 # neighbour i = j - e_a: g_a(i) has +mu_j
        sl_plus[axis] = slice(2, None)                # neighbour i = j + e_a: g_a(i) has -mu_j
        grad += c[tuple(sl_minus)] - c[tuple(sl_plus)]
    return grad


# ------------------------------------------------------------------ losses

def l2_loss(a, b):
    """L = sum (a - b)^2 and dL/da (Eq. forward_loss / back_loss)."""
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    return float(np.sum(d * d)), 2.0 * d


def ncc(a, b):
    """Pearson correlation of two images (two-pass form)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    da, db = a - a.mean(), b - b.mean()
    return float(np.dot(da, db) / np.sqrt(np.dot(da, da) * np.dot(db, db)))


def ncc_grad(a, b):
    """NCC(a, b) and dNCC/da (two-pass form):
    dNCC/da_i = (b_i - mean b)/sqrt(Saa Sbb) - A (a_i - mean a)/(Saa^1.5 Sbb^0.5)
    with A = sum (a-ma)(b-mb), Saa = sum (a-ma)^2, Sbb = sum (b-mb)^2."""
    shape = np.shape(a)
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    da, db = a - a.mean(), b - b.mean()
    A, Saa, Sbb = np.dot(da, db), np.dot(da, da), np.dot(db, db)
    g = db / np.sqrt(Saa * Sbb) - A * da / (Saa ** 1.5 * Sbb ** 0.5)
    return float(A / np.sqrt(Saa * Sbb)), g.reshape(shape)


def pose_loss_weights(kind, proj, target, inst_view, inst_pose, n_pose):
    """Per-pose loss and dL/dl for every instance.

    kind 'l2':  L_p = sum over the pose's instances of sum (l - b)^2.
    kind 'ncc': L_p = -(1/n_p) sum over the pose's instances of NCC(l, b).
    target is indexed by physical view; proj by instance."""
    loss = np.zeros(n_pose)
    w = np.zeros_like(np.asarray(proj, dtype=np.float64))
    counts = np.bincount(np.asarray(inst_pose), minlength=n_pose)
    for n in range(len(inst_view)):
        a, b = proj[n], target[inst_view[n]]
        p = inst_pose[n]
        if kind == "l2":
            L, g = l2_loss(a, b)
            loss[p] += L
            w[n] = g
        elif kind == "ncc":
            L, g = ncc_grad(a, b)
            loss[p] -= L / counts[p]
            w[n] = -g / counts[p]
        else:
            raise ValueError(kind)
    return loss, w


def cosine(a, b):
    """Cosine similarity d(g_p, g_t) of two gradient vectors (Sec. II-D.1)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.dot(a, b) / np.sqrt(np.dot(a, a) * np.dot(b, b)))

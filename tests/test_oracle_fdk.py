"""Pins of the FDK filtering and sharpness functions of the oracle (the
motion-compensated reconstruction experiment, Sec. II-D.3)."""
import numpy as np

import oracle
import synth
from helpers import central_fd


def test_ramlak_transfer_function_is_the_ramp():
    """DTFT of the spatial Ram-Lak kernel = |w| / (2 pi) (in units of 1/du^2),
    up to the truncation of the kernel."""
    k, h = oracle.ramlak_taps(4096)
    for w in np.linspace(-np.pi, np.pi, 13):
        H = float(np.sum(h * np.cos(w * k)))
        assert abs(H - abs(w) / (2 * np.pi)) < 1e-4, (w, H)


def test_fdk_reconstructs_a_ball_from_its_chord_lengths():
    """Projections of a uniform ball (analytic chord lengths) on a full
    circular orbit, filtered and back-projected with the FDK weight and
    scale pi / n_views, reconstruct the ball's attenuation near its centre."""
    n_views, nd, pix = 90, 96, 1.0
    views = synth.circular_views(n_views, 300.0, 450.0, pix, pix)
    g = synth.Geometry(33, 33, 33, 1.0, 1.0, 1.0, nd, nd, views, 0.5)
    mu0, rad = 0.02, 12.0
    proj = np.zeros((n_views, nd, nd))
    iu, iv = np.meshgrid(np.arange(nd), np.arange(nd))
    for vi in range(n_views):
        s, c, U, V = views[vi, :3], views[vi, 3:6], views[vi, 6:9], views[vi, 9:12]
        q = c + (iu[..., None] - (nd - 1) / 2) * U + (iv[..., None] - (nd - 1) / 2) * V
        d = q - s
        d = d / np.linalg.norm(d, axis=-1, keepdims=True)
        along = -(s @ d.reshape(-1, 3).T).reshape(nd, nd)
        dist2 = s @ s - along ** 2
        proj[vi] = mu0 * 2 * np.sqrt(np.clip(rad ** 2 - dist2, 0, None))
    q = oracle.fdk_filter(g, proj, np.arange(n_views), np.pi / n_views)
    vol = oracle.back(g, q, np.zeros(6), weight=oracle.W_FDK)
    centre = vol[12:21, 12:21, 12:21]
    assert abs(centre.mean() / mu0 - 1) < 0.03, centre.mean() / mu0
    assert abs(vol[16, 16, 1]) < 0.2 * mu0


def test_sharpness_matches_its_definition_and_gradient():
    rng = np.random.default_rng(51)
    mu = rng.uniform(0, 1, (7, 6, 8))
    vox = (1.0, 1.2, 0.9)
    gx = np.gradient(np.pad(mu, 1), vox[0], axis=2)[1:-1, 1:-1, 1:-1]
    gy = np.gradient(np.pad(mu, 1), vox[1], axis=1)[1:-1, 1:-1, 1:-1]
    gz = np.gradient(np.pad(mu, 1), vox[2], axis=0)[1:-1, 1:-1, 1:-1]
    m = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2)
    assert abs(oracle.sharpness(mu, vox) + np.var(m)) < 1e-14
    g = oracle.sharpness_grad(mu, vox)
    h = 1e-6
    for _ in range(20):
        idx = tuple(rng.integers(0, s) for s in mu.shape)
        e = np.zeros_like(mu)
        e[idx] = h
        fd = (oracle.sharpness(mu + e, vox) - oracle.sharpness(mu - e, vox)) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8 * max(1.0, abs(fd)), (idx, fd, g[idx])

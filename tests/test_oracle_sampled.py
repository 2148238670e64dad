"""The sampled-output oracle entry points agree with the full ones (they
apply the same definitions to a subset of rays / voxels)."""
import numpy as np

import oracle
from helpers import small_geom, smooth_volume


def test_forward_pixels_match_full_forward():
    rng = np.random.default_rng(41)
    g = small_geom(n=(14, 12, 16), det=(20, 18), n_views=3)
    mu = smooth_volume(g, rng)
    poses = np.array([[1.0, -0.5, 0.3, 0.1, 0.2, -0.3], [0.0, 1.0, 0.0, -0.2, 0.0, 0.4]])
    iv, ip = [0, 1, 2], [0, 1, 1]
    full = oracle.forward(g, mu, poses, iv, ip)
    pix = np.stack([rng.integers(0, 3, 50), rng.integers(0, g.nu, 50), rng.integers(0, g.nv, 50)], axis=1)
    got = oracle.forward_pixels(g, mu, poses, pix, iv, ip)
    np.testing.assert_array_equal(got, full[pix[:, 0], pix[:, 2], pix[:, 1]])


def test_back_voxels_match_full_back():
    rng = np.random.default_rng(42)
    g = small_geom(n=(10, 12, 9), det=(15, 13), n_views=2)
    poses = np.array([[0.5, -0.5, 0.3, 0.1, 0.2, -0.3], [0.0, 1.0, 0.0, -0.2, 0.0, 0.4]])
    y = rng.standard_normal((2, g.nv, g.nu))
    for weight in (oracle.W_NONE, oracle.W_FDK):
        full = oracle.back(g, y, poses, [0, 1], [0, 1], weight=weight)
        vox = np.stack([rng.integers(0, g.nx, 40), rng.integers(0, g.ny, 40), rng.integers(0, g.nz, 40)], axis=1)
        got = oracle.back_voxels(g, y, poses, vox, [0, 1], [0, 1], weight=weight)
        np.testing.assert_allclose(got, full[vox[:, 2], vox[:, 1], vox[:, 0]], rtol=1e-13, atol=1e-13)

"""Pins of the oracle's losses: L2 (Eq. forward_loss) and the NCC used for
registration (Sec. II-D.3), including the single-pass moment form of the
NCC gradient that the fused kernel evaluates."""
import numpy as np

import oracle


def test_ncc_matches_numpy_corrcoef():
    rng = np.random.default_rng(31)
    a, b = rng.uniform(0, 2, (17, 13)), rng.uniform(0, 2, (17, 13))
    assert abs(oracle.ncc(a, b) - np.corrcoef(a.ravel(), b.ravel())[0, 1]) < 1e-14
    assert abs(oracle.ncc(a, 3 * a + 1) - 1.0) < 1e-14
    assert abs(oracle.ncc(a, -a) + 1.0) < 1e-14


def test_ncc_gradient_matches_finite_differences():
    rng = np.random.default_rng(32)
    a, b = rng.uniform(0, 2, 40), rng.uniform(0, 2, 40)
    _, g = oracle.ncc_grad(a, b)
    h = 1e-6
    for i in range(40):
        e = np.zeros(40)
        e[i] = h
        fd = (oracle.ncc(a + e, b) - oracle.ncc(a - e, b)) / (2 * h)
        assert abs(fd - g[i]) < 1e-8


def test_single_pass_moment_form_equals_two_pass():
    """sum_i dNCC/da_i G_i from the moments S_a, S_aa, S_ab, S_b, S_bb, n and
    the three weighted sums sum G, sum a G, sum b G equals the two-pass
    residual form (G_i: arbitrary per-pixel 12-vectors)."""
    rng = np.random.default_rng(33)
    n = 500
    a, b = rng.uniform(0, 3, n), rng.uniform(1, 2, n)
    G = rng.standard_normal((n, 12))
    _, w = oracle.ncc_grad(a, b)
    two_pass = w @ G
    Sa, Saa, Sab, Sb, Sbb = a.sum(), a @ a, a @ b, b.sum(), b @ b
    ma, mb = Sa / n, Sb / n
    A = Sab - n * ma * mb
    Va = Saa - n * ma * ma
    Vb = Sbb - n * mb * mb
    SG, SaG, SbG = G.sum(0), a @ G, b @ G
    one_pass = (SbG - mb * SG) / np.sqrt(Va * Vb) - A * (SaG - ma * SG) / (Va ** 1.5 * Vb ** 0.5)
    np.testing.assert_allclose(one_pass, two_pass, rtol=1e-12, atol=1e-12 * np.abs(two_pass).max())


def test_pose_loss_weights_average_ncc_over_instances():
    rng = np.random.default_rng(34)
    proj = rng.uniform(0, 1, (4, 6, 5))
    target = rng.uniform(0, 1, (2, 6, 5))
    iv, ip = [0, 1, 0, 1], [0, 0, 1, 1]
    loss, w = oracle.pose_loss_weights("ncc", proj, target, iv, ip, 2)
    assert abs(loss[0] + 0.5 * (oracle.ncc(proj[0], target[0]) + oracle.ncc(proj[1], target[1]))) < 1e-14
    h = 1e-6
    for n in range(4):
        for k in range(5):
            e = np.zeros_like(proj)
            e[n, 0, k] = h
            lp, _ = oracle.pose_loss_weights("ncc", proj + e, target, iv, ip, 2)
            lm, _ = oracle.pose_loss_weights("ncc", proj - e, target, iv, ip, 2)
            assert abs((lp - lm).sum() / (2 * h) - w[n, 0, k]) < 1e-8
    loss2, w2 = oracle.pose_loss_weights("l2", proj, target, iv, ip, 2)
    assert abs(loss2[1] - np.sum((proj[2] - target[0]) ** 2) - np.sum((proj[3] - target[1]) ** 2)) < 1e-12
    np.testing.assert_allclose(w2[3], 2 * (proj[3] - target[1]))

"""Pins of the network oracle (CPU): the convolution against SciPy's 2-D
cross-correlation (an independent library routine), every gradient against
central finite differences, and the input preparation against closed forms."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import posenet as on


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    for H, W in ((8, 8), (7, 10)):
        x = rng.standard_normal((2, H, W, 3))
        w = rng.standard_normal((4, 3, 3, 3))
        b = rng.standard_normal(4)
        y = on.conv3x3s2(x, w, b)
        assert y.shape == (2, (H + 1) // 2, (W + 1) // 2, 4)
        for bb in range(2):
            for o in range(4):
                ref = b[o] + sum(correlate2d(np.pad(x[bb, :, :, i], 1), w[o, :, :, i], mode="valid")
                                 for i in range(3))
                np.testing.assert_allclose(y[bb, :, :, o], ref[::2, ::2], rtol=1e-12, atol=1e-12)


def test_conv_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 5, 6, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    g = rng.standard_normal(on.conv3x3s2(x, w, b).shape)
    dx, dw, db = on.conv3x3s2_grad(x, w, g)

    def f(xx, ww, bb):
        return float(np.sum(on.conv3x3s2(xx, ww, bb) * g))

    h = 1e-6
    for arr, grad, args in ((x, dx, lambda a: (a, w, b)), (w, dw, lambda a: (x, a, b)), (b, db, lambda a: (x, w, a))):
        idx = [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(12)]
        for i in idx:
            e = np.zeros_like(arr)
            e[i] = h
            fd = (f(*args(arr + e)) - f(*args(arr - e))) / (2 * h)
            assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def tiny_params(rng):
    return dict(conv=[(0.5 * rng.standard_normal((4, 3, 3, 2)), 0.1 * rng.standard_normal(4)),
                      (0.3 * rng.standard_normal((8, 3, 3, 4)), 0.1 * rng.standard_normal(8))],
                fc=[(0.2 * rng.standard_normal((5, 8 * 2 * 2)), 0.1 * rng.standard_normal(5)),
                    (0.3 * rng.standard_normal((3, 5)), 0.1 * rng.standard_normal(3))])


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    P = tiny_params(rng)
    x = rng.standard_normal((3, 8, 8, 2))
    t = rng.standard_normal((3, 3))

    def loss(params, xx=x):
        out, _ = on.net_forward(params, xx)
        return on.mse(out, t)[0]

    out, cache = on.net_forward(P, x)
    _, dout = on.mse(out, t)
    G = on.net_backward(P, cache, dout)
    h = 1e-6
    checks = [("conv", 0, 0), ("conv", 1, 0), ("conv", 0, 1), ("fc", 0, 0), ("fc", 1, 1), ("fc", 1, 0)]
    for kind, l, j in checks:
        arr = P[kind][l][j]
        for _ in range(6):
            i = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[i]
            arr[i] = old + h
            lp = loss(P)
            arr[i] = old - h
            lm = loss(P)
            arr[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[kind][l][j][i]) <= 1e-5 * max(1e-3, abs(fd)) + 1e-9, (kind, l, j, i)
    # input gradient
    for _ in range(6):
        i = tuple(rng.integers(0, s) for s in x.shape)
        e = np.zeros_like(x)
        e[i] = h
        fd = (loss(P, x + e) - loss(P, x - e)) / (2 * h)
        assert abs(fd - G["input"][i]) <= 1e-5 * max(1e-3, abs(fd)) + 1e-9


def test_mse_gradient():
    rng = np.random.default_rng(3)
    y, t = rng.standard_normal((4, 6)), rng.standard_normal((4, 6))
    L, g = on.mse(y, t)
    assert L == pytest.approx(np.sum((y - t) ** 2) / 24)
    e = np.zeros_like(y)
    e[1, 2] = 1e-6
    assert (on.mse(y + e, t)[0] - on.mse(y - e, t)[0]) / 2e-6 == pytest.approx(g[1, 2], rel=1e-6)


def test_prepare_closed_forms():
    # a constant image maps to zeros; a ramp in u, box-averaged over 3 x 3,
    # is the ramp of the block centres, and standardising a ramp of n equal
    # steps gives (k - (n-1)/2) / sqrt((n^2 - 1)/12)
    nu = nv = 12
    const = np.full((2, nv, nu), 3.5)
    ramp = np.tile(np.arange(nu, dtype=np.float64), (nv, 1))[None].repeat(2, 0)
    z = on.prepare(np.concatenate([const, ramp]), 2, 3)
    assert z.shape == (2, 4, 4, 2)
    np.testing.assert_allclose(z[0], 0.0, atol=0)
    n = 4
    k = np.arange(n)
    expect = (k - (n - 1) / 2) / np.sqrt((n * n - 1) / 12.0)
    for c in range(2):
        np.testing.assert_allclose(z[1, :, :, c], np.tile(expect, (4, 1)), rtol=1e-12)


def test_bf16_round_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    vals = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-20, 20, 20000),
                           # exact ties: bit patterns with the dropped half exactly 0x8000
                           (np.arange(1, 2001, dtype=np.uint32) << 16 | 0x8000).view(np.float32).astype(np.float64),
                           [0.0, -0.0, 1.0, -1.5, 3.0e38]])
    ref = torch.from_numpy(vals.astype(np.float32)).bfloat16().float().numpy().astype(np.float64)
    np.testing.assert_array_equal(on.bf16_round(vals), ref)


def test_bf16_network_rounds_only_stored_values():
    """With bf16=True every stored activation is a BF16 value; without it
    the result equals the plain network; the two differ by BF16-sized
    amounts."""
    rng = np.random.default_rng(5)
    P = tiny_params(rng)
    x = on.bf16_round(rng.standard_normal((2, 8, 8, 2)))
    out_f, cache_f = on.net_forward(P, x)
    out_b, cache_b = on.net_forward(P, x, bf16=True)
    for a in cache_b["acts"][1:] + cache_b["fcs"][1:-1]:
        np.testing.assert_array_equal(a, on.bf16_round(a))
    assert 0 < np.linalg.norm(out_b - out_f) <= 2e-2 * np.linalg.norm(out_f)
    g_b = on.net_backward(P, cache_b, np.ones_like(out_b), bf16=True)
    g_f = on.net_backward(P, cache_f, np.ones_like(out_f))
    for (a, _), (b, _) in zip(g_b["conv"], g_f["conv"]):
        assert np.linalg.norm(a - b) <= 0.1 * np.linalg.norm(b)

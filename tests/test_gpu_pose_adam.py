"""proj_pose_adam (the optimiser of the registration and motion-compensation
loops) against Adam written out in numpy: per-parameter step sizes, per-pose
step counts, masked poses left untouched.  FP32 arithmetic against FP64:
rel <= 1e-5 after five steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()


import paper_2508_13304_b300 as pb  # noqa: E402


def adam_numpy(pose, grads, masks, lr, b1, b2, eps):
    n = pose.shape[0]
    m = np.zeros((n, 6))
    v = np.zeros((n, 6))
    t = np.zeros(n)
    p = pose.copy()
    for g, a in zip(grads, masks):
        for i in range(n):
            if not a[i]:
                continue
            t[i] += 1
            m[i] = b1 * m[i] + (1 - b1) * g[i]
            v[i] = b2 * v[i] + (1 - b2) * g[i] ** 2
            p[i] -= lr * (m[i] / (1 - b1 ** t[i])) / (np.sqrt(v[i] / (1 - b2 ** t[i])) + eps)
    return p, m, v, t


def test_pose_adam_matches_numpy():
    rng = np.random.default_rng(4)
    n = 37
    lr = np.array([10.0, 10.0, 10.0, 0.035, 0.035, 0.035])
    b1, b2, eps = 0.9, 0.999, 1e-8
    pose0 = rng.standard_normal((n, 6)).astype(np.float32)
    grads = [rng.standard_normal((n, 6)).astype(np.float32) for _ in range(5)]
    masks = [rng.uniform(size=n) < 0.7 for _ in range(5)]
    masks[0][:] = True
    pose = torch.from_numpy(pose0).cuda()
    m = torch.zeros((n, 6), device="cuda")
    v = torch.zeros((n, 6), device="cuda")
    t = torch.zeros(n, device="cuda")
    for g, a in zip(grads, masks):
        pb.proj_pose_adam(pose, torch.from_numpy(g).cuda(), m, v, t, torch.from_numpy(a).cuda(), lr, b1, b2, eps)
    torch.cuda.synchronize()
    # the ABI takes b1, b2 as FP32 values (0.999 -> 0.99900001287), so 1 - b2 is that of the FP32 value
    p_ref, m_ref, v_ref, t_ref = adam_numpy(pose0.astype(np.float64), [g.astype(np.float64) for g in grads], masks,
                                            lr.astype(np.float32).astype(np.float64), float(np.float32(b1)),
                                            float(np.float32(b2)), eps)
    np.testing.assert_array_equal(t.cpu().numpy(), t_ref)
    got = pose.cpu().numpy()
    step = got - pose0
    assert np.linalg.norm(step - (p_ref - pose0)) <= 1e-5 * np.linalg.norm(p_ref - pose0)
    assert np.linalg.norm(m.cpu().numpy() - m_ref) <= 1e-5 * np.linalg.norm(m_ref)
    assert np.linalg.norm(v.cpu().numpy() - v_ref) <= 1e-5 * np.linalg.norm(v_ref)
    never = ~np.any(np.stack(masks), axis=0)
    assert np.array_equal(got[never], pose0[never])


def test_pose_adam_all_active_and_arguments():
    pose = torch.zeros((3, 6), device="cuda")
    g = torch.ones((3, 6), device="cuda")
    m, v, t = torch.zeros((3, 6), device="cuda"), torch.zeros((3, 6), device="cuda"), torch.zeros(3, device="cuda")
    pb.proj_pose_adam(pose, g, m, v, t, None, [1.0] * 6)
    torch.cuda.synchronize()
    # first step of Adam moves every parameter by lr * g / (|g| + eps)
    assert np.allclose(pose.cpu().numpy(), -1.0, atol=1e-6)
    assert np.array_equal(t.cpu().numpy(), [1.0, 1.0, 1.0])
    with pytest.raises(pb.ProjError):
        pb.proj_pose_adam(pose, g, m, v, t, None, [1.0] * 6, b1=1.0)

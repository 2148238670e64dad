"""proj_registration_step (one launch per registration iteration) against the
same bookkeeping written with torch operations: hit test, stopping rules,
masked Adam step (proj_pose_adam, the same arithmetic), loss history and the
refill of the slots of stopped starts.  Every state tensor must agree bit
for bit over a sequence of iterations with random losses and gradients that
trigger every stopping rule."""
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


def reference_step(st, grad, loss, tp, tol, ncc_stop, dloss_stop, max_iter, lr):
    n = st["pose"].shape[0]
    sl = st["slots"].long()
    listed = torch.zeros(n + 1, dtype=torch.bool, device="cuda")
    listed.index_fill_(0, torch.where(sl >= 0, sl, n), True)
    listed = listed[:n]
    if tp is not None:
        d = (st["pose"] - tp).abs()
        hit = listed & (d[:, :3].amax(1) <= tol[0]) & ((d[:, 3:] * 57.295779513082321).amax(1) <= tol[1])
        st["hit"].logical_or_(hit.any())
    done = listed & ((-loss >= ncc_stop) | ((st["last"] - loss).abs() < dloss_stop) | (st["iters"] >= max_iter))
    st["alive"].logical_and_(~done)
    upd = st["alive"] & listed
    st["iters"].add_(upd)
    pb.proj_pose_adam(st["pose"], grad, st["m"], st["v"], st["t"], upd, lr)
    st["last"].copy_(torch.where(listed, loss, st["last"]))
    free = (sl < 0) | ~st["alive"][sl.clamp(min=0)]
    cand = st["next"] + torch.cumsum(free.long(), 0) - 1
    take = free & (cand < n)
    st["slots"].copy_(torch.where(take, cand, torch.where(free, torch.full_like(cand, -1), sl)).int())
    st["next"].add_(take.long().sum())


def fresh_state(pose0, n_slots):
    n = pose0.shape[0]
    return {"pose": pose0.clone(), "m": torch.zeros((n, 6), device="cuda"), "v": torch.zeros((n, 6), device="cuda"),
            "t": torch.zeros(n, device="cuda"), "alive": torch.ones(n, dtype=torch.bool, device="cuda"),
            "iters": torch.zeros(n, dtype=torch.int64, device="cuda"),
            "last": torch.full((n,), float("inf"), device="cuda"),
            "slots": torch.arange(n_slots, dtype=torch.int32, device="cuda"),
            "next": torch.full((), n_slots, dtype=torch.int64, device="cuda"),
            "hit": torch.zeros((), dtype=torch.bool, device="cuda")}


@pytest.mark.parametrize("n,n_slots,n_truth", [(13, 4, 1), (13, 13, 13), (40, 7, 0), (1, 1, 1)])
def test_registration_step_matches_torch_bookkeeping(n, n_slots, n_truth):
    rng = np.random.default_rng(n * 100 + n_slots)
    lr = [10.0, 10.0, 10.0, 0.035, 0.035, 0.035]
    ncc_stop, dloss_stop, max_iter, tol = 0.999, 1e-5, 9, (2.0, 3.0)
    pose0 = torch.from_numpy(rng.standard_normal((n, 6)).astype(np.float32)).cuda()
    tp = None
    if n_truth:
        tp = torch.from_numpy((rng.standard_normal((n_truth, 6)) * 0.5).astype(np.float32)).cuda()
    params = pb.reg_params(lr, 0.9, 0.999, 1e-8, ncc_stop, dloss_stop, max_iter, tol)
    a, b = fresh_state(pose0, n_slots), fresh_state(pose0, n_slots)
    listed = torch.zeros(n, dtype=torch.bool, device="cuda")
    prev = None
    for it in range(14):
        loss = -rng.uniform(0.5, 0.998, n)
        loss[rng.uniform(size=n) < 0.08] = -0.9995                       # NCC above the stop
        if prev is not None:
            same = rng.uniform(size=n) < 0.08
            loss[same] = prev[same]                                       # no loss change
        prev = loss.copy()
        loss_d = torch.from_numpy(loss.astype(np.float32)).cuda()
        grad = torch.from_numpy(rng.standard_normal((n, 6)).astype(np.float32)).cuda()
        reference_step(a, grad, loss_d, tp, tol, ncc_stop, dloss_stop, max_iter, lr)
        pb.proj_registration_step(b["pose"], grad, loss_d, b["last"], b["m"], b["v"], b["t"], b["alive"],
                                  b["iters"], b["slots"], b["next"], tp, b["hit"] if tp is not None else None,
                                  listed, params)
        torch.cuda.synchronize()
        for k in a:
            assert torch.equal(a[k], b[k]), (it, k, a[k], b[k])
    assert int(b["next"]) <= n

"""Streams and graphs.  Two plans with their own workspaces on two CUDA streams, launched
interleaved so that their kernels can overlap: every result equals the one
of the same calls run one after another on the default stream (the library
keeps no state outside the plan and the caller's workspace)."""
import numpy as np
import pytest

from helpers import small_geom, smooth_volume

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_13304_b300 import build
    build.build()


import paper_2508_13304_b300 as pb  # noqa: E402


def make(seed, n, det, n_views, n_pose):
    rng = np.random.default_rng(seed)
    g = small_geom(n=n, det=det, pix=1.5, n_views=n_views)
    mu = torch.from_numpy(smooth_volume(g, rng, n_blobs=6).astype(np.float32)).cuda()
    iv = np.tile(np.arange(n_views), n_pose).astype(np.int32)
    ip = np.repeat(np.arange(n_pose), n_views).astype(np.int32)
    P = pb.Projector(g, n_pose=n_pose, inst_view=iv, inst_pose=ip)
    pose = torch.from_numpy(np.concatenate([rng.uniform(-2, 2, (n_pose, 3)), rng.uniform(-0.1, 0.1, (n_pose, 3))],
                                           axis=1).astype(np.float32)).cuda()
    ref = torch.from_numpy(rng.uniform(0, 1, (n_views, g.nv, g.nu)).astype(np.float32)).cuda()
    img = torch.from_numpy(rng.uniform(0, 1, (len(iv), g.nv, g.nu)).astype(np.float32)).cuda()
    wv = torch.from_numpy(rng.standard_normal(g.vol_shape).astype(np.float32)).cuda()
    return dict(P=P, g=g, mu=mu, pose=pose, ref=ref, img=img, wv=wv, n_pose=n_pose, n_inst=len(iv))


def run(c, stream):
    P, g = c["P"], c["g"]
    out = dict(grad=torch.empty((c["n_pose"], 6), device="cuda"), loss=torch.empty(c["n_pose"], device="cuda"),
               proj=torch.empty((c["n_inst"], g.nv, g.nu), device="cuda"),
               vol=torch.empty((g.nz, g.ny, g.nx), device="cuda"),
               bgrad=torch.empty((c["n_pose"], 6), device="cuda"))
    pb.proj_set_volume(P.plan, c["mu"], P.ws, stream=stream)
    pb.proj_forward_pose_grad(P.plan, c["pose"], pb.PROJ_LOSS_NCC, c["ref"], out["grad"], out["loss"], out["proj"],
                              P.ws, stream=stream)
    pb.proj_back(P.plan, c["img"], c["pose"], pb.PROJ_W_FDK, out["vol"], P.ws, stream=stream)
    pb.proj_back_pose_grad(P.plan, c["img"], c["pose"], pb.PROJ_W_FDK, c["wv"], out["bgrad"], P.ws, stream=stream)
    return out


def test_two_plans_on_two_streams_match_sequential_runs():
    a = make(1, (44, 40, 36), (50, 42), 3, 2)
    b = make(2, (30, 34, 38), (37, 45), 2, 3)
    seq = [run(a, None), run(b, None)]
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        oa = run(a, s1)
    with torch.cuda.stream(s2):
        ob = run(b, s2)
    torch.cuda.synchronize()
    for got, want in ((oa, seq[0]), (ob, seq[1])):
        for k in ("grad", "loss", "proj", "vol", "bgrad"):
            assert torch.equal(got[k], want[k]), k


def test_calls_replay_from_a_cuda_graph():
    """Every hot-path call is asynchronous and allocation-free, so a step of
    them can be captured once and replayed; the replay reproduces the eager
    results bit for bit."""
    c = make(3, (40, 36, 42), (48, 40), 2, 2)
    want = run(c, None)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run(c, s)                            # warm-up on the capture stream
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        got = run(c, s)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    for k in ("grad", "loss", "proj", "vol", "bgrad"):
        assert torch.equal(got[k], want[k]), k

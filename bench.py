#!/usr/bin/env python
"""Benchmark of the batched 2D/3D registration step.

Workload (synthetic, seeded): a 256^3 FP32 phantom at 0.8 mm (ten ellipsoids
plus two high-contrast cylinders), two views 90 deg apart on 384 x 384
detectors at 0.8 mm, SAD 800 / SDD 1200 mm, ray step 0.4 mm, 64 candidate
poses (rot +-15 deg, trans +-20 mm).  One step = prepare the volume
(grad mu stencil) + the fused NCC pose-gradient march of all 64 x 2 view
instances + the deterministic reduction: 64 pose-gradient evaluations.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import csv
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "pose-gradient evals/s & ray-samples/s, batched vs plain, at ≤1e-3 grad err"
UNIT = "pose-gradient evals/s"
FLOP_PER_SAMPLE = 95      # FP32 work of one gathered fused-march sample: trilinear weights 15, 4 channels x (1 mul + 7 FMA) 60, position 6, fractions 3, sample offset 1, accumulation 10
L1_BYTES_PER_SAMPLE = 128  # 8 trilinear corners x float4 (mu, grad mu) delivered to registers
L1_BYTES_PER_CLK_SM = 128  # L1 data-pipe width per SM per clock
L2_FLUSH_BYTES = 256 << 20
# Counters of the fused march from ncu captures (they cannot be read live):
# the L1 data-pipe wavefront utilisation of the 8-instance case, and the DRAM
# bytes (read + write) of one full-size launch of this workload taken with
# one-pass metrics.  NCU_SOURCE_SHA16 is the hash (kernel_source_sha16) of
# the march's sources they were taken on; when the built sources hash
# differently the line reports them as null.
NCU_SOURCE_SHA16 = "c9f6b15863013dad"
NCU_L1_WAVEFRONT_PCT = 58.7
NCU_ISSUE_ACTIVE_PCT = 55.9
TRAFFIC_PER_LAUNCH = 78.98e6  # 70.19 MB read + 8.79 MB written
MARCH_SOURCES = ("paper_2508_13304_b300/csrc/proj_forward.cu", "paper_2508_13304_b300/csrc/proj_internal.cuh")


def kernel_source_sha16():
    """First 16 hex digits of the SHA-256 of the fused march's source files."""
    import hashlib
    h = hashlib.sha256()
    for f in MARCH_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-cand", type=int, default=64)
    ap.add_argument("--cpu-sample", type=int, default=8,
                    help="candidates timed on the CPU oracle (about 1.5 s of 16-core FP64 work each)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the other kernels' measurements")
    ap.add_argument("--section", default=None,
                    choices=["gemm", "forward", "back", "accuracy", "tables", "registration500", "moco", "c1",
                             "batch"],
                    help="run only one secondary measurement and print it (gemm: the tensor-core GEMM shapes; "
                         "forward: forward projection of the 128 registration instances; back: FDK "
                         "back-projection and its pose gradient, 360 views of 512^2 on 256^3; batch: the "
                         "uneven single-view problems in one persistent launch)")
    ap.add_argument("--batch-problems", type=int, default=24,
                    help="--section batch: how many of the 24 single-view problems")
    ap.add_argument("--posenet-eval", action="store_true",
                    help="also train the pose-proposal network on 200k DRRs and compare proposal + registration "
                         "with 16-start registration (about 3 minutes)")
    return ap.parse_args()


def workload(n_cand):
    w = synth.workload_registration(n_cand=n_cand)
    w["mu"] = np.ascontiguousarray(w["mu"], dtype=np.float32)
    w["poses"] = np.ascontiguousarray(w["poses"], dtype=np.float32)
    w["pose_true"] = np.ascontiguousarray(w["pose_true"], dtype=np.float32)
    return w


def instance_maps(n_cand, n_views):
    iv = np.tile(np.arange(n_views, dtype=np.int32), n_cand)
    ip = np.repeat(np.arange(n_cand, dtype=np.int32), n_views)
    return iv, ip


# ------------------------------------------------------------------ clocks

class NvmlClockSampler:
    """SM clock, power and clock-event reasons read through NVML (the driver's
    libnvidia-ml, called with ctypes) every 10 ms in a thread during the timed
    region: read-only queries, so short timed regions still get many samples.
    Same summary as ClockSampler."""

    # clock-event reason bits of nvmlDeviceGetCurrentClocksEventReasons (nvml.h)
    BITS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20, "sw_power_cap": 0x4}

    def __init__(self, torch_device):
        import ctypes
        import threading
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.lib, self.ct = lib, ctypes
        prop = __import__("torch").cuda.get_device_properties(torch_device)
        h = ctypes.c_void_p()
        bus = b"%08x:%02x:%02x.0" % (prop.pci_domain_id, prop.pci_bus_id, prop.pci_device_id)
        if lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) != 0:
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(torch_device.index or 0), ctypes.byref(h)) != 0:
                raise OSError("no NVML handle")
        self.h = h
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) != 0:  # 1 = NVML_CLOCK_SM
            raise OSError("nvmlDeviceGetMaxClockInfo failed")
        self.smax = float(mx.value)
        self.rows, self.stop = [], threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        ct, lib, h = self.ct, self.lib, self.h
        sm, pw, rs = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, ct.c_int(1), ct.byref(sm)) == 0 and
                    lib.nvmlDeviceGetPowerUsage(h, ct.byref(pw)) == 0 and self.reasons_fn(h, ct.byref(rs)) == 0):
                self.rows.append((float(sm.value), pw.value / 1000.0, int(rs.value)))
            self.stop.wait(0.01)

    def __enter__(self):
        self.thread.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": self.smax, "reasons": ["no samples"]}
        sm = [r[0] for r in self.rows]
        hot = [x for x in sm if x > 0.3 * self.smax] or sm
        reasons = sorted({k for r in self.rows for k, b in self.BITS.items() if r[2] & b})
        return {"sm_mhz": statistics.median(hot), "sm_max_mhz": self.smax, "reasons": reasons,
                "samples": len(self.rows), "power_w_max": max(r[1] for r in self.rows), "sampler": "nvml, 10 ms"}


def clock_sampler(torch_device, index):
    """NVML sampler when pynvml works, else nvidia-smi."""
    try:
        return NvmlClockSampler(torch_device)
    except Exception:
        return ClockSampler(index)


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for r in csv.reader(f):
                r = [x.strip() for x in r]
                if len(r) >= 9 and r[0] == str(self.gpu):
                    rows.append(r)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        hot = [s for s in sm if s > 0.3 * smax] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(hot), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


# ------------------------------------------------------------------ CPU oracle leg

def cpu_oracle_eval(w, cands, target=None):
    """Oracle NCC loss and gradient for the given candidates; returns
    (grads, seconds, threads).  Target rendered by the oracle when absent."""
    import oracle
    g = w["geom"]
    iv = np.arange(g.n_views)
    ip = np.zeros(g.n_views, dtype=np.int32)
    mu = w["mu"].astype(np.float64)
    if target is None:
        target = oracle.forward(g, mu, w["pose_true"].astype(np.float64), iv, ip)
    grads = []
    t0 = time.perf_counter()
    for c in cands:
        pose = w["poses"][c].astype(np.float64)
        proj = oracle.forward(g, mu, pose, iv, ip)
        _, wts = oracle.pose_loss_weights("ncc", proj, target, iv, ip, 1)
        gth, _ = oracle.forward_grad(g, mu, pose, wts, iv, ip)
        grads.append(gth[0])
    dt = time.perf_counter() - t0
    return np.array(grads), dt, oracle.max_threads(), target


def reference_arm(args):
    """FP64 oracle on the host cores, each step a bounded sample (one
    candidate) of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.n_cand)
    _, _, threads, target = cpu_oracle_eval(w, [], None)
    times = []
    for s in range(args.warmup + args.steps):
        _, dt, _, _ = cpu_oracle_eval(w, [s % args.n_cand], target)
        if s >= args.warmup:
            times.append(dt)
    per = sum(times) / len(times)
    v = 1.0 / per
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "1 of %d candidates per step (2 views 384^2, 256^3)" % args.n_cand},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(args):
    return {"workload": "batched 2D/3D registration: 256^3 @0.8 mm, 2 views 384^2 @0.8 mm, %d candidate poses, "
                        "NCC loss + pose gradient fused" % args.n_cand,
            "volume": [256, 256, 256], "detector": [384, 384], "views": 2, "candidates": args.n_cand,
            "step_mm": 0.4, "loss": "ncc",
            "timing": "per-step CUDA events on the launching stream; L2 flushed (256 MiB write) between steps",
            "parallelism": "independent candidates per rank (no collective)" if args.gpus > 1 else "single GPU"}


# ------------------------------------------------------------------ other kernels

def _timed(fn, plan, pb, flush, reps=3):
    """Median main-kernel time (ms) of fn() over reps, L2 flushed before each."""
    fn()
    ks = []
    for _ in range(reps):
        flush.zero_()
        fn()
        ks.append(pb.proj_kernel_time_ms(plan))
    return float(np.median(ks))


def secondary(pb, torch, dev, w, mu_d, flush):
    """Main-kernel times of the other calls on full-size configurations."""
    out = {}
    g = w["geom"]
    # forward projection (DRR batch) and its exact transpose: the 128 registration instances
    nc = len(w["poses"])
    iv, ip = instance_maps(nc, g.n_views)
    P = pb.Projector(g, n_pose=nc, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_ADJOINT)
    pb.proj_enable_kernel_timing(P.plan)
    P.set_volume(mu_d)
    pose = torch.from_numpy(w["poses"]).to(dev)
    proj = torch.empty((P.n_inst, g.nv, g.nu), device=dev)
    samples = int(P.count_samples(pose).sum().item())
    ms = _timed(lambda: pb.proj_forward(P.plan, pose, proj, P.ws), P.plan, pb, flush)
    out["forward"] = {"kernel": "k_forward", "config": "256^3, %d view instances of 384^2" % P.n_inst, "kernel_ms": ms,
                      "rays_per_s": P.n_inst * g.nu * g.nv / (ms * 1e-3), "ray_samples_per_s": samples / (ms * 1e-3)}
    vol = torch.empty_like(mu_d)
    ms = _timed(lambda: pb.proj_forward_adjoint(P.plan, proj, pose, vol, P.ws), P.plan, pb, flush)
    out["forward_adjoint"] = {"kernel": "k_forward_adjoint", "config": "256^3, %d view instances of 384^2" % P.n_inst,
                              "kernel_ms": ms, "ray_samples_per_s": samples / (ms * 1e-3)}
    del P
    # FDK-weighted back-projection and its pose gradient: 360 views, 512^2, 256^3
    gm = synth.Geometry(256, 256, 256, 0.8, 0.8, 0.8, 512, 512,
                        synth.circular_views(360, synth.SAD, synth.SDD, 0.6, 0.6), 0.4)
    rng = np.random.default_rng(1003)
    motion = torch.from_numpy(synth.smooth_motion(rng, 360, 2.0, 3.0).astype(np.float32)).to(dev)
    Pb = pb.Projector(gm, n_pose=360, inst_view=np.arange(360), inst_pose=np.arange(360),
                      ops=pb.PROJ_OP_BACK | pb.PROJ_OP_BACK_GRAD)
    pb.proj_enable_kernel_timing(Pb.plan)
    img = torch.rand((360, 512, 512), device=dev)
    volb = torch.empty((256, 256, 256), device=dev)
    wvol = torch.randn((256, 256, 256), device=dev)
    gradb = torch.empty((360, 6), device=dev)
    vv = 360 * 256 ** 3
    ms = _timed(lambda: pb.proj_back(Pb.plan, img, motion, pb.PROJ_W_FDK, volb, Pb.ws), Pb.plan, pb, flush)
    out["back"] = {"kernel": "k_detector_records + k_back", "config": "256^3, 360 views of 512^2, FDK weight",
                   "kernel_ms": ms, "voxel_view_updates_per_s": vv / (ms * 1e-3)}
    imgb = torch.empty_like(img)
    ms = _timed(lambda: pb.proj_back_adjoint(Pb.plan, volb, motion, pb.PROJ_W_FDK, imgb, Pb.ws), Pb.plan, pb, flush)
    out["back_adjoint"] = {"kernel": "k_back_adjoint + k_detector_unrecord",
                           "config": "256^3, 360 views of 512^2, FDK weight", "kernel_ms": ms,
                           "voxel_view_updates_per_s": vv / (ms * 1e-3)}
    del imgb
    ms = _timed(lambda: pb.proj_back_pose_grad(Pb.plan, img, motion, pb.PROJ_W_FDK, wvol, gradb, Pb.ws), Pb.plan,
                pb, flush)
    out["back_pose_grad"] = {"kernel": "k_back_grad", "config": "256^3, 360 views of 512^2, FDK weight",
                             "kernel_ms": ms, "voxel_view_updates_per_s": vv / (ms * 1e-3),
                             "pose_gradient_evals_per_s": 360 / (ms * 1e-3)}
    shape, bt = pb.proj_autotune_back_grad(Pb.plan, img, motion, pb.PROJ_W_FDK, wvol, Pb.ws, reps=2)
    out["brick_shape_autotune"] = {"config": "256^3, 360 views of 512^2, FDK weight",
                                   "ms_per_launch": {"%dx%dx%d/%d views" % (32, 8, gz, nv): bt[k]
                                                     for k, (gz, nv) in enumerate(pb.BRICK_SHAPES)},
                                   "chosen": "%dx%dx%d/%d views" % ((32, 8) + pb.BRICK_SHAPES[shape])}
    # one motion-compensated FDK iteration at the same size (BP, sharpness, BP gradient, Adam step)
    from paper_2508_13304_b300.registration import Adam
    Pm = pb.Projector(gm, n_pose=360, inst_view=np.arange(360), inst_pose=np.arange(360),
                      ops=pb.PROJ_OP_BACK | pb.PROJ_OP_BACK_GRAD | pb.PROJ_OP_SHARPNESS)
    qf = Pm.fdk_filter(img, np.pi / 360)
    pose_m = motion.clone()
    opt = Adam(360, [0.1] * 3 + [1e-3] * 3, device=dev)
    act = torch.ones(360, dtype=torch.bool, device=dev)

    def moco_iter():
        v = Pm.back(qf, pose_m, pb.PROJ_W_FDK)
        _, dv = Pm.sharpness(v)
        gg = Pm.back_pose_grad(qf, pose_m, dv, pb.PROJ_W_FDK)
        opt.step(pose_m, gg, act)

    moco_iter()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        moco_iter()
    e1.record()
    e1.synchronize()
    out["moco_fdk_iteration"] = {"config": "256^3, 360 views of 512^2", "ms": e0.elapsed_time(e1) / 3,
                                 "what": "FDK back-projection + sharpness and its gradient + back-projection "
                                         "pose gradient (360 x 6) + Adam step"}
    del Pm, Pb
    # registration: time to the first candidate within 0.5 mm / 0.5 deg, 64 starts, batched vs plain multi-start
    from paper_2508_13304_b300 import registration as reg
    starts = w["poses"]
    true = w["pose_true"][0]
    tgt = None
    Pt = pb.Projector(g, n_pose=1, inst_view=np.arange(g.n_views), inst_pose=np.zeros(g.n_views, np.int32),
                      ops=pb.PROJ_OP_FORWARD)
    Pt.set_volume(mu_d)
    tgt = Pt.forward(torch.from_numpy(w["pose_true"]).to(dev)).cpu().numpy()
    mu_h = mu_d.cpu().numpy()
    # one untimed call first: the first registration in a process pays one-off set-up costs
    reg.register(g, mu_h, tgt, starts[:2], max_iter=3, batched=True, true_pose=true)
    reg.register(g, mu_h, tgt, starts[:4], max_iter=3, wave=2, true_pose=true)
    rb = reg.register(g, mu_h, tgt, starts, max_iter=150, batched=True, true_pose=true)
    t_plain, found, tried, plain_iters = 0.0, None, 0, []
    for c in range(len(starts)):
        rp = reg.register(g, mu_h, tgt, starts[c:c + 1], max_iter=150, batched=True, true_pose=true)
        plain_iters.append(int(rp["iters"][0]))
        if found is None:
            tried += 1
            if rp["first_hit_s"] is not None:
                found = t_plain + rp["first_hit_s"]
        t_plain += rp["seconds"]
    # the time to the first hit is a wall time with a host check per iteration: medians of 3 runs
    plain_reps = [found]
    for _ in range(2):
        t_rep, hit = 0.0, None
        for c in range(tried):
            rp = reg.register(g, mu_h, tgt, starts[c:c + 1], max_iter=150, batched=True, true_pose=true)
            if hit is None and rp["first_hit_s"] is not None:
                hit = t_rep + rp["first_hit_s"]
            t_rep += rp["seconds"]
        plain_reps.append(hit)
    if all(x is not None for x in plain_reps):
        found = float(np.median(plain_reps))
    waves = {}
    for B in (4, 8, 16):
        runs = [reg.register(g, mu_h, tgt, starts, max_iter=150, wave=B, true_pose=true, stop_at_hit=True)
                for _ in range(3)]
        hits = [rw["first_hit_s"] for rw in runs]
        waves[str(B)] = {"time_to_pose_s": float(np.median(hits)) if all(h is not None for h in hits) else None,
                         "runs_s": hits, "starts_begun": runs[0]["started"]}
    te, re = reg.pose_error(rb["poses"], true)
    out["registration"] = {
        "config": "256^3, 2 views of 384^2, %d starts (rot +-15 deg, trans +-20 mm), NCC, Adam 10 mm / 2 deg, "
                  "stop at dloss < 1e-5 or NCC > 0.999 or 150 iterations; time to the first pose within "
                  "0.5 mm / 0.5 deg of the truth" % len(starts),
        "batched_waves_time_to_pose_s": waves["8"]["time_to_pose_s"], "waves": waves,
        "batched_all_time_to_pose_s": rb["first_hit_s"], "batched_all_total_s": rb["seconds"],
        "batched_all_within_tol_at_end": int(np.sum((te <= 0.5) & (re <= 0.5))),
        "plain_time_to_pose_s": found, "plain_runs_s": plain_reps, "plain_starts_tried_to_first_hit": tried,
        "plain_iterations_per_start": plain_iters[:tried],
        "plain_total_s_all_starts": t_plain,
        "note": "plain = one start per launch, starts run one after another; batched waves = at most B starts "
                "in flight in one launch per iteration (proj_forward_pose_grad_list), a stopped start's slot "
                "taken by the next start on the device; batched all = every start in one launch"}
    # ray-tile shape autotuner on the benchmark's own launch (64 candidates x 2 views)
    Pa = pb.Projector(g, n_pose=nc, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD_GRAD)
    Pa.set_volume(mu_d)
    tg = torch.from_numpy(np.ascontiguousarray(tgt, dtype=np.float32)).to(dev)
    width, times = pb.proj_autotune_forward_grad(Pa.plan, pose, pb.PROJ_LOSS_NCC, tg, Pa.ws, reps=2)
    out["warp_shape_autotune"] = {"config": "256^3, 128 view instances of 384^2, NCC, default skipping",
                                  "ms_per_launch": {"%dx%d" % (k, 32 // k): v for k, v in times.items()},
                                  "chosen": "%dx%d" % (width, 32 // width)}
    # the same launch over (skip brick edge, cell test, warp shape)
    width, edge, cells, times = pb.proj_autotune_march(Pa.plan, pose, pb.PROJ_LOSS_NCC, tg, Pa.ws, reps=2)
    out["march_autotune"] = {"config": "256^3, 128 view instances of 384^2, NCC",
                             "ms_per_launch": {"edge %d, cells %d, %dx%d" % (e, c, k, 32 // k): v
                                               for (e, c, k), v in times.items()},
                             "chosen": "edge %d, cells %d, %dx%d" % (edge, cells, width, 32 // width)}
    del Pa
    # volume layouts of the fused march on the same launch: rows along x and along y (default), rows along
    # x only (PROJ_FLAG_ONE_COPY), bricks of 4^3 cells (PROJ_FLAG_BRICKS); march and gathers alone (probe),
    # with the default skipping and without
    layouts = {}
    gl = torch.empty((nc, 6), device=dev)
    ll = torch.empty((nc,), device=dev)
    for name, flag in (("rows_x_and_y", 0), ("rows_x", pb.PROJ_FLAG_ONE_COPY), ("bricks_4", pb.PROJ_FLAG_BRICKS)):
        Pl = pb.Projector(g, n_pose=nc, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD_GRAD | flag)
        pb.proj_enable_kernel_timing(Pl.plan)
        Pl.set_volume(mu_d)
        row = {"workspace_gb": pb.proj_workspace_size(Pl.plan) / 1e9}
        for tag in ("", "_without_skipping"):
            if tag:
                pb.proj_set_skip_brick(Pl.plan, 0)
                pb.proj_set_skip_cells(Pl.plan, pb.SKIP_CELLS_OFF)
            row["kernel_ms" + tag] = _timed(
                lambda: pb.proj_forward_pose_grad(Pl.plan, pose, pb.PROJ_LOSS_NCC, tg, gl, ll, None, Pl.ws),
                Pl.plan, pb, flush)
            row["probe_ms" + tag] = _timed(lambda: pb.proj_gather_probe(Pl.plan, pose, Pl.ws), Pl.plan, pb, flush)
        layouts[name] = row
        del Pl
    out["march_layouts"] = {"config": "256^3, 128 view instances of 384^2, NCC, 4x8 warps", **layouts}
    out["c1_small"] = c1_small(pb, torch, dev, flush)
    out["moco_quality"] = moco_quality(pb, torch, dev)
    out["gradient_accuracy"] = gradient_accuracy(pb, torch, dev, mu_d)
    out["paper_tables"] = paper_tables(pb, torch, dev, flush)
    out["registration_cuda_graph"] = graph_timing(pb, torch, g, mu_h, tgt, starts)
    out["posenet"] = posenet_measure(pb, torch, dev, flush, g, mu_d, load_peaks())
    out["uneven_batch_small"] = uneven_batch(pb, torch, dev, flush, with_large=False)
    out["uneven_batch_c4"] = uneven_batch(pb, torch, dev, flush, with_large=True)
    out["cpu_baseline_subsets"] = oracle_subset_rates(out)   # CPU-baseline leg: the oracle beside the GPU
    return out


def oracle_subset_rates(sec):
    """The FP64 oracle (all host cores) on seeded subsets of the
    motion-compensated and calibration workloads, its rate per voxel-view or
    ray sample extrapolated to the full call, beside the GPU's rate on the
    full call: FDK back-projection on 32 of the 360 views, its pose gradient
    on 8, and the fused L2 pose gradient of the 512^3 / 768^2 problem on the
    64 central detector rows of 4 of its 720 views."""
    import oracle
    out = {"threads": oracle.max_threads(), "kind": "oracle"}
    rng = np.random.default_rng(1003)
    gm = synth.Geometry(256, 256, 256, 0.8, 0.8, 0.8, 512, 512,
                        synth.circular_views(360, synth.SAD, synth.SDD, 0.6, 0.6), 0.4)
    motion = synth.smooth_motion(rng, 360, 2.0, 3.0)
    views = np.arange(0, 360, 360 // 32)[:32]
    img = rng.random((32, 512, 512))
    t0 = time.perf_counter()
    oracle.back(gm, img, motion[views], inst_view=views, inst_pose=np.arange(32), weight=oracle.W_FDK)
    r = 32 * 256 ** 3 / (time.perf_counter() - t0)
    gpu = sec["back"]["voxel_view_updates_per_s"]
    out["fdk_back_projection"] = {"sample": "32 of 360 views", "oracle_voxel_view_updates_per_s": r,
                                  "gpu_voxel_view_updates_per_s": gpu, "speedup": gpu / r}
    wvol = rng.standard_normal((256, 256, 256))
    t0 = time.perf_counter()
    oracle.back_grad(gm, img[:8], motion[views[:8]], wvol, inst_view=views[:8], inst_pose=np.arange(8),
                     weight=oracle.W_FDK)
    r = 8 * 256 ** 3 / (time.perf_counter() - t0)
    gpu = sec["back_pose_grad"]["voxel_view_updates_per_s"]
    out["fdk_back_projection_pose_grad"] = {"sample": "8 of 360 views", "oracle_voxel_view_updates_per_s": r,
                                            "gpu_voxel_view_updates_per_s": gpu, "speedup": gpu / r}
    q = synth.workload_uneven(with_large=True, n_extra=0)[0]
    g4 = q["geom"]
    vsel = np.array([0, 180, 360, 540])
    band = synth.Geometry(g4.nx, g4.ny, g4.nz, g4.vx, g4.vy, g4.vz, g4.nu, 64, g4.views[vsel], g4.step)
    mu4 = rng.random((g4.nz, g4.ny, g4.nx))
    pose = q["poses"][vsel]
    iv = np.arange(4)
    _, ns = oracle.forward(band, mu4, pose, iv, iv, return_samples=True)
    resid = rng.standard_normal((4, 64, g4.nu))
    t0 = time.perf_counter()
    oracle.forward_grad(band, mu4, pose, resid, iv, iv)
    r = float(np.sum(ns)) / (time.perf_counter() - t0)
    gpu = sec["uneven_batch_c4"]["batched_ray_samples_per_s"]
    out["calibration_pose_grad"] = {"sample": "64 central rows of 4 of the 720 views of 768^2 (512^3)",
                                    "oracle_ray_samples_per_s": r, "gpu_ray_samples_per_s": gpu, "speedup": gpu / r,
                                    "oracle_s_per_full_eval_extrapolated": sec["uneven_batch_c4"]["ray_samples"] / r}
    return out


def _event_ms(torch, fn, flush, reps=2):
    """Median CUDA-event time (ms) of fn() on the current stream, L2 flushed
    before each repetition, after one warm-up call."""
    fn()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def uneven_batch(pb, torch, dev, flush, with_large, n_extra=24):
    """Independent L2 pose-gradient problems of uneven size: one persistent
    batched launch (proj_batch_run) against one proj_forward_pose_grad call
    per problem on the same stream.  Both include the pose set-ups and the
    reductions.  n_extra: how many of the single-view problems (the first
    ones of the same seeded sequence)."""
    probs = synth.workload_uneven(with_large=with_large, n_extra=n_extra)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1004)
    items, keep, samples = [], [], 0
    for q in probs:
        g = q["geom"]
        nvw, npose = g.n_views, len(q["poses"])
        P = pb.Projector(g, n_pose=npose, inst_view=np.arange(nvw),
                         inst_pose=np.arange(nvw) if npose == nvw else np.zeros(nvw, np.int32),
                         ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_FORWARD_GRAD)
        P.set_volume(torch.rand((g.nz, g.ny, g.nx), device=dev, generator=gen))
        pose = torch.from_numpy(q["poses"].astype(np.float32)).to(dev)
        samples += int(P.count_samples(pose).sum().item())
        keep.append(P)
        items.append(dict(plan=P.plan, loss=pb.PROJ_LOSS_L2, pose=pose,
                          ref=torch.rand((nvw, g.nv, g.nu), device=dev, generator=gen),
                          grad=torch.zeros((npose, 6), device=dev), loss_out=torch.zeros(npose, device=dev),
                          ws=P.ws))
    b = pb.proj_batch_create(items)

    def separate():
        for it in items:
            pb.proj_forward_pose_grad(it["plan"], it["pose"], it["loss"], it["ref"], it["grad"], it["loss_out"],
                                      None, it["ws"])

    ms_sep = _event_ms(torch, separate, flush)
    g_sep = torch.cat([it["grad"].reshape(-1) for it in items]).clone()
    ms_bat = _event_ms(torch, lambda: pb.proj_batch_run(b), flush)
    g_bat = torch.cat([it["grad"].reshape(-1) for it in items])
    diff = float(((g_bat - g_sep).norm() / g_sep.norm()).item())
    sizes = [(q["geom"].nx, q["geom"].nu, q["geom"].n_views) for q in probs]
    del b, items, keep
    torch.cuda.empty_cache()
    return {"config": ("512^3 / 720 views of 768^2 (per-view poses) + " if with_large else "")
            + "%d single-view problems, volumes %d..%d^3, detectors %d..%d^2, L2 loss"
            % (len(probs) - int(with_large), min(s_[0] for s_ in sizes[int(with_large):]),
               max(s_[0] for s_ in sizes[int(with_large):]), min(s_[1] for s_ in sizes[int(with_large):]),
               max(s_[1] for s_ in sizes[int(with_large):])),
            "problems": len(probs), "ray_samples": samples,
            "batched_ms": ms_bat, "separate_ms": ms_sep, "speedup": ms_sep / ms_bat,
            "batched_ray_samples_per_s": samples / (ms_bat * 1e-3),
            "grad_rel_diff_batched_vs_separate": diff,
            "what": "batched = set-ups, one persistent work-queue launch over all problems' ray tiles, "
                    "reductions; separate = proj_forward_pose_grad per problem, back to back"}


def gradient_accuracy(pb, torch, dev, mu_d, n_motion=128, n_views=8):
    """The paper's accuracy protocol (Sec. II-D.1 / III-A) on the GPU: 8 views
    over 0-90 deg, 128 random motions per view (translations N(0, 20 mm),
    rotations N(0, 10 deg)), L2 loss against the projection at zero motion;
    cosine similarity per motion between the fused analytic pose gradient and
    a central finite difference of the same loss (projections by the forward
    projector, loss summed in FP64)."""
    import math
    g0 = workload(1)["geom"]
    views = synth.circular_views(n_views, synth.SAD, synth.SDD, 0.8, 0.8,
                                 angles=np.linspace(0.0, math.pi / 2, n_views))
    g = synth.Geometry(g0.nx, g0.ny, g0.nz, g0.vx, g0.vy, g0.vz, g0.nu, g0.nv, views, g0.step)
    rng = np.random.default_rng(1009)
    n = n_motion * n_views
    pose = np.zeros((n, 6), np.float32)
    pose[:, :3] = rng.normal(0.0, 20.0, (n, 3))
    pose[:, 3:] = np.deg2rad(rng.normal(0.0, 10.0, (n, 3)))
    iv = np.repeat(np.arange(n_views), n_motion).astype(np.int32)
    ip = np.arange(n, dtype=np.int32)
    P = pb.Projector(g, n_pose=n, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_FORWARD_GRAD)
    P.set_volume(mu_d)
    P0 = pb.Projector(g, n_pose=1, inst_view=np.arange(n_views), inst_pose=np.zeros(n_views, np.int32),
                      ops=pb.PROJ_OP_FORWARD)
    P0.set_volume(mu_d)
    target = P0.forward(torch.zeros((1, 6), device=dev)).contiguous()          # [views][nv][nu]
    tgt_inst = target[torch.from_numpy(iv).long().to(dev)]
    pose_d = torch.from_numpy(pose).to(dev)
    grad, _ = P.forward_pose_grad(pose_d, pb.PROJ_LOSS_L2, target)

    def losses(pz):
        d = (P.forward(pz) - tgt_inst).double()
        return (d * d).sum(dim=(1, 2))

    steps = [0.05] * 3 + [5e-4] * 3
    fd = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    for j in range(6):
        e = torch.zeros((1, 6), device=dev)
        e[0, j] = steps[j]
        fd[:, j] = (losses((pose_d + e).contiguous()) - losses((pose_d - e).contiguous())) / (2 * steps[j])
    ga = grad.double()
    cos = (ga * fd).sum(1) / (ga.norm(dim=1) * fd.norm(dim=1)).clamp_min(1e-300)
    valid = fd.norm(dim=1) > 0
    c = cos[valid].cpu().numpy()
    return {"config": "256^3 registration phantom, %d views over 0-90 deg of 384^2, %d motions (t N(0, 20 mm), "
                      "rot N(0, 10 deg)), L2 loss vs zero motion; FD steps 0.05 mm / 5e-4 rad" % (n_views, n),
            "motions": int(valid.sum().item()), "mean_cosine": float(c.mean()), "p5_cosine": float(np.percentile(c, 5)),
            "min_cosine": float(c.min()), "paper_rd_mean": 0.9952,
            "back": back_gradient_accuracy(pb, torch, dev, mu_d, g, target, n_motion=n_motion // 4)}


def back_gradient_accuracy(pb, torch, dev, mu_d, g, target, n_motion=32):
    """The back-projection half of the accuracy protocol: per (view, motion)
    the L2 loss between the voxel-driven back-projection of that view's
    zero-motion projection at the moved pose and the volume, its analytic pose
    gradient (back-projection pose gradient with dL/dmu = 2 (b - mu)) and a
    central finite difference (losses summed in FP64)."""
    n_views = g.n_views
    rng = np.random.default_rng(1010)
    mu64 = mu_d.double()
    steps = [0.05] * 3 + [5e-4] * 3
    cos = []
    for v in range(n_views):
        P = pb.Projector(g, n_pose=1, inst_view=np.array([v], np.int32), inst_pose=np.zeros(1, np.int32),
                         ops=pb.PROJ_OP_BACK | pb.PROJ_OP_BACK_GRAD)
        img = target[v:v + 1].contiguous()
        for _ in range(n_motion):
            th = np.zeros((1, 6), np.float32)
            th[0, :3] = rng.normal(0.0, 20.0, 3)
            th[0, 3:] = np.deg2rad(rng.normal(0.0, 10.0, 3))
            pose = torch.from_numpy(th).to(dev)
            b = P.back(img, pose)
            ga = P.back_pose_grad(img, pose, (2.0 * (b.double() - mu64)).float())[0].double()
            fd = torch.zeros(6, dtype=torch.float64, device=dev)
            for j in range(6):
                e = torch.zeros((1, 6), device=dev)
                e[0, j] = steps[j]
                lp = ((P.back(img, (pose + e).contiguous()).double() - mu64) ** 2).sum()
                lm = ((P.back(img, (pose - e).contiguous()).double() - mu64) ** 2).sum()
                fd[j] = (lp - lm) / (2 * steps[j])
            cos.append(float((ga @ fd) / (ga.norm() * fd.norm())))
    c = np.array(cos)
    return {"config": "%d views over 0-90 deg, %d motions, plain back-projection, L2 loss vs the volume" %
                      (n_views, len(c)),
            "mean_cosine": float(c.mean()), "p5_cosine": float(np.percentile(c, 5)), "min_cosine": float(c.min()),
            "paper_vd_mean": 0.9984, "paper_vd_p95": 0.9938}


PAPER_TABLES = (  # volume, detector, paper Table III (RD, 100 iterations) s, Table IV (VD, 256 views, 1 iteration) s
    (128, 192, 1.25, 0.17), (256, 384, 2.44, 1.21), (384, 576, 6.24, 3.99), (512, 768, 12.70, 9.50))


def paper_tables(pb, torch, dev, flush):
    """The paper's timing tables at their sizes, each time covering the whole
    step as the paper's do (loss, pose gradient, one gradient-descent update):
    Table III = 100 iterations of the L2 pose gradient of one view's
    projection; Table IV = one iteration of the L2 image loss of the
    back-projection of 256 views and its per-view pose gradient.  Volumes
    span 204.8 mm, the detector covers them (SAD 800 / SDD 1200 mm); the
    volume values are uniform noise (they do not change the work)."""
    gen = torch.Generator(device=dev)
    gen.manual_seed(1011)
    rows = []
    for n, d, t3_paper, t4_paper in PAPER_TABLES:
        vox = 204.8 / n
        pix = 1.1 * 204.8 * math.sqrt(2.0) * (synth.SDD / synth.SAD) / d
        mu = torch.rand((n, n, n), device=dev, generator=gen)
        # Table III: one view, 100 iterations of loss + pose gradient + update
        g1 = synth.Geometry(n, n, n, vox, vox, vox, d, d, synth.circular_views(1, synth.SAD, synth.SDD, pix, pix),
                            0.5 * vox)
        # the target is rendered by a plan of its own, so the measured workspace is the gradient path's
        Pt = pb.Projector(g1, n_pose=1, inst_view=np.zeros(1, np.int32), inst_pose=np.zeros(1, np.int32),
                          ops=pb.PROJ_OP_FORWARD)
        Pt.set_volume(mu)
        target = Pt.forward(torch.zeros((1, 6), device=dev)).contiguous()
        del Pt
        P1 = pb.Projector(g1, n_pose=1, inst_view=np.zeros(1, np.int32), inst_pose=np.zeros(1, np.int32),
                          ops=pb.PROJ_OP_FORWARD_GRAD)
        P1.set_volume(mu)
        pose = torch.tensor([[2.0, -1.0, 1.5, 0.02, -0.03, 0.01]], device=dev)
        gbuf = torch.empty((1, 6), device=dev)
        lbuf = torch.empty(1, device=dev)
        lr = torch.tensor([[0.1, 0.1, 0.1, 1e-3, 1e-3, 1e-3]], device=dev)

        def t3():
            for _ in range(100):
                pb.proj_forward_pose_grad(P1.plan, pose, pb.PROJ_LOSS_L2, target, gbuf, lbuf, None, P1.ws)
                pose.sub_(lr * gbuf.sign())

        ms3 = _event_ms(torch, t3, flush, reps=2)
        ws3 = pb.proj_workspace_size(P1.plan)
        del P1
        # the same with one copy of the prepared volume (PROJ_FLAG_ONE_COPY): the memory-lean plan
        pose.copy_(torch.tensor([[2.0, -1.0, 1.5, 0.02, -0.03, 0.01]], device=dev))
        P1 = pb.Projector(g1, n_pose=1, inst_view=np.zeros(1, np.int32), inst_pose=np.zeros(1, np.int32),
                          ops=pb.PROJ_OP_FORWARD_GRAD | pb.PROJ_FLAG_ONE_COPY)
        P1.set_volume(mu)
        ms3c = _event_ms(torch, t3, flush, reps=2)
        ws3c = pb.proj_workspace_size(P1.plan)
        del P1
        # Table IV: 256 views, one iteration of back-projection, image loss, pose gradient, update
        g4 = synth.Geometry(n, n, n, vox, vox, vox, d, d, synth.circular_views(256, synth.SAD, synth.SDD, pix, pix),
                            0.5 * vox)
        P4 = pb.Projector(g4, n_pose=256, inst_view=np.arange(256), inst_pose=np.arange(256),
                          ops=pb.PROJ_OP_BACK | pb.PROJ_OP_BACK_GRAD)
        img = torch.rand((256, d, d), device=dev, generator=gen)
        pose4 = torch.zeros((256, 6), device=dev)
        vol = torch.empty((n, n, n), device=dev)
        g4buf = torch.empty((256, 6), device=dev)

        def t4():
            pb.proj_back(P4.plan, img, pose4, pb.PROJ_W_NONE, vol, P4.ws)
            resid = 2.0 * (vol - mu)                 # d/dvol of the L2 image loss
            pb.proj_back_pose_grad(P4.plan, img, pose4, pb.PROJ_W_NONE, resid, g4buf, P4.ws)
            pose4.sub_(1e-6 * g4buf)

        ms4 = _event_ms(torch, t4, flush, reps=2)
        ws4 = pb.proj_workspace_size(P4.plan)
        del P4, img, vol, mu
        torch.cuda.empty_cache()
        rows.append({"volume": n, "detector": d,
                     "table3_100_iter_s": ms3 * 1e-3, "table3_paper_s": t3_paper, "table3_ratio": t3_paper / (ms3 * 1e-3),
                     "table3_workspace_gb": ws3 / 1e9,
                     "table3_one_copy_100_iter_s": ms3c * 1e-3, "table3_one_copy_workspace_gb": ws3c / 1e9,
                     "table4_iter_s": ms4 * 1e-3, "table4_paper_s": t4_paper, "table4_ratio": t4_paper / (ms4 * 1e-3),
                     "table4_workspace_gb": ws4 / 1e9})
    return {"rows": rows, "note": "paper: RTX 4090, whole autograd steps in PyTorch with the authors' kernels and "
                                  "the exact path-length projector; ratios are context, not a like-for-like "
                                  "comparison"}


def registration_500(pb, torch, dev, n_prob=500, max_iter=200):
    """The shape of the paper's end-to-end registration experiment (Table V,
    Sec. II-D.3) on the synthetic registration phantom: n_prob independent
    single-view 2D/3D registrations (views spread over 360 deg, 384^2), each
    target rendered at the true pose with Poisson noise of 1e5 photons per
    pixel, starts perturbed by N(0, 20 mm) / N(0, 20 deg), NCC loss, Adam with
    the paper's 10 mm / 2 deg steps, stop at loss change < 1e-5 or NCC >
    0.999, failure if the final NCC < 0.99.  All problems advance together in
    one fused launch per iteration."""
    from paper_2508_13304_b300 import registration as reg
    w = workload(1)
    g0 = w["geom"]
    views = synth.circular_views(n_prob, synth.SAD, synth.SDD, 0.8, 0.8)
    g = synth.Geometry(g0.nx, g0.ny, g0.nz, g0.vx, g0.vy, g0.vz, g0.nu, g0.nv, views, g0.step)
    mu_d = torch.from_numpy(w["mu"].astype(np.float32)).to(dev)
    P0 = pb.Projector(g, n_pose=1, inst_view=np.arange(n_prob), inst_pose=np.zeros(n_prob, np.int32),
                      ops=pb.PROJ_OP_FORWARD)
    P0.set_volume(mu_d)
    clean = P0.forward(torch.zeros((1, 6), device=dev))
    gen = torch.Generator(device=dev)
    gen.manual_seed(1012)
    counts = torch.poisson(1e5 * torch.exp(-clean), generator=gen)
    target = (-torch.log(counts.clamp_min(1.0) / 1e5)).cpu().numpy()
    del P0, clean, counts
    rng = np.random.default_rng(1012)
    init = np.zeros((n_prob, 6), np.float32)
    init[:, :3] = rng.normal(0.0, 20.0, (n_prob, 3))
    init[:, 3:] = np.deg2rad(rng.normal(0.0, 20.0, (n_prob, 3)))
    truth = np.zeros((n_prob, 6), np.float32)
    mu_h = w["mu"].astype(np.float32)
    iv = np.arange(n_prob)
    reg.register(g, mu_h, target, init[:8], max_iter=3, inst_view=iv[:8])      # untimed warm-up
    r = reg.register(g, mu_h, target, init, max_iter=max_iter, inst_view=iv)
    te, re = reg.pose_error(r["poses"], truth)
    ok = r["ncc"] >= 0.99
    return {"config": "%d single-view registrations, 256^3 / 384^2, Poisson 1e5 photons, starts N(0, 20 mm) / "
                      "N(0, 20 deg), NCC, Adam 10 mm / 2 deg, stop at dloss < 1e-5 or NCC > 0.999" % n_prob,
            "total_s": r["seconds"], "per_problem_s": r["seconds"] / n_prob,
            "successes_ncc_ge_0.99": int(ok.sum()), "problems": n_prob,
            "median_error_of_successes_mm_deg": [float(np.median(te[ok])) if ok.any() else None,
                                                 float(np.median(re[ok])) if ok.any() else None],
            "iterations_max": int(r["iters"].max()),
            "paper": "RTX 4090, CQ500 head: 18.45 min for 500 views (2.21 s each), 343 successes"}


def moco_quality(pb, torch, dev):
    """Motion-compensated FDK on the 360-view workload (256^3 at 0.8 mm,
    512^2 at 0.6 mm, smooth per-view motion rot <= 2 deg, trans <= 3 mm):
    projections rendered at the moving poses, then 240 iterations of the
    sharpness loss with a centred 24-node spline motion model (translations
    and rotations).  Errors are relative L2 distances to the FDK of
    motion-free projections."""
    from paper_2508_13304_b300 import moco
    w = synth.workload_moco()
    g = w["geom"]
    n = g.n_views
    motion = w["poses"].astype(np.float32)
    motion -= motion.mean(axis=0)
    F = pb.Projector(g, n_pose=n, inst_view=np.arange(n), inst_pose=np.arange(n),
                     ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_BACK)
    F.set_volume(torch.from_numpy(w["mu"].astype(np.float32)).to(dev))
    proj = F.forward(motion)
    zero = np.zeros((n, 6), np.float32)
    ref = F.back(F.fdk_filter(F.forward(zero), math.pi / n), zero, pb.PROJ_W_FDK)
    best = F.back(F.fdk_filter(proj, math.pi / n), motion, pb.PROJ_W_FDK)

    def rel(a):
        return float((a - ref).norm() / ref.norm())

    out = moco.moco_fdk(g, proj.cpu().numpy(), n_iter=240, lr=[0.05] * 3 + [math.radians(0.02)] * 3,
                        spline_nodes=24, device=dev)
    d = out["poses"] - motion
    return {"config": "256^3, 360 views of 512^2, 24-node spline (translations and rotations), 240 iterations",
            "recon_err_uncompensated": rel(torch.from_numpy(out["fdk0"]).to(dev)),
            "recon_err_compensated": rel(torch.from_numpy(out["fdk"]).to(dev)),
            "recon_err_true_motion": rel(best),
            "trans_rms_mm_before_after": [float(np.sqrt((motion[:, :3] ** 2).mean())),
                                          float(np.sqrt((d[:, :3] ** 2).mean()))],
            "rot_rms_deg_before_after": [float(np.degrees(np.sqrt((motion[:, 3:] ** 2).mean()))),
                                         float(np.degrees(np.sqrt((d[:, 3:] ** 2).mean())))],
            "sharpness_before_after": [float(out["sharpness"][0]), float(out["sharpness"][-1])],
            "seconds": out["seconds"]}


def c1_small(pb, torch, dev, flush):
    """The small configuration (64^3 at 1 mm, 8 views of 128^2 at 1.5 mm, one
    pose, L2 target at a second pose): the four hot-path calls on the GPU, and
    the FP64 oracle's forward pose gradient on the same work with one thread
    and with all host threads (ray-samples/s)."""
    import oracle
    w = synth.workload_tiny()
    g = w["geom"]
    P = pb.Projector(g, n_pose=1, inst_view=np.arange(g.n_views), inst_pose=np.zeros(g.n_views, np.int32))
    pb.proj_enable_kernel_timing(P.plan)
    mu = torch.from_numpy(w["mu"].astype(np.float32)).to(dev)
    P.set_volume(mu)
    pose = torch.from_numpy(w["pose"].astype(np.float32)).to(dev)
    target = P.forward(torch.from_numpy(w["pose_true"].astype(np.float32)).to(dev)).contiguous()
    det = torch.from_numpy(w["det_image"].astype(np.float32)).to(dev)
    samples = int(P.count_samples(pose).sum().item())
    proj = torch.empty_like(target)
    vol = torch.empty_like(mu)
    grad = torch.empty((1, 6), device=dev)
    loss = torch.empty(1, device=dev)
    wv = torch.randn(mu.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(1001))
    out = {"config": "64^3 at 1 mm, 8 views of 128^2 at 1.5 mm, one pose", "ray_samples": samples}
    out["forward_ms"] = _timed(lambda: pb.proj_forward(P.plan, pose, proj, P.ws), P.plan, pb, flush)
    out["forward_pose_grad_ms"] = _timed(
        lambda: pb.proj_forward_pose_grad(P.plan, pose, pb.PROJ_LOSS_L2, target, grad, loss, None, P.ws), P.plan, pb,
        flush)
    out["back_ms"] = _timed(lambda: pb.proj_back(P.plan, det, pose, pb.PROJ_W_NONE, vol, P.ws), P.plan, pb, flush)
    out["back_pose_grad_ms"] = _timed(
        lambda: pb.proj_back_pose_grad(P.plan, det, pose, pb.PROJ_W_NONE, wv, grad, P.ws), P.plan, pb, flush)
    # oracle: forward pose gradient of the same L2 loss, 1 thread and all threads
    mu64 = w["mu"].astype(np.float64)
    pose64 = w["pose"].astype(np.float64)
    tgt64 = target.double().cpu().numpy()
    iv = np.arange(g.n_views)
    ip = np.zeros(g.n_views, dtype=np.int32)
    rates = {}
    n_all = oracle.max_threads()
    for n_thr in (1, n_all):
        oracle.set_threads(n_thr)
        t0 = time.perf_counter()
        p64 = oracle.forward(g, mu64, pose64, iv, ip)
        _, wts = oracle.pose_loss_weights("l2", p64, tgt64, iv, ip, 1)
        oracle.forward_grad(g, mu64, pose64, wts, iv, ip)
        rates[n_thr] = samples / (time.perf_counter() - t0)
    oracle.set_threads(n_all)
    out["oracle_forward_pose_grad_samples_per_s"] = {"1_thread": rates[1], "%d_threads" % n_all: rates[n_all]}
    out["gpu_forward_pose_grad_samples_per_s"] = samples / (out["forward_pose_grad_ms"] * 1e-3)
    return out


def graph_timing(pb, torch, g, mu_h, tgt, starts):
    """Registration iterations eager (one host check per iteration) vs
    replayed CUDA graphs of 10 iterations; every candidate kept running."""
    from paper_2508_13304_b300 import registration as reg
    out = {}
    for label, st, n_it in (("1_start", starts[:1], 101), ("%d_starts" % len(starts), starts, 31)):
        res = {}
        for mode, k in (("eager", 0), ("graph", 10)):
            reg.register(g, mu_h, tgt, st, max_iter=11, ncc_stop=2.0, dloss_stop=-1.0, graph_steps=k)
            r = reg.register(g, mu_h, tgt, st, max_iter=n_it, ncc_stop=2.0, dloss_stop=-1.0, graph_steps=k)
            res[mode + "_ms_per_iteration"] = r["seconds"] * 1e3 / n_it
        res["speedup"] = res["eager_ms_per_iteration"] / res["graph_ms_per_iteration"]
        out[label] = res
    out["what"] = ("wall time per registration iteration (pose-gradient launch, stopping test, Adam step): eager "
                   "with a host check each iteration vs CUDA graphs of 10 captured iterations")
    return out


GEMM_SHAPES = ((8192, 8192, 8192), (262144, 64, 288), (65536, 128, 576), (16384, 128, 1152), (16384, 1152, 128))


def gemm_throughput(pb, torch, dev, flush, bf16_peak, shapes=GEMM_SHAPES):
    """Tensor-core GEMM (pn_gemm_bf16, BF16 in, FP32 accumulate, BF16 out)
    on a square shape and on the convolution shapes of the pose network."""
    out = []
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    for i, (M, N, K) in enumerate(shapes):
        A = torch.randn((M, K), device=dev, generator=gen).bfloat16()
        B = torch.randn((N, K), device=dev, generator=gen).bfloat16()
        D = torch.empty((M, N), device=dev, dtype=torch.bfloat16)
        names = {2: "2-SM 256x256 persistent", 1: "2-SM 256x256 per tile", 0: "1-SM 128x256"}
        for mode in ((2, 1, 0) if i == 0 else (2,)):
            pb.pn_gemm_use_pair_tiles(mode)
            ms = _event_ms(torch, lambda: pb.pn_gemm_bf16(M, N, K, A, K, B, K, D16=D), flush, reps=5)
            tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
            byts = 2.0 * (M * K + N * K + M * N)
            wide = N > 128 and M > 128
            out.append({"M": M, "N": N, "K": K, "tiles": names[mode] if wide else "1-SM",
                        "ms": ms, "tflops": tf, "frac_of_bf16_peak": tf / bf16_peak,
                        "hbm_gbs_min_traffic": byts / (ms * 1e-3) / 1e9})
        pb.pn_gemm_use_pair_tiles(2)
        del A, B, D
    return out


# convolution layers 2..6 of the pose network at batch 256: (input side, input channels, output channels)
CONV_LAYERS = ((64, 32, 64), (32, 64, 128), (16, 128, 128), (8, 128, 128), (4, 128, 128))


def conv_layers(pb, torch, dev, flush, bf16_peak, B=256):
    """The network's 3x3 stride-2 convolutions (bias + ReLU, BF16 out): im2col
    + GEMM against the implicit-GEMM kernel that gathers the patches itself,
    and their input gradients: GEMM + col2im against the implicit GEMM (which
    multiplies 9 taps per input pixel, about 2.25 of them non-zero, so its
    useful rate is quoted)."""
    out = []
    gen = torch.Generator(device=dev)
    gen.manual_seed(8)
    for H, C, Co in CONV_LAYERS:
        Ho = (H + 1) // 2
        M, K = B * Ho * Ho, 9 * C
        x = torch.randn((B, H, H, C), device=dev, generator=gen).bfloat16()
        w = torch.randn((Co, K), device=dev, generator=gen).bfloat16()
        bias = torch.zeros(Co, device=dev)
        col = torch.empty((M, K), device=dev, dtype=torch.bfloat16)
        y = torch.empty((M, Co), device=dev, dtype=torch.bfloat16)

        def explicit():
            pb.pn_im2col_3x3s2(x, B, H, H, C, K, col)
            pb.pn_gemm_bf16(M, Co, K, col, K, w, K, bias=bias, relu=True, D16=y)

        ms_e = _event_ms(torch, explicit, flush, reps=5)
        ms_i = _event_ms(torch, lambda: pb.pn_conv3x3s2_bf16(x, B, H, H, C, w, Co, bias=bias, relu=True, y16=y),
                         flush, reps=5)
        # input gradient (ReLU mask of x): GEMM into the FP32 column matrix + col2im, against the implicit GEMM
        wT = torch.empty((K, Co), device=dev, dtype=torch.bfloat16)
        pb.pn_transpose_bf16(w, Co, K, wT, Co)
        wt = torch.empty((C, 9 * Co), device=dev, dtype=torch.bfloat16)
        pb.pn_conv_dgrad_weights(w, Co, C, wt)
        dcol = torch.empty((M, K), device=dev)
        dx = torch.empty((B, H, H, C), device=dev, dtype=torch.bfloat16)

        def dgrad_explicit():
            pb.pn_gemm_bf16(M, K, Co, y, Co, wT, Co, D32=dcol)
            pb.pn_col2im_3x3s2(dcol, B, H, H, C, K, mask=x, dx16=dx)

        ms_de = _event_ms(torch, dgrad_explicit, flush, reps=5)
        ms_di = _event_ms(torch, lambda: pb.pn_conv3x3s2_dgrad_bf16(y, B, H, H, C, wt, Co, mask=x, dx16=dx),
                          flush, reps=5)
        fl = 2.0 * M * Co * K
        out.append({"input": "%dx%dx%dx%d" % (B, H, H, C), "cout": Co, "gemm_MNK": [M, Co, K],
                    "im2col_gemm_ms": ms_e, "implicit_ms": ms_i, "implicit_tflops": fl / (ms_i * 1e-3) / 1e12,
                    "implicit_frac_of_bf16_peak": fl / (ms_i * 1e-3) / 1e12 / bf16_peak,
                    "col_matrix_bytes_avoided": M * K * 2,
                    "dgrad_gemm_col2im_ms": ms_de, "dgrad_implicit_ms": ms_di,
                    "dgrad_implicit_tflops_useful": fl / (ms_di * 1e-3) / 1e12,
                    "dgrad_fp32_col_matrix_bytes_avoided": M * K * 4})
        del x, w, col, y, wT, wt, dcol, dx
    return out


def posenet_measure(pb, torch, dev, flush, g, mu_d, peaks):
    """Pose-proposal network: GEMM roofline, DRR batch generation, network
    training step (batch 256, 2 views of 128^2 from 384^2 DRRs)."""
    from paper_2508_13304_b300 import posenet as pn
    bf16_peak = float(peaks.get("bf16_tflops", 1800.0))
    gem = gemm_throughput(pb, torch, dev, flush, bf16_peak)
    top = gem[0]
    B = 256
    net = pn.PoseNet(B, in_hw=128, n_views=2)
    src = pn.DrrSource(g, mu_d, B, factor=3, seed=1)
    tgt = torch.empty((B, 6), device=dev)
    ms_drr = _event_ms(torch, lambda: src.batch(net.x, tgt), flush, reps=3)

    def step():
        net.forward()
        net.loss_grad(tgt)
        net.backward()

    ms_net = _event_ms(torch, step, flush, reps=5)
    ms_fwd = _event_ms(torch, net.forward, flush, reps=5)
    net.implicit = False
    ms_fwd_explicit = _event_ms(torch, net.forward, flush, reps=5)
    net.implicit = True
    convs = conv_layers(pb, torch, dev, flush, bf16_peak)
    status = pb.pn_status()
    return {"gemm": gem, "conv_layers": convs,
            "roofline": {"bound": "tensor", "kernel": "k_gemm_bf16 (tcgen05.mma kind::f16, TMEM accumulator, TMA)",
                         "achieved": top["tflops"], "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": top["tflops"] / bf16_peak,
                         "shape": "%dx%dx%d" % (top["M"], top["N"], top["K"]),
                         "peak_from": "MEASURED_PEAKS.json bf16_tflops (cuBLAS 8192^3 burst)"},
            "drr_batch_ms": ms_drr, "drr_batch": "256 poses x 2 views of 384^2 (K2), box-downsampled to 128^2",
            "net_train_step_ms": ms_net, "net_forward_ms": ms_fwd,
            "net_forward_ms_im2col_gemm": ms_fwd_explicit,
            "training_drrs_per_s": B / ((ms_drr + ms_net) * 1e-3),
            "device_status": status}


def posenet_eval(pb, torch, dev, g, mu_d):
    from paper_2508_13304_b300 import posenet as pn
    net = pn.PoseNet(256, in_hw=128, n_views=2)
    src = pn.DrrSource(g, mu_d, 256, factor=3, seed=1)
    t0 = time.perf_counter()
    hist = pn.train(net, src, 200000, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    res = pn.proposal_vs_multistart(net, src, mu_d, n_targets=8, n_starts=16,
                                    lr_refine=[0.5] * 3 + [math.radians(0.2)] * 3)
    res.update({"train_s": train_s, "train_drrs": 200000, "final_loss": float(hist[-50:].mean()),
                "config": "256^3 / 2 x 384^2 (registration phantom), poses +-40 mm / +-30 deg, 8 targets, "
                          "16 random starts, Adam 10 mm / 2 deg, stops off, tolerance 0.5 mm / 0.5 deg"})
    return res


# ------------------------------------------------------------------ main arm

def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import paper_2508_13304_b300 as pb
    from paper_2508_13304_b300 import build
    build.build()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.section == "forward":
        dev0 = torch.device("cuda", local)
        fl = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev0)
        w0 = workload(64)
        g0 = w0["geom"]
        iv0, ip0 = instance_maps(64, g0.n_views)
        P0 = pb.Projector(g0, n_pose=64, inst_view=iv0, inst_pose=ip0, ops=pb.PROJ_OP_FORWARD | pb.PROJ_OP_ADJOINT)
        pb.proj_enable_kernel_timing(P0.plan)
        P0.set_volume(torch.from_numpy(w0["mu"]).to(dev0))
        pose0 = torch.from_numpy(w0["poses"]).to(dev0)
        out0 = torch.empty((P0.n_inst, g0.nv, g0.nu), device=dev0)
        ms0 = _timed(lambda: pb.proj_forward(P0.plan, pose0, out0, P0.ws), P0.plan, pb, fl)
        vol0 = torch.empty((g0.nz, g0.ny, g0.nx), device=dev0)
        ms1 = _timed(lambda: pb.proj_forward_adjoint(P0.plan, out0, pose0, vol0, P0.ws), P0.plan, pb, fl)
        print(json.dumps({"section": "forward", "kernel": "k_forward", "kernel_ms": ms0,
                          "k_forward_adjoint_ms": ms1, "config": "256^3, 128 view instances of 384^2"}), flush=True)
        return
    if args.section == "batch":
        dev0 = torch.device("cuda", local)
        fl = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev0)
        print(json.dumps({"section": "batch", **uneven_batch(pb, torch, dev0, fl, False, args.batch_problems)}),
              flush=True)
        return
    if args.section == "c1":
        dev0 = torch.device("cuda", local)
        fl = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev0)
        print(json.dumps({"section": "c1", **c1_small(pb, torch, dev0, fl)}), flush=True)
        return
    if args.section == "moco":
        print(json.dumps({"section": "moco", **moco_quality(pb, torch, torch.device("cuda", local))}), flush=True)
        return
    if args.section == "registration500":
        print(json.dumps({"section": "registration500", **registration_500(pb, torch, torch.device("cuda", local))}),
              flush=True)
        return
    if args.section == "tables":
        dev0 = torch.device("cuda", local)
        fl = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev0)
        print(json.dumps({"section": "tables", **paper_tables(pb, torch, dev0, fl)}), flush=True)
        return
    if args.section == "accuracy":
        dev0 = torch.device("cuda", local)
        mu0 = torch.from_numpy(workload(1)["mu"]).to(dev0)
        print(json.dumps({"section": "accuracy", **gradient_accuracy(pb, torch, dev0, mu0)}), flush=True)
        return
    if args.section == "back":
        dev0 = torch.device("cuda", local)
        fl = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev0)
        gm = synth.Geometry(256, 256, 256, 0.8, 0.8, 0.8, 512, 512,
                            synth.circular_views(360, synth.SAD, synth.SDD, 0.6, 0.6), 0.4)
        rng0 = np.random.default_rng(1003)
        motion = torch.from_numpy(synth.smooth_motion(rng0, 360, 2.0, 3.0).astype(np.float32)).to(dev0)
        Pb = pb.Projector(gm, n_pose=360, inst_view=np.arange(360), inst_pose=np.arange(360),
                          ops=pb.PROJ_OP_BACK | pb.PROJ_OP_BACK_GRAD)
        pb.proj_enable_kernel_timing(Pb.plan)
        gen = torch.Generator(device=dev0)
        gen.manual_seed(1003)
        img = torch.rand((360, 512, 512), device=dev0, generator=gen)
        wvol = torch.randn((256, 256, 256), device=dev0, generator=gen)
        volb = torch.empty((256, 256, 256), device=dev0)
        gradb = torch.empty((360, 6), device=dev0)
        ms_b = _timed(lambda: pb.proj_back(Pb.plan, img, motion, pb.PROJ_W_FDK, volb, Pb.ws), Pb.plan, pb, fl)
        ms_g = _timed(lambda: pb.proj_back_pose_grad(Pb.plan, img, motion, pb.PROJ_W_FDK, wvol, gradb, Pb.ws),
                      Pb.plan, pb, fl)
        imgb = torch.empty_like(img)
        ms_a = _timed(lambda: pb.proj_back_adjoint(Pb.plan, volb, motion, pb.PROJ_W_FDK, imgb, Pb.ws), Pb.plan, pb, fl)
        print(json.dumps({"section": "back", "k_back_ms": ms_b, "k_back_grad_ms": ms_g, "k_back_adjoint_ms": ms_a,
                          "config": "256^3, 360 views of 512^2, FDK weight"}), flush=True)
        return
    if args.section == "gemm":
        dev0 = torch.device("cuda", local)
        fl = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev0)
        pk = float(load_peaks().get("bf16_tflops", 1800.0))
        print(json.dumps({"section": "gemm", "gemm": gemm_throughput(pb, torch, dev0, fl, pk),
                          "conv_layers": conv_layers(pb, torch, dev0, fl, pk)}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    w = workload(args.n_cand)
    if world > 1 and rank > 0:
        # every rank registers its own candidates against the same target: rank 0 keeps the
        # single-GPU workload's, the others draw theirs from seeds of their own (same ranges)
        w["poses"] = np.ascontiguousarray(
            synth.random_poses(np.random.default_rng(1002 + 7919 * rank), args.n_cand, 15.0, 20.0), dtype=np.float32)
    g = w["geom"]
    iv, ip = instance_maps(args.n_cand, g.n_views)
    P = pb.Projector(g, n_pose=args.n_cand, inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_FORWARD_GRAD)
    mu_d = torch.from_numpy(w["mu"]).to(dev)
    pose_d = torch.from_numpy(w["poses"]).to(dev)
    # target projections at the true pose, rendered once by the forward projector (input data only)
    Pt = pb.Projector(g, n_pose=1, inst_view=np.arange(g.n_views), inst_pose=np.zeros(g.n_views, np.int32),
                      ops=pb.PROJ_OP_FORWARD)
    Pt.set_volume(mu_d)
    target_d = Pt.forward(torch.from_numpy(w["pose_true"]).to(dev)).contiguous()
    grad_d = torch.empty((args.n_cand, 6), device=dev)
    loss_d = torch.empty((args.n_cand,), device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    samples = int(P.count_samples(pose_d).sum().item())
    pb.proj_set_volume(P.plan, mu_d, P.ws)
    marched = int(P.count_marched_samples(pose_d).sum().item())   # gathered after empty-space skipping
    skip_edge = pb.proj_get_skip_brick(P.plan)
    skip_cells = pb.proj_get_skip_cells(P.plan)
    pb.proj_set_skip_cells(P.plan, pb.SKIP_CELLS_OFF)
    brick_range = int(P.count_marched_samples(pose_d).sum().item())  # samples inside the occupied bricks' range
    pb.proj_set_skip_cells(P.plan, skip_cells)
    pb.proj_enable_kernel_timing(P.plan)

    def step():
        pb.proj_set_volume(P.plan, mu_d, P.ws)
        pb.proj_forward_pose_grad(P.plan, pose_d, pb.PROJ_LOSS_NCC, target_d, grad_d, loss_d, None, P.ws)

    stream = torch.cuda.current_stream()
    clocks = clock_sampler(dev, local).__enter__()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms, kern_ms = [], []
    if True:
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(pb.proj_kernel_time_ms(P.plan))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    clocks.__exit__()
    # the same launch's gathers without the arithmetic: the empirical gather ceiling
    probe_ms = []
    for _ in range(3):
        flush.zero_()
        pb.proj_gather_probe(P.plan, pose_d, P.ws)
        probe_ms.append(pb.proj_kernel_time_ms(P.plan))
    probe_ms = float(np.median(probe_ms))
    # the same march with empty-space skipping off (every sample of the box gathered): results are identical
    pb.proj_set_skip_brick(P.plan, 0)
    pb.proj_set_skip_cells(P.plan, pb.SKIP_CELLS_OFF)
    dense_ms, dense_probe_ms = [], []
    for _ in range(3):
        flush.zero_()
        pb.proj_forward_pose_grad(P.plan, pose_d, pb.PROJ_LOSS_NCC, target_d, grad_d, loss_d, None, P.ws)
        dense_ms.append(pb.proj_kernel_time_ms(P.plan))
        flush.zero_()
        pb.proj_gather_probe(P.plan, pose_d, P.ws)
        dense_probe_ms.append(pb.proj_kernel_time_ms(P.plan))
    dense_marched = int(P.count_marched_samples(pose_d).sum().item())
    pb.proj_set_skip_brick(P.plan, skip_edge)
    pb.proj_set_skip_cells(P.plan, skip_cells)
    pb.proj_forward_pose_grad(P.plan, pose_d, pb.PROJ_LOSS_NCC, target_d, grad_d, loss_d, None, P.ws)
    dense_ms, dense_probe_ms = float(np.median(dense_ms)), float(np.median(dense_probe_ms))
    if dist:
        dist.barrier()
    from paper_2508_13304_b300.multigpu import aggregate_rate, max_over_ranks
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms_per_step = total_ms / args.steps
    value = aggregate_rate(world * args.n_cand, args.steps, total_ms)
    k_ms = sum(kern_ms) / len(kern_ms)
    clk = clocks.summary()
    grad_h = grad_d.cpu().numpy().astype(np.float64)

    # -------------------------------------------------------------- plain path
    plain = None
    if not args.no_plain:
        P1 = pb.Projector(g, n_pose=1, inst_view=np.arange(g.n_views), inst_pose=np.zeros(g.n_views, np.int32),
                          ops=pb.PROJ_OP_FORWARD_GRAD)
        g1 = torch.empty((1, 6), device=dev)
        l1 = torch.empty((1,), device=dev)
        singles = [pose_d[c:c + 1].contiguous() for c in range(args.n_cand)]

        def plain_step():
            pb.proj_set_volume(P1.plan, mu_d, P1.ws)
            for c in range(args.n_cand):
                pb.proj_forward_pose_grad(P1.plan, singles[c], pb.PROJ_LOSS_NCC, target_d, g1, l1, None, P1.ws)

        plain_step()
        torch.cuda.synchronize()
        pms = []
        for _ in range(max(2, args.steps // 3)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plain_step()
            e1.record(stream)
            e1.synchronize()
            pms.append(e0.elapsed_time(e1))
        pm = sum(pms) / len(pms)
        plain = {"value": args.n_cand / (pm * 1e-3), "unit": UNIT, "ms_per_step": pm,
                 "what": "64 sequential single-candidate calls (2 instances each), same kernels"}

    # -------------------------------------------------------------- end to end
    mu_h = torch.from_numpy(w["mu"]).pin_memory()
    pose_h = torch.from_numpy(w["poses"]).pin_memory()
    target_h = target_d.cpu().pin_memory()
    grad_o = torch.empty((args.n_cand, 6)).pin_memory()
    loss_o = torch.empty((args.n_cand,)).pin_memory()
    mu_e = torch.empty_like(mu_d)
    pose_e = torch.empty_like(pose_d)
    target_e = torch.empty_like(target_d)

    def e2e_step():
        mu_e.copy_(mu_h, non_blocking=True)
        target_e.copy_(target_h, non_blocking=True)
        pose_e.copy_(pose_h, non_blocking=True)
        pb.proj_set_volume(P.plan, mu_e, P.ws)
        pb.proj_forward_pose_grad(P.plan, pose_e, pb.PROJ_LOSS_NCC, target_e, grad_d, loss_d, None, P.ws)
        grad_o.copy_(grad_d, non_blocking=True)
        loss_o.copy_(loss_d, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    ems = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        ems.append(e0.elapsed_time(e1))
    em_serial = sum(ems) / len(ems)
    # the same steps through the streaming pipeline: step k+1's inputs are copied while step k computes
    from paper_2508_13304_b300.pipeline import PoseGradPipeline
    pipe = PoseGradPipeline(P, pb.PROJ_LOSS_NCC, g.n_views)
    for _ in range(2):
        pipe.submit(mu_h, target_h, pose_h, grad_o, loss_o)
    pipe.synchronize()
    flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        pipe.submit(mu_h, target_h, pose_h, grad_o, loss_o)
    e1.record(stream)
    e1.synchronize()
    if world > 1:
        dist.barrier()
    # whole job: every rank's candidates over the slowest rank's time
    em = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    em_serial = max_over_ranks(em_serial, dist, dev)
    h2d = mu_h.numel() * 4 + target_h.numel() * 4 + pose_h.numel() * 4
    d2h = grad_o.numel() * 4 + loss_o.numel() * 4

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks = load_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    l1_peak = n_sm * L1_BYTES_PER_CLK_SM * sm_max * 1e6 / 1e9                 # GB/s
    alu_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12                            # TFLOP/s
    l1_achieved = marched * L1_BYTES_PER_SAMPLE / (k_ms * 1e-3) / 1e9
    alu_achieved = marched * FLOP_PER_SAMPLE / (k_ms * 1e-3) / 1e12
    l1_dense = dense_marched * L1_BYTES_PER_SAMPLE / (dense_ms * 1e-3) / 1e9
    npad = (g.nx + 2) * (g.ny + 2) * (g.nz + 2)
    hbm_bytes = npad * 16 + g.n_views * g.nu * g.nv * 4 + args.n_cand * 6 * 4  # compulsory: float4 volume, targets
    hbm_achieved = hbm_bytes / (k_ms * 1e-3) / 1e9
    src_sha = kernel_source_sha16()
    ncu_current = src_sha == NCU_SOURCE_SHA16
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_dict(args),
        "ray_samples_per_s": world * marched * args.steps / (total_ms * 1e-3),
        "effective_ray_samples_per_s": world * samples * args.steps / (total_ms * 1e-3),
        "rays_per_s": world * args.n_cand * g.n_views * g.nu * g.nv * args.steps / (total_ms * 1e-3),
        "samples_per_step": samples,
        "marched_samples_per_step": marched,
        "kernel_ms": k_ms,
        "empty_space_skipping": {
            "brick_edge": skip_edge, "cell_test": skip_cells, "marched_samples": marched,
            "brick_range_samples": brick_range, "box_samples": samples,
            "gradient_box_samples": dense_marched, "kernel_ms_without_skipping": dense_ms,
            "value_without_skipping_kernel_only": world * args.n_cand / (dense_ms * 1e-3),
            "l1_frac_without_skipping": l1_dense / l1_peak,
            "probe_ms_without_skipping": dense_probe_ms,
            "what": "each ray marches only its samples around the occupied 8^3-cell bricks it crosses, and "
                    "within them gathers only the samples whose cell has a non-zero corner (the left-out "
                    "samples read eight zero corners); results are bit-identical with skipping off.  "
                    "ray_samples_per_s counts the samples gathered, effective_ray_samples_per_s all samples of "
                    "the box (the sum of Eq. forward)"},
        "plain": plain,
        "roofline": {"bound": "l1", "achieved": l1_achieved, "peak": l1_peak, "unit": "GB/s",
                     "frac": l1_achieved / l1_peak, "traffic": TRAFFIC_PER_LAUNCH if ncu_current else None,
                     "ncu_source_sha16": NCU_SOURCE_SHA16, "built_source_sha16": src_sha,
                     "kernel": "k_forward_grad<NCC> (fused pose-gradient march)",
                     "what": "L1->register gather bytes: %d B per ray sample (8 corners x float4); peak = %d SMs x "
                             "%d B/clk x %.0f MHz" % (L1_BYTES_PER_SAMPLE, n_sm, L1_BYTES_PER_CLK_SM, sm_max),
                     "alu": {"achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                             "frac": alu_achieved / alu_peak, "flop_per_sample": FLOP_PER_SAMPLE},
                     # the units that bind, from the committed ncu capture of the same kernel (a small case of
                     # this launch; not measured live): instruction issue, then the L1 data pipe
                     "ncu_l1_wavefront_utilisation": {
                         "pct_of_peak": NCU_L1_WAVEFRONT_PCT if ncu_current else None,
                         "source": "ncu l1tex__data_pipe_lsu_wavefronts of the same kernel, 8-instance case "
                                   "(summary under profiles/)"},
                     "ncu_issue_active": {
                         "pct_of_peak": NCU_ISSUE_ACTIVE_PCT if ncu_current else None,
                         "source": "ncu smsp__issue_active of the same kernel, 8-instance case"},
                     "empirical_gather_ceiling": {
                         "kernel_ms": probe_ms, "ray_samples_per_s": marched / (probe_ms * 1e-3),
                         "frac": probe_ms / k_ms,
                         "what": "proj_gather_probe: the same launch's rays, samples, volume copies and eight "
                                 "16-byte corner loads per sample without the interpolation and accumulation"},
                     "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                             "frac": hbm_achieved / hbm_peak, "compulsory_bytes": hbm_bytes,
                             "peak_from": "MEASURED_PEAKS.json hbm_gbs"}},
        "e2e": {"value": world * args.n_cand / (em * 1e-3), "unit": UNIT, "h2d_bytes_per_step": world * h2d,
                "d2h_bytes_per_step": world * d2h, "ms_per_step": em,
                "what": "PoseGradPipeline: pinned host volume, targets and poses copied in and gradients and "
                        "losses copied out every step; step k+1's copies overlap step k's compute; no L2 flush "
                        "between steps (the two 285 MB (mu, grad mu) copies exceed L2)",
                "serial_value": world * args.n_cand / (em_serial * 1e-3), "serial_ms_per_step": em_serial},
        # per step and rank: k_volume_prep (both (mu, grad mu) copies), k_cell_bits, k_brick_maps8,
        # k_brick_maps16, k_cell_decide (proj_set_volume, plus one memset of the cell-test counters), k_setup,
        # k_forward_grad, k_forward_grad_reduce (proj_forward_pose_grad)
        "gpu_launches": 8 * args.steps * world,
        "clocks": clk,
        "wall_s_timed_region": wall,
    }
    if not args.no_secondary:
        line["secondary"] = secondary(pb, torch, dev, w, mu_d, flush)
    if args.posenet_eval:
        line["posenet_eval"] = posenet_eval(pb, torch, dev, g, mu_d)
    if not args.no_cpu_baseline and world == 1:
        cands = list(range(min(args.cpu_sample, args.n_cand)))
        og, dt, threads, _ = cpu_oracle_eval(w, cands)
        err = 0.0
        for i, c in enumerate(cands):
            for blk in (slice(0, 3), slice(3, 6)):
                err = max(err, float(np.linalg.norm(grad_h[c, blk] - og[i, blk]) / np.linalg.norm(og[i, blk])))
        line["cpu_baseline"] = {"value": len(cands) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "%d of %d candidates (2 views 384^2, 256^3), NCC forward + gradient"
                                          % (len(cands), args.n_cand)}
        line["grad_rel_err_vs_oracle"] = err
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

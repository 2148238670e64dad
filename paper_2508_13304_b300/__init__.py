"""Python binding of the sm_103a cone-beam projector library (libproj.so).

The functions below carry the names of the C ABI in include/proj.h and only
marshal arguments: torch CUDA tensors become device pointers, the current
torch stream becomes the cudaStream_t, and a non-zero status becomes a
``ProjError``.  Every step of the computation runs in the library's CUDA
kernels; there is no CPU fallback.  ``Projector`` bundles a plan with a
torch-allocated workspace for convenience.

Importing this package does not load the library; the first call does, and
raises ``RuntimeError`` if libproj.so has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libproj.so")

# Constants of include/proj.h.
PROJ_OK, PROJ_E_ARG, PROJ_E_CUDA, PROJ_E_WORKSPACE, PROJ_E_UNSUPPORTED, PROJ_E_DEVICE = 0, -1, -2, -3, -4, -5
PROJ_LOSS_RESIDUAL, PROJ_LOSS_L2, PROJ_LOSS_NCC = 0, 1, 2
PROJ_W_NONE, PROJ_W_FDK, PROJ_W_FDK_CONST = 0, 1, 2
PROJ_OP_FORWARD, PROJ_OP_FORWARD_GRAD, PROJ_OP_BACK, PROJ_OP_BACK_GRAD, PROJ_OP_ADJOINT = 1, 2, 4, 8, 16
PROJ_OP_SHARPNESS = 32
PROJ_OP_ALL = 63
PROJ_FLAG_ONE_COPY = 256
PROJ_FLAG_BRICKS = 512
PROJ_STATUS_BAD_POSE = 1
PROJ_STATUS_BAD_INDEX = 2


class ProjError(RuntimeError):
    """A library call returned a non-zero status."""

    def __init__(self, code, msg):
        super().__init__("proj error %d: %s" % (code, msg))
        self.code = code


class proj_geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("vz", ctypes.c_double),
                ("vol_offset", ctypes.c_double * 3),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int), ("n_views", ctypes.c_int),
                ("views", ctypes.POINTER(ctypes.c_double)),
                ("step", ctypes.c_double)]


_P = ctypes.c_void_p
_SZ = ctypes.c_size_t
_I = ctypes.c_int
_SIGS = {
    "proj_plan_create": [ctypes.POINTER(proj_geometry), _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), _I,
                         ctypes.POINTER(_P)],
    "proj_plan_destroy": [_P],
    "proj_workspace_size": [_P, ctypes.POINTER(_SZ)],
    "proj_set_volume": [_P, _P, _P, _SZ, _P],
    "proj_forward": [_P, _P, _P, _P, _SZ, _P],
    "proj_forward_pose_grad": [_P, _P, _I, _P, _P, _P, _P, _P, _SZ, _P],
    "proj_forward_pose_grad_list": [_P, _P, _P, _I, _I, _P, _P, _P, _P, _P, _SZ, _P],
    "proj_back": [_P, _P, _P, _I, _P, _P, _SZ, _P],
    "proj_back_pose_grad": [_P, _P, _P, _I, _P, _P, _P, _SZ, _P],
    "proj_back_adjoint": [_P, _P, _P, _I, _P, _P, _SZ, _P],
    "proj_forward_adjoint": [_P, _P, _P, _P, _P, _SZ, _P],
    "proj_check": [_P, _P, _SZ, _P, ctypes.POINTER(_I)],
    "proj_count_samples": [_P, _P, _P, _P, _SZ, _P],
    "proj_forward_pose_grad_static": [ctypes.POINTER(proj_geometry), _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                      _P, _P, _I, _P, _P, _P, _P],
    "proj_fdk_filter": [_P, _P, ctypes.c_float, _P, _P],
    "proj_sharpness": [_P, _P, _P, _P, _P, _SZ, _P],
    "proj_pose_adam": [_P, _P, _P, _P, _P, _P, _I, ctypes.POINTER(ctypes.c_float)] + [ctypes.c_float] * 3 + [_P],
    "proj_registration_step": [_I, _I] + [_P] * 12 + [_I, _P, _P, _P, _P],
    "proj_gather_probe": [_P, _P, _P, _SZ, _P],
    "proj_set_warp_shape": [_P, _I],
    "proj_get_warp_shape": [_P, ctypes.POINTER(_I)],
    "proj_autotune_forward_grad": [_P, _P, _I, _P, _P, _SZ, _P, _I, ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(_I)],
    "proj_set_skip_brick": [_P, _I],
    "proj_get_skip_brick": [_P, ctypes.POINTER(_I)],
    "proj_set_skip_cells": [_P, _I],
    "proj_get_skip_cells": [_P, ctypes.POINTER(_I)],
    "proj_autotune_march": [_P, _P, _I, _P, _P, _SZ, _P, _I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I),
                            ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "proj_count_marched_samples": [_P, _P, _P, _P, _SZ, _P],
    "proj_set_brick_shape": [_P, _I],
    "proj_get_brick_shape": [_P, ctypes.POINTER(_I)],
    "proj_autotune_back_grad": [_P, _P, _P, _I, _P, _P, _SZ, _P, _I, ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(_I)],
    "proj_batch_create": [_I, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_P), ctypes.POINTER(_P),
                          ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_SZ),
                          ctypes.POINTER(_P)],
    "proj_batch_run": [_P, _P],
    "proj_batch_destroy": [_P],
    "pn_gemm_bf16": [_I, _I, _I, _P, _I, _P, _I, _P, _P, _I, _I, _P, _P, _I, _I, _P, _P],
    "pn_gemm_split_hint": [_I, _I, _I],
    "pn_gemm_use_pair_tiles": [_I],
    "pn_im2col_3x3s2": [_P, _I, _I, _I, _I, _I, _P, _P],
    "pn_conv3x3s2_bf16": [_P, _I, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P],
    "pn_col2im_3x3s2": [_P, _I, _I, _I, _I, _I, _P, _P, _P, _P],
    "pn_conv3x3s2_dgrad_bf16": [_P, _I, _I, _I, _I, _P, _I, _P, _P, _P, _P],
    "pn_conv_dgrad_weights": [_P, _I, _I, _P, _P],
    "pn_adam_step": [_P, _P, _P, _P, ctypes.c_longlong] + [ctypes.c_float] * 7 + [_P, _P],
    "pn_transpose_bf16": [_P, _I, _I, _P, _I, _P],
    "pn_colsum_scratch_floats": [_I, _I],
    "pn_colsum_bf16": [_P, _I, _I, _I, _P, _P, _P],
    "pn_prepare_images": [_P, _I, _I, _I, _I, _I, _P, _P],
    "pn_mse_loss": [_P, _I, _I, _I, _P, _P, _P, _I, _P],
    "pn_to_bf16": [_P, ctypes.c_longlong, _P, _P],
    "pn_status": [_P, ctypes.POINTER(_I)],
    "pn_gemm_test_hooks": [ctypes.c_ulonglong, _I],
    "proj_enable_kernel_timing": [_P, _I],
    "proj_kernel_time_ms": [_P, ctypes.POINTER(ctypes.c_float)],
    "proj_last_error": [],
    "proj_version": [],
}

_lib = None


def lib():
    """The loaded libproj.so (loaded on first use)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libproj.so is not built; run python -m paper_2508_13304_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = (ctypes.c_char_p if name in ("proj_last_error", "proj_version") else
                         ctypes.c_size_t if name == "pn_colsum_scratch_floats" else ctypes.c_int)
        _lib = L
    return _lib


def proj_last_error() -> str:
    return lib().proj_last_error().decode()


def proj_version() -> str:
    return lib().proj_version().decode()


def _check(rc):
    if rc != PROJ_OK:
        raise ProjError(rc, proj_last_error())
    return rc


def _ptr(t, dtype=None, numel=None, name="tensor", allow_none=False):
    """Device pointer of a contiguous CUDA tensor (argument checks only)."""
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Plan:
    """Handle of a proj_plan plus the host-side sizes the binding checks."""

    def __init__(self, handle, geom, n_pose, inst_view, inst_pose, ops):
        self.handle = handle
        self.geom = geom
        self.n_pose = n_pose
        self.inst_view = np.asarray(inst_view, dtype=np.int32)
        self.inst_pose = np.asarray(inst_pose, dtype=np.int32)
        self.n_inst = len(self.inst_view)
        self.ops = ops

    @property
    def vol_numel(self):
        return self.geom.nx * self.geom.ny * self.geom.nz

    @property
    def img_numel(self):
        return self.geom.nu * self.geom.nv

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.proj_plan_destroy(self.handle)
            self.handle = None


def make_geometry(geom):
    """proj_geometry from any object with the fields nx..step (views as a
    [n_views][12] array); returns (struct, views array kept alive)."""
    views = np.ascontiguousarray(geom.views, dtype=np.float64).reshape(-1, 12)
    off = tuple(getattr(geom, "off", (0.0, 0.0, 0.0)))
    g = proj_geometry(int(geom.nx), int(geom.ny), int(geom.nz), float(geom.vx), float(geom.vy), float(geom.vz),
                      (ctypes.c_double * 3)(*off), int(geom.nu), int(geom.nv), views.shape[0],
                      views.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(geom.step))
    return g, views


def proj_plan_create(geom, n_pose, inst_view, inst_pose, ops=PROJ_OP_ALL) -> Plan:
    g, views = make_geometry(geom)
    iv = np.ascontiguousarray(inst_view, dtype=np.int32)
    ip = np.ascontiguousarray(inst_pose, dtype=np.int32)
    if iv.shape != ip.shape:
        raise ValueError("inst_view and inst_pose differ in length")
    h = ctypes.c_void_p()
    _check(lib().proj_plan_create(ctypes.byref(g), int(n_pose), int(iv.size),
                                  iv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  ip.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(ops), ctypes.byref(h)))
    del views
    return Plan(h, geom, int(n_pose), iv, ip, ops)


def proj_plan_destroy(plan: Plan):
    if plan.handle:
        _check(lib().proj_plan_destroy(plan.handle))
        plan.handle = None


def proj_workspace_size(plan: Plan) -> int:
    n = ctypes.c_size_t()
    _check(lib().proj_workspace_size(plan.handle, ctypes.byref(n)))
    return int(n.value)


def _ws(ws):
    return _ptr(ws, name="workspace"), ws.numel() * ws.element_size()


def proj_set_volume(plan: Plan, mu, ws, stream=None):
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_set_volume(plan.handle, _ptr(mu, torch.float32, plan.vol_numel, "mu"), p, nb,
                                 _stream(stream)))


def proj_forward(plan: Plan, pose, proj, ws, stream=None):
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_forward(plan.handle, _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"),
                              _ptr(proj, torch.float32, plan.n_inst * plan.img_numel, "proj"), p, nb,
                              _stream(stream)))


def proj_forward_pose_grad(plan: Plan, pose, loss, ref, grad, loss_out=None, proj_out=None, ws=None,
                           stream=None):
    import torch
    p, nb = _ws(ws)
    n_ref = (plan.n_inst if loss == PROJ_LOSS_RESIDUAL else plan.geom.n_views) * plan.img_numel
    _check(lib().proj_forward_pose_grad(
        plan.handle, _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"), int(loss),
        _ptr(ref, torch.float32, n_ref, "ref"), _ptr(grad, torch.float32, 6 * plan.n_pose, "grad"),
        _ptr(loss_out, torch.float32, plan.n_pose, "loss", allow_none=True),
        _ptr(proj_out, torch.float32, plan.n_inst * plan.img_numel, "proj", allow_none=True), p, nb,
        _stream(stream)))


def proj_forward_pose_grad_list(plan: Plan, pose, pose_list, loss, ref, grad, loss_out=None, proj_out=None, ws=None,
                                stream=None):
    """Pose gradient of the poses in pose_list (int32 CUDA tensor, -1 = empty
    slot); rows of grad / loss_out / proj_out of other poses are untouched."""
    import torch
    p, nb = _ws(ws)
    n_ref = (plan.n_inst if loss == PROJ_LOSS_RESIDUAL else plan.geom.n_views) * plan.img_numel
    n_list = pose_list.numel() if pose_list is not None else 0
    _check(lib().proj_forward_pose_grad_list(
        plan.handle, _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"), _ptr(pose_list, torch.int32, None, "pose_list"),
        int(n_list), int(loss), _ptr(ref, torch.float32, n_ref, "ref"),
        _ptr(grad, torch.float32, 6 * plan.n_pose, "grad"),
        _ptr(loss_out, torch.float32, plan.n_pose, "loss", allow_none=True),
        _ptr(proj_out, torch.float32, plan.n_inst * plan.img_numel, "proj", allow_none=True), p, nb,
        _stream(stream)))


def proj_back(plan: Plan, proj, pose, weight, vol, ws, stream=None):
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_back(plan.handle, _ptr(proj, torch.float32, plan.n_inst * plan.img_numel, "proj"),
                           _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"), int(weight),
                           _ptr(vol, torch.float32, plan.vol_numel, "vol"), p, nb, _stream(stream)))


def proj_back_adjoint(plan: Plan, vol, pose, weight, proj, ws, stream=None):
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_back_adjoint(plan.handle, _ptr(vol, torch.float32, plan.vol_numel, "vol"),
                                   _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"), int(weight),
                                   _ptr(proj, torch.float32, plan.n_inst * plan.img_numel, "proj"), p, nb,
                                   _stream(stream)))


def proj_back_pose_grad(plan: Plan, proj, pose, weight, vol_resid, grad, ws, stream=None):
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_back_pose_grad(plan.handle, _ptr(proj, torch.float32, plan.n_inst * plan.img_numel, "proj"),
                                     _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"), int(weight),
                                     _ptr(vol_resid, torch.float32, plan.vol_numel, "vol_resid"),
                                     _ptr(grad, torch.float32, 6 * plan.n_pose, "grad"), p, nb, _stream(stream)))


def proj_forward_adjoint(plan: Plan, y, pose, vol, ws, stream=None):
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_forward_adjoint(plan.handle, _ptr(y, torch.float32, plan.n_inst * plan.img_numel, "y"),
                                      _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"),
                                      _ptr(vol, torch.float32, plan.vol_numel, "vol"), p, nb, _stream(stream)))


def proj_count_samples(plan: Plan, pose, count, ws, stream=None):
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_count_samples(plan.handle, _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"),
                                    _ptr(count, torch.int64, plan.n_inst, "count"), p, nb, _stream(stream)))


def proj_check(plan: Plan, ws, stream=None) -> int:
    """Synchronise, read and clear the device status bits (0 = clean)."""
    p, nb = _ws(ws)
    st = ctypes.c_int(0)
    rc = lib().proj_check(plan.handle, p, nb, _stream(stream), ctypes.byref(st))
    if rc not in (PROJ_OK, PROJ_E_DEVICE):
        _check(rc)
    return int(st.value)


def proj_forward_pose_grad_static(geom, n_pose, inst_view, inst_pose, mu, pose, loss, ref, grad, loss_out=None,
                                  stream=None):
    """Allocation-free forward pose gradient (no plan, no workspace): for
    callers that cannot allocate device memory.  Sizes are limited by the
    library's static scratch (a 64^3 volume, 64 instances / poses / views)."""
    import torch
    g, views = make_geometry(geom)
    iv = np.ascontiguousarray(inst_view, dtype=np.int32)
    ip = np.ascontiguousarray(inst_pose, dtype=np.int32)
    if iv.shape != ip.shape:
        raise ValueError("inst_view and inst_pose differ in length")
    # the library uses the current device's scratch and stream: every tensor must live there
    cur = torch.cuda.current_device()
    for t, nm in ((mu, "mu"), (pose, "pose"), (ref, "ref"), (grad, "grad"), (loss_out, "loss")):
        if isinstance(t, torch.Tensor) and t.is_cuda and t.device.index != cur:
            raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (nm, t.device.index, cur))
    n_img = int(geom.nu) * int(geom.nv)
    n_ref = (iv.size if loss == PROJ_LOSS_RESIDUAL else views.shape[0]) * n_img
    _check(lib().proj_forward_pose_grad_static(
        ctypes.byref(g), int(n_pose), int(iv.size), iv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        ip.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        _ptr(mu, torch.float32, int(geom.nx) * int(geom.ny) * int(geom.nz), "mu"),
        _ptr(pose, torch.float32, 6 * int(n_pose), "pose"), int(loss), _ptr(ref, torch.float32, n_ref, "ref"),
        _ptr(grad, torch.float32, 6 * int(n_pose), "grad"),
        _ptr(loss_out, torch.float32, int(n_pose), "loss", allow_none=True), _stream(stream)))


def proj_fdk_filter(plan: Plan, proj, scale, out, stream=None):
    import torch
    n = plan.n_inst * plan.img_numel
    _check(lib().proj_fdk_filter(plan.handle, _ptr(proj, torch.float32, n, "proj"), float(scale),
                                 _ptr(out, torch.float32, n, "out"), _stream(stream)))


def proj_sharpness(plan: Plan, vol, loss, grad=None, ws=None, stream=None):
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_sharpness(plan.handle, _ptr(vol, torch.float32, plan.vol_numel, "vol"),
                                _ptr(loss, torch.float32, 1, "loss"),
                                _ptr(grad, torch.float32, plan.vol_numel, "grad", allow_none=True), p, nb,
                                _stream(stream)))


def proj_pose_adam(pose, grad, m, v, t, active, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    """One Adam step on [n][6] poses in one launch (include/proj.h):
    m, v [n][6] and t [n] (step counts) FP32 state; active [n] bool or None."""
    import torch
    n = pose.shape[0]
    lr6 = (ctypes.c_float * 6)(*[float(x) for x in lr])
    _check(lib().proj_pose_adam(_ptr(pose, torch.float32, 6 * n, "pose"), _ptr(grad, torch.float32, 6 * n, "grad"),
                                _ptr(m, torch.float32, 6 * n, "m"), _ptr(v, torch.float32, 6 * n, "v"),
                                _ptr(t, torch.float32, n, "t"), _ptr(active, torch.bool, n, "active", allow_none=True),
                                int(n), lr6, float(b1), float(b2), float(eps), _stream(stream)))


class RegParams(ctypes.Structure):
    """proj_reg_params of include/proj.h."""
    _fields_ = [("lr", ctypes.c_float * 6), ("b1", ctypes.c_float), ("b2", ctypes.c_float), ("eps", ctypes.c_float),
                ("ncc_stop", ctypes.c_float), ("dloss_stop", ctypes.c_float), ("max_iter", ctypes.c_longlong),
                ("tol_mm", ctypes.c_float), ("tol_deg", ctypes.c_float)]


def reg_params(lr, b1=0.9, b2=0.999, eps=1e-8, ncc_stop=0.999, dloss_stop=1e-5, max_iter=1 << 62, tol=(0.5, 0.5)):
    return RegParams((ctypes.c_float * 6)(*[float(x) for x in lr]), b1, b2, eps, ncc_stop, dloss_stop,
                     int(max_iter), float(tol[0]), float(tol[1]))


def proj_registration_step(pose, grad, loss, last, m, v, t, alive, iters, slots, nxt, truth, hit_any, listed,
                           params, stream=None):
    """One iteration's bookkeeping of a multi-start registration in one launch
    (include/proj.h): hit test, stopping test, masked Adam step, refill of the
    slots of stopped starts.  params: a RegParams (reg_params())."""
    import torch
    n, ns = pose.shape[0], slots.numel()
    n_truth = 0 if truth is None else truth.numel() // 6
    if truth is not None and truth.numel() not in (6, 6 * n):
        raise ValueError("truth must hold 1 or n = %d poses" % n)
    _check(lib().proj_registration_step(
        int(n), int(ns), _ptr(pose, torch.float32, 6 * n, "pose"), _ptr(grad, torch.float32, 6 * n, "grad"),
        _ptr(loss, torch.float32, n, "loss"), _ptr(last, torch.float32, n, "last"),
        _ptr(m, torch.float32, 6 * n, "m"), _ptr(v, torch.float32, 6 * n, "v"), _ptr(t, torch.float32, n, "t"),
        _ptr(alive, torch.bool, n, "alive"), _ptr(iters, torch.int64, n, "iters"),
        _ptr(slots, torch.int32, ns, "slots"), _ptr(nxt, torch.int64, 1, "next"),
        _ptr(truth, torch.float32, None, "truth", allow_none=True), int(n_truth),
        _ptr(hit_any, torch.bool, 1, "hit_any", allow_none=True), _ptr(listed, torch.bool, n, "listed"),
        ctypes.byref(params), _stream(stream)))


WARP_WIDTHS = (2, 4, 8, 16)


def proj_gather_probe(plan: Plan, pose, ws, stream=None):
    """The fused march's gathers without its arithmetic (empirical ceiling)."""
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_gather_probe(plan.handle, _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"), p, nb,
                                   _stream(stream)))


def proj_set_warp_shape(plan: Plan, warp_width: int):
    _check(lib().proj_set_warp_shape(plan.handle, int(warp_width)))


def proj_get_warp_shape(plan: Plan) -> int:
    w = ctypes.c_int()
    _check(lib().proj_get_warp_shape(plan.handle, ctypes.byref(w)))
    return int(w.value)


def proj_autotune_forward_grad(plan: Plan, pose, loss, ref, ws, reps=3, stream=None):
    """Time the fused march per warp shape on this data, keep the fastest in
    the plan; returns (warp_width, {width: ms per launch})."""
    import torch
    p, nb = _ws(ws)
    n_ref = (plan.n_inst if loss == PROJ_LOSS_RESIDUAL else plan.geom.n_views) * plan.img_numel
    times = (ctypes.c_float * 4)()
    w = ctypes.c_int()
    _check(lib().proj_autotune_forward_grad(plan.handle, _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"),
                                            int(loss), _ptr(ref, torch.float32, n_ref, "ref"), p, nb,
                                            _stream(stream), int(reps), times, ctypes.byref(w)))
    return int(w.value), dict(zip(WARP_WIDTHS, [float(t) for t in times]))


SKIP_BRICK_EDGES = (0, 8, 16)


def proj_set_skip_brick(plan: Plan, edge: int):
    """Empty-space skipping of the forward marches: brick edge 8, 16 or 0 (off)."""
    _check(lib().proj_set_skip_brick(plan.handle, int(edge)))


def proj_get_skip_brick(plan: Plan) -> int:
    e = ctypes.c_int()
    _check(lib().proj_get_skip_brick(plan.handle, ctypes.byref(e)))
    return int(e.value)


SKIP_CELLS_OFF, SKIP_CELLS_ON, SKIP_CELLS_AUTO = 0, 1, 2


def proj_set_skip_cells(plan: Plan, mode: int):
    """Per-sample cell test of the fused march (empty-space skipping inside the
    brick range): SKIP_CELLS_OFF, SKIP_CELLS_ON or SKIP_CELLS_AUTO (default)."""
    _check(lib().proj_set_skip_cells(plan.handle, int(mode)))


def proj_get_skip_cells(plan: Plan) -> int:
    v = ctypes.c_int()
    _check(lib().proj_get_skip_cells(plan.handle, ctypes.byref(v)))
    return int(v.value)


def proj_autotune_march(plan: Plan, pose, loss, ref, ws, reps=3, stream=None):
    """Time the fused march per (skip brick edge, cell test, warp shape) on this
    data, keep the fastest in the plan; returns (warp_width, brick_edge,
    skip_cells, {(edge, cells, width): ms})."""
    import torch
    p, nb = _ws(ws)
    n_ref = (plan.n_inst if loss == PROJ_LOSS_RESIDUAL else plan.geom.n_views) * plan.img_numel
    times = (ctypes.c_float * 24)()
    w, e, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().proj_autotune_march(plan.handle, _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"), int(loss),
                                     _ptr(ref, torch.float32, n_ref, "ref"), p, nb, _stream(stream), int(reps), times,
                                     ctypes.byref(w), ctypes.byref(e), ctypes.byref(c)))
    tt = {(SKIP_BRICK_EDGES[j], cl, WARP_WIDTHS[i]): float(times[4 * (2 * j + cl) + i])
          for j in range(3) for cl in (0, 1) for i in range(4)}
    return int(w.value), int(e.value), int(c.value), tt


def proj_count_marched_samples(plan: Plan, pose, count, ws, stream=None):
    import torch
    p, nb = _ws(ws)
    _check(lib().proj_count_marched_samples(plan.handle, _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"),
                                            _ptr(count, torch.int64, plan.n_inst, "count"), p, nb, _stream(stream)))


# brick shapes of the back-projection gradient: (voxels per thread along z, instances per block)
BRICK_SHAPES = ((16, 8), (8, 8), (16, 16), (8, 16))


def proj_set_brick_shape(plan: Plan, shape: int):
    _check(lib().proj_set_brick_shape(plan.handle, int(shape)))


def proj_get_brick_shape(plan: Plan) -> int:
    b = ctypes.c_int()
    _check(lib().proj_get_brick_shape(plan.handle, ctypes.byref(b)))
    return int(b.value)


def proj_autotune_back_grad(plan: Plan, proj, pose, weight, vol_resid, ws, reps=3, stream=None):
    """Time the back-projection gradient per brick shape on this data, keep
    the fastest in the plan; returns (shape, {shape: ms per launch})."""
    import torch
    p, nb = _ws(ws)
    times = (ctypes.c_float * 4)()
    b = ctypes.c_int()
    _check(lib().proj_autotune_back_grad(plan.handle, _ptr(proj, torch.float32, plan.n_inst * plan.img_numel, "proj"),
                                         _ptr(pose, torch.float32, 6 * plan.n_pose, "pose"), int(weight),
                                         _ptr(vol_resid, torch.float32, plan.vol_numel, "vol_resid"), p, nb,
                                         _stream(stream), int(reps), times, ctypes.byref(b)))
    return int(b.value), {k: float(t) for k, t in enumerate(times)}


class Batch:
    """Handle of a proj_batch; keeps the bound plans and tensors alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().proj_batch_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def proj_batch_create(problems) -> Batch:
    """Bind independent forward pose-gradient problems for one persistent
    launch.  problems: sequence of dicts with keys plan, loss, pose, ref, grad,
    ws and optionally loss_out (same meaning as in proj_forward_pose_grad)."""
    import torch
    n = len(problems)
    if n < 1:
        raise ValueError("need at least one problem")
    plans = (_P * n)()
    losses = (_I * n)()
    poses, refs, grads, louts, wss = (_P * n)(), (_P * n)(), (_P * n)(), (_P * n)(), (_P * n)()
    nbs = (_SZ * n)()
    for i, q in enumerate(problems):
        plan, loss = q["plan"], int(q["loss"])
        n_ref = (plan.n_inst if loss == PROJ_LOSS_RESIDUAL else plan.geom.n_views) * plan.img_numel
        plans[i] = plan.handle
        losses[i] = loss
        poses[i] = _ptr(q["pose"], torch.float32, 6 * plan.n_pose, "pose")
        refs[i] = _ptr(q["ref"], torch.float32, n_ref, "ref")
        grads[i] = _ptr(q["grad"], torch.float32, 6 * plan.n_pose, "grad")
        louts[i] = _ptr(q.get("loss_out"), torch.float32, plan.n_pose, "loss", allow_none=True)
        wss[i], nbs[i] = _ws(q["ws"])
    h = _P()
    _check(lib().proj_batch_create(n, plans, losses, poses, refs, grads, louts, wss, nbs, ctypes.byref(h)))
    return Batch(h.value, list(problems))


def proj_batch_run(batch: Batch, stream=None):
    _check(lib().proj_batch_run(batch.handle, _stream(stream)))


def proj_batch_destroy(batch: Batch):
    if batch.handle:
        _check(lib().proj_batch_destroy(batch.handle))
        batch.handle = None


def proj_enable_kernel_timing(plan: Plan, enable=True):
    _check(lib().proj_enable_kernel_timing(plan.handle, 1 if enable else 0))


def proj_kernel_time_ms(plan: Plan) -> float:
    ms = ctypes.c_float()
    _check(lib().proj_kernel_time_ms(plan.handle, ctypes.byref(ms)))
    return float(ms.value)


# ------------------------------------------------------- network kernels (posenet.h)

def _bf(t, numel=None, name="tensor", allow_none=False):
    import torch
    return _ptr(t, torch.bfloat16, numel, name, allow_none)


def _f32(t, numel=None, name="tensor", allow_none=False):
    import torch
    return _ptr(t, torch.float32, numel, name, allow_none)


def pn_gemm_bf16(M, N, K, A, lda, B, ldb, bias=None, mask=None, ldm=0, relu=False, D32=None, D16=None, ldd=None,
                 split_k=1, part=None, stream=None):
    """D = epilogue(A . B^T) on the tensor cores (see include/posenet.h)."""
    ldd = N if ldd is None else ldd
    if A is None or B is None or A.numel() < (M - 1) * lda + K or B.numel() < (N - 1) * ldb + K:
        raise ValueError("A or B smaller than the stated shape")
    for t, nm in ((D32, "D32"), (D16, "D16")):
        if t is not None and t.numel() < (M - 1) * ldd + N:
            raise ValueError("%s smaller than the stated shape" % nm)
    if mask is not None and mask.numel() < (M - 1) * ldm + N:
        raise ValueError("mask smaller than the stated shape")
    if split_k > 1 and (part is None or part.numel() < split_k * M * N):
        raise ValueError("part must hold split_k * M * N floats")
    _check(lib().pn_gemm_bf16(int(M), int(N), int(K), _bf(A, name="A"), int(lda), _bf(B, name="B"), int(ldb),
                              _f32(bias, N, "bias", allow_none=True), _bf(mask, name="mask", allow_none=True),
                              int(ldm), 1 if relu else 0, _f32(D32, name="D32", allow_none=True),
                              _bf(D16, name="D16", allow_none=True), int(ldd), int(split_k),
                              _f32(part, name="part", allow_none=True), _stream(stream)))


def pn_gemm_use_pair_tiles(mode=2) -> int:
    """Tiles of wide GEMMs: 2 persistent 2-SM (default), 1 2-SM per tile, 0 1-SM;
    returns the previous mode."""
    return int(lib().pn_gemm_use_pair_tiles(int(mode)))


def pn_gemm_split_hint(M, N, K) -> int:
    return int(lib().pn_gemm_split_hint(int(M), int(N), int(K)))


def pn_conv3x3s2_bf16(x, B, H, W, C, w, cout, bias=None, relu=False, y32=None, y16=None, stream=None):
    """Implicit-GEMM 3x3 stride-2 convolution (see include/posenet.h)."""
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    _check(lib().pn_conv3x3s2_bf16(_bf(x, B * H * W * C, "x"), B, H, W, C, _bf(w, cout * 9 * C, "w"), int(cout),
                                   _f32(bias, cout, "bias", allow_none=True), 1 if relu else 0,
                                   _f32(y32, B * Ho * Wo * cout, "y32", allow_none=True),
                                   _bf(y16, B * Ho * Wo * cout, "y16", allow_none=True), _stream(stream)))


def pn_conv3x3s2_dgrad_bf16(dy, B, H, W, C, wt, cout, mask=None, dx32=None, dx16=None, stream=None):
    """Implicit-GEMM input gradient of pn_conv3x3s2_bf16 (see include/posenet.h)."""
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    n = B * H * W * C
    _check(lib().pn_conv3x3s2_dgrad_bf16(_bf(dy, B * Ho * Wo * cout, "dy"), B, H, W, C, _bf(wt, C * 9 * cout, "wt"),
                                         int(cout), _bf(mask, n, "mask", allow_none=True),
                                         _f32(dx32, n, "dx32", allow_none=True), _bf(dx16, n, "dx16", allow_none=True),
                                         _stream(stream)))


def pn_conv_dgrad_weights(w, cout, C, wt, stream=None):
    _check(lib().pn_conv_dgrad_weights(_bf(w, cout * 9 * C, "w"), int(cout), int(C), _bf(wt, C * 9 * cout, "wt"),
                                       _stream(stream)))


def pn_adam_step(p, g, m, v, step, b1, b2, eps, decay=1.0, p16=None, stream=None):
    """One Adam step on flat FP32 tensors p, g, m, v (see include/posenet.h)."""
    n = p.numel()
    _check(lib().pn_adam_step(_f32(p, n, "p"), _f32(g, n, "g"), _f32(m, n, "m"), _f32(v, n, "v"), n, float(step),
                              float(b1), 1.0 - float(b1), float(b2), 1.0 - float(b2), float(eps), float(decay),
                              _bf(p16, n, "p16", allow_none=True), _stream(stream)))


def pn_im2col_3x3s2(x, B, H, W, C, kp, col, stream=None):
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    _check(lib().pn_im2col_3x3s2(_bf(x, B * H * W * C, "x"), B, H, W, C, kp, _bf(col, B * Ho * Wo * kp, "col"),
                                 _stream(stream)))


def pn_col2im_3x3s2(dcol, B, H, W, C, kp, mask=None, dx16=None, dx32=None, stream=None):
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    n = B * H * W * C
    _check(lib().pn_col2im_3x3s2(_f32(dcol, B * Ho * Wo * kp, "dcol"), B, H, W, C, kp,
                                 _bf(mask, n, "mask", allow_none=True), _bf(dx16, n, "dx16", allow_none=True),
                                 _f32(dx32, n, "dx32", allow_none=True), _stream(stream)))


def pn_transpose_bf16(src, rows, cols, dst, ld_dst=None, stream=None):
    ld_dst = rows if ld_dst is None else ld_dst
    _check(lib().pn_transpose_bf16(_bf(src, rows * cols, "src"), rows, cols, _bf(dst, cols * ld_dst, "dst"),
                                   int(ld_dst), _stream(stream)))


def pn_colsum_scratch_floats(M, N) -> int:
    return int(lib().pn_colsum_scratch_floats(int(M), int(N)))


def pn_colsum_bf16(y, M, N, ld, out, scratch, stream=None):
    if y.numel() < (M - 1) * ld + N or scratch.numel() < pn_colsum_scratch_floats(M, N):
        raise ValueError("y or scratch smaller than the stated shape")
    _check(lib().pn_colsum_bf16(_bf(y, name="y"), M, N, ld, _f32(out, N, "out"), _f32(scratch, name="scratch"),
                                _stream(stream)))


def pn_prepare_images(proj, n_img, n_views, nu, nv, factor, out, stream=None):
    _check(lib().pn_prepare_images(_f32(proj, n_img * n_views * nu * nv, "proj"), n_img, n_views, nu, nv, factor,
                                   _bf(out, n_img * n_views * (nu // factor) * (nv // factor), "out"),
                                   _stream(stream)))


def pn_mse_loss(y, B, n_out, ldy, target, loss=None, dy=None, lddy=None, stream=None):
    lddy = n_out if lddy is None else lddy
    _check(lib().pn_mse_loss(_f32(y, B * ldy, "y"), B, n_out, ldy, _f32(target, B * n_out, "target"),
                             _f32(loss, 1, "loss", allow_none=True), _bf(dy, B * lddy, "dy", allow_none=True),
                             int(lddy), _stream(stream)))


def pn_to_bf16(src, dst, stream=None):
    _check(lib().pn_to_bf16(_f32(src, name="src"), src.numel(), _bf(dst, src.numel(), "dst"), _stream(stream)))


def pn_gemm_test_hooks(wait_ns=0, stall_tma=False):
    """Failure-path test hook of the GEMM (see include/posenet.h)."""
    _check(lib().pn_gemm_test_hooks(int(wait_ns), 1 if stall_tma else 0))


def pn_status(stream=None) -> int:
    st = ctypes.c_int(0)
    _check(lib().pn_status(_stream(stream), ctypes.byref(st)))
    return int(st.value)


class Projector:
    """A plan plus its workspace (a zero-filled torch uint8 tensor on the
    current CUDA device); methods allocate their outputs with torch."""

    def __init__(self, geom, n_pose=1, inst_view=None, inst_pose=None, ops=PROJ_OP_ALL, device=None):
        import torch
        if inst_view is None:
            inst_view = np.arange(geom.views.shape[0])
        if inst_pose is None:
            inst_pose = np.zeros(len(inst_view), dtype=np.int32) if n_pose == 1 else np.arange(len(inst_view))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.plan = proj_plan_create(geom, n_pose, inst_view, inst_pose, ops)
            self.ws = torch.zeros(proj_workspace_size(self.plan), dtype=torch.uint8, device=self.device)
        self.geom = geom

    @property
    def n_inst(self):
        return self.plan.n_inst

    def _t(self, x, dtype=None):
        import torch
        return torch.as_tensor(x, dtype=dtype or torch.float32, device=self.device).contiguous()

    def set_volume(self, mu):
        proj_set_volume(self.plan, self._t(mu), self.ws)

    def forward(self, pose, out=None):
        import torch
        g = self.geom
        out = out if out is not None else torch.empty((self.n_inst, g.nv, g.nu), device=self.device)
        proj_forward(self.plan, self._t(pose), out, self.ws)
        return out

    def forward_pose_grad(self, pose, loss, ref, want_proj=False):
        import torch
        g = self.geom
        grad = torch.empty((self.plan.n_pose, 6), device=self.device)
        lossv = torch.empty((self.plan.n_pose,), device=self.device)
        proj = torch.empty((self.n_inst, g.nv, g.nu), device=self.device) if want_proj else None
        proj_forward_pose_grad(self.plan, self._t(pose), loss, self._t(ref), grad, lossv, proj, self.ws)
        return (grad, lossv, proj) if want_proj else (grad, lossv)

    def autotune(self, pose, loss, ref, reps=3):
        return proj_autotune_forward_grad(self.plan, self._t(pose), loss, self._t(ref), self.ws, reps)

    def autotune_back(self, proj, pose, vol_resid, weight=PROJ_W_NONE, reps=3):
        return proj_autotune_back_grad(self.plan, self._t(proj), self._t(pose), weight, self._t(vol_resid), self.ws,
                                       reps)

    def back(self, proj, pose, weight=PROJ_W_NONE):
        import torch
        g = self.geom
        vol = torch.empty((g.nz, g.ny, g.nx), device=self.device)
        proj_back(self.plan, self._t(proj), self._t(pose), weight, vol, self.ws)
        return vol

    def back_pose_grad(self, proj, pose, vol_resid, weight=PROJ_W_NONE):
        import torch
        grad = torch.empty((self.plan.n_pose, 6), device=self.device)
        proj_back_pose_grad(self.plan, self._t(proj), self._t(pose), weight, self._t(vol_resid), grad, self.ws)
        return grad

    def back_adjoint(self, vol, pose, weight=PROJ_W_NONE):
        import torch
        g = self.geom
        out = torch.empty((self.n_inst, g.nv, g.nu), device=self.device)
        proj_back_adjoint(self.plan, self._t(vol), self._t(pose), weight, out, self.ws)
        return out

    def forward_adjoint(self, y, pose):
        import torch
        g = self.geom
        vol = torch.empty((g.nz, g.ny, g.nx), device=self.device)
        proj_forward_adjoint(self.plan, self._t(y), self._t(pose), vol, self.ws)
        return vol

    def fdk_filter(self, proj, scale):
        import torch
        out = torch.empty((self.n_inst, self.geom.nv, self.geom.nu), device=self.device)
        proj_fdk_filter(self.plan, self._t(proj), scale, out)
        return out

    def sharpness(self, vol, want_grad=True):
        import torch
        loss = torch.empty((1,), device=self.device)
        grad = torch.empty((self.geom.nz, self.geom.ny, self.geom.nx), device=self.device) if want_grad else None
        proj_sharpness(self.plan, self._t(vol), loss, grad, self.ws)
        return (loss, grad) if want_grad else loss

    def count_samples(self, pose):
        import torch
        c = torch.empty((self.n_inst,), dtype=torch.int64, device=self.device)
        proj_count_samples(self.plan, self._t(pose), c, self.ws)
        return c

    def count_marched_samples(self, pose):
        import torch
        c = torch.empty((self.n_inst,), dtype=torch.int64, device=self.device)
        proj_count_marched_samples(self.plan, self._t(pose), c, self.ws)
        return c

    def check(self):
        return proj_check(self.plan, self.ws)

"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/*.h declares, and rejects invalid arguments on
the host (before any CUDA call) with the documented error codes."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2508_13304_b300 as pb
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def L():
    from paper_2508_13304_b300 import build
    build.build()
    return pb.lib()


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b((?:proj|pn)_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 30 and any(n.startswith("pn_") for n in names)
    out = subprocess.run(["nm", "-D", "--defined-only", pb.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT ((?:proj|pn)_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(L, n)


def test_binding_covers_the_abi():
    for n in declared_functions():
        assert hasattr(pb, n), n


def test_version_string(L):
    assert "sm_103a" in pb.proj_version()


def tiny_geom(**kw):
    g = synth.Geometry(8, 7, 6, 1.0, 1.0, 1.0, 10, 9, synth.circular_views(2, 100.0, 160.0, 1.0, 1.0), 0.5)
    for k, v in kw.items():
        setattr(g, k, v)
    return g


def create(geom, n_pose=1, inst_view=(0, 1), inst_pose=(0, 0), ops=pb.PROJ_OP_ALL):
    g, views = pb.make_geometry(geom)
    iv = np.ascontiguousarray(inst_view, dtype=np.int32)
    ip = np.ascontiguousarray(inst_pose, dtype=np.int32)
    h = ctypes.c_void_p()
    rc = pb.lib().proj_plan_create(ctypes.byref(g), n_pose, len(iv), iv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   ip.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ops, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("field,value,msg", [
    ("nx", 0, "volume size"), ("nu", 0, "detector size"), ("vx", 0.0, "voxel pitch"),
    ("vy", float("nan"), "voxel pitch"), ("step", -1.0, "ray step"), ("off", (0.0, float("inf"), 0.0), "offset"),
])
def test_bad_geometry_is_rejected_on_the_host(L, field, value, msg):
    rc, h = create(tiny_geom(**{field: value}))
    assert rc == pb.PROJ_E_ARG and not h.value
    assert msg in pb.proj_last_error()


def test_singular_detector_basis_is_rejected(L):
    g = tiny_geom()
    views = g.views.copy()
    views[0, 9:12] = views[0, 6:9]          # V parallel to U
    g.views = views
    rc, _ = create(g)
    assert rc == pb.PROJ_E_ARG and "singular" in pb.proj_last_error()


def test_non_finite_view_is_rejected(L):
    g = tiny_geom()
    views = g.views.copy()
    views[1, 2] = np.nan
    g.views = views
    rc, _ = create(g)
    assert rc == pb.PROJ_E_ARG and "non-finite" in pb.proj_last_error()


@pytest.mark.parametrize("iv,ip,n_pose,msg", [
    ((0, 2), (0, 0), 1, "view 2 out of range"), ((0, 1), (0, 1), 1, "pose 1 out of range"),
    ((0, -1), (0, 0), 1, "view -1"), ((0, 1), (0, 0), 0, "n_pose"),
])
def test_instance_indices_are_checked(L, iv, ip, n_pose, msg):
    rc, _ = create(tiny_geom(), n_pose=n_pose, inst_view=iv, inst_pose=ip)
    assert rc == pb.PROJ_E_ARG and msg in pb.proj_last_error()


def test_empty_instance_list_is_rejected(L):
    rc, h = create(tiny_geom(), inst_view=(), inst_pose=())
    assert rc == pb.PROJ_E_ARG and not h.value and "n_inst" in pb.proj_last_error()


@pytest.mark.parametrize("sizes,msg", [
    (dict(ny=65001), "<= 65000"), (dict(nz=65001), "<= 65000"), (dict(nv=65001), "<= 65000"),
    (dict(nx=2000, ny=2000, nz=600), "volume too large"),   # padded voxel count >= 2^31
])
def test_size_limits_are_enforced_on_the_host(L, sizes, msg):
    rc, h = create(tiny_geom(**sizes))
    assert rc == pb.PROJ_E_ARG and not h.value and msg in pb.proj_last_error()


def test_instance_limit_of_the_voxel_driven_calls(L):
    n = 65536
    iv, ip = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
    rc, _ = create(tiny_geom(), inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_BACK)
    assert rc == pb.PROJ_E_ARG and "65535" in pb.proj_last_error()
    rc, _ = create(tiny_geom(), inst_view=iv, inst_pose=ip, ops=pb.PROJ_OP_BACK_GRAD)
    assert rc == pb.PROJ_E_ARG and "65535" in pb.proj_last_error()


def test_bad_ops_and_null_arguments(L):
    rc, _ = create(tiny_geom(), ops=0)
    assert rc == pb.PROJ_E_ARG
    rc, _ = create(tiny_geom(), ops=128)
    assert rc == pb.PROJ_E_ARG
    rc, _ = create(tiny_geom(), ops=pb.PROJ_FLAG_ONE_COPY)       # an option flag alone enables no operation
    assert rc == pb.PROJ_E_ARG and "non-empty" in pb.proj_last_error()
    assert L.proj_forward_pose_grad_list(None, None, None, 1, 0, None, None, None, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_plan_create(None, 1, 1, None, None, 1, None) == pb.PROJ_E_ARG
    n = ctypes.c_size_t()
    assert L.proj_workspace_size(None, ctypes.byref(n)) == pb.PROJ_E_ARG
    assert L.proj_forward(None, None, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_forward_pose_grad(None, None, 0, None, None, None, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_back(None, None, None, 0, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_back_pose_grad(None, None, None, 0, None, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_back_adjoint(None, None, None, 0, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_forward_adjoint(None, None, None, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_set_volume(None, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_check(None, None, 0, None, None) == pb.PROJ_E_ARG
    assert L.proj_count_samples(None, None, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_fdk_filter(None, None, 1.0, None, None) == pb.PROJ_E_ARG
    assert L.proj_sharpness(None, None, None, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_enable_kernel_timing(None, 1) == pb.PROJ_E_ARG
    assert L.proj_kernel_time_ms(None, None) == pb.PROJ_E_ARG
    assert L.proj_plan_destroy(None) == pb.PROJ_OK
    out = ctypes.c_void_p()
    assert L.proj_batch_create(1, None, None, None, None, None, None, None, None, None) == pb.PROJ_E_ARG
    assert L.proj_batch_create(0, None, None, None, None, None, None, None, None, ctypes.byref(out)) == pb.PROJ_E_ARG
    assert out.value is None
    assert L.proj_batch_run(None, None) == pb.PROJ_E_ARG
    assert L.proj_batch_destroy(None) == pb.PROJ_OK
    assert L.proj_set_warp_shape(None, 4) == pb.PROJ_E_ARG
    assert L.proj_gather_probe(None, None, None, 0, None) == pb.PROJ_E_ARG
    assert L.proj_get_warp_shape(None, None) == pb.PROJ_E_ARG
    assert L.proj_autotune_forward_grad(None, None, 0, None, None, 0, None, 1, None, None) == pb.PROJ_E_ARG
    assert L.proj_set_brick_shape(None, 0) == pb.PROJ_E_ARG
    assert L.proj_get_brick_shape(None, None) == pb.PROJ_E_ARG
    assert L.proj_autotune_back_grad(None, None, None, 0, None, None, 0, None, 1, None, None) == pb.PROJ_E_ARG
    assert L.proj_set_skip_brick(None, 8) == pb.PROJ_E_ARG
    assert L.proj_get_skip_brick(None, None) == pb.PROJ_E_ARG
    assert L.proj_set_skip_cells(None, 1) == pb.PROJ_E_ARG
    assert L.proj_get_skip_cells(None, None) == pb.PROJ_E_ARG
    assert L.proj_autotune_march(None, None, 0, None, None, 0, None, 1, None, None, None, None) == pb.PROJ_E_ARG
    assert L.proj_count_marched_samples(None, None, None, None, 0, None) == pb.PROJ_E_ARG
    # the option flags alone, or together, enable no operation
    rc, _ = create(tiny_geom(), ops=pb.PROJ_FLAG_BRICKS | pb.PROJ_FLAG_ONE_COPY)
    assert rc == pb.PROJ_E_ARG and "non-empty" in pb.proj_last_error()
    rc, _ = create(tiny_geom(), ops=pb.PROJ_OP_FORWARD_GRAD | 1024)            # an unknown flag bit
    assert rc == pb.PROJ_E_ARG


def test_valid_plan_without_a_gpu_reports_a_cuda_error(L):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    rc, h = create(tiny_geom())
    assert rc == pb.PROJ_E_CUDA and not h.value
    assert pb.proj_last_error()


def test_binding_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        pb._ptr(torch.zeros(3), name="x")


def test_c_program_uses_the_abi_without_python(tmp_path, L):
    """The headers compile as C, a C program links libproj.so and gets the
    documented host-side errors (gcc; no GPU, no Python binding)."""
    import shutil
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "abi_host")
    libdir = os.path.dirname(pb.LIB_PATH)
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_host.c"), "-L", libdir, "-lproj",
                    "-Wl,-rpath," + libdir, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr


def test_pose_adam_checks_its_arguments_on_the_host():
    lr = (ctypes.c_float * 6)(*([1.0] * 6))
    f = pb.lib().proj_pose_adam
    assert f(None, None, None, None, None, None, 0, lr, 0.9, 0.999, 1e-8, None) == pb.PROJ_OK   # nothing to do
    assert f(None, None, None, None, None, None, 1, lr, 0.9, 0.999, 1e-8, None) == pb.PROJ_E_ARG
    assert "NULL" in pb.proj_last_error()
    assert f(None, None, None, None, None, None, -1, lr, 0.9, 0.999, 1e-8, None) == pb.PROJ_E_ARG


def test_registration_step_checks_its_arguments_on_the_host():
    f = pb.lib().proj_registration_step
    prm = pb.reg_params([1.0] * 6)
    nul = [None] * 12
    assert f(0, 0, *nul, 0, None, None, ctypes.byref(prm), None) == pb.PROJ_OK        # nothing to do
    assert f(2, 2, *nul, 0, None, None, ctypes.byref(prm), None) == pb.PROJ_E_ARG
    assert "NULL" in pb.proj_last_error()
    assert f(-1, 2, *nul, 0, None, None, ctypes.byref(prm), None) == pb.PROJ_E_ARG

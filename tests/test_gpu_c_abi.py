"""The C ABI used from C alone on the GPU: tests/c/abi_gpu.c (gcc, the CUDA
runtime and libproj.so; no Python binding, no torch) runs a plan, the
caller-owned workspace, a volume, proj_forward and proj_forward_pose_grad,
and checks the fused L2 loss against the host sum of squares of
proj_forward's output and two gradient components against central
differences of that loss."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def test_c_program_runs_the_gpu_path(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    from paper_2508_13304_b300 import build
    build.build()
    import paper_2508_13304_b300 as pb
    libdir = os.path.dirname(pb.LIB_PATH)
    exe = str(tmp_path / "abi_gpu")
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c", "abi_gpu.c"),
                    "-L", libdir, "-lproj", "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm",
                    "-Wl,-rpath," + libdir + ":" + os.path.join(CUDA, "lib64"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("abi_gpu ok"), out.stdout + out.stderr

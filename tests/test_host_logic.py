"""Host-side logic of the library, tested without a GPU (compiled with g++
from the library's own headers): the range allocator the server admits
requests with, the image geometry the kernels are launched with, and the
batch plan (linked from the built library; planning touches no device)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_range_allocator(tmp_path):
    exe = tmp_path / "range_alloc"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I",
                           os.path.join(ROOT, "paper_1401_5245_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "test_range_alloc.cpp"),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"


def test_image_geometry(tmp_path):
    exe = tmp_path / "geometry"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.check_call(["g++", "-O2", "-std=c++17",
                           "-I", os.path.join(ROOT, "paper_1401_5245_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                           os.path.join(ROOT, "tests", "host", "test_geometry.cpp"),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"


def test_batch_plan(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    pkg = os.path.join(ROOT, "paper_1401_5245_gb300")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = tmp_path / "plan"
    subprocess.check_call(["g++", "-O2", "-std=c++17",
                           "-I", os.path.join(pkg, "csrc"), "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(cuda, "include"),
                           os.path.join(ROOT, "tests", "host", "test_plan.cpp"),
                           "-L", pkg, "-lme", "-Wl,-rpath," + pkg,
                           "-L", os.path.join(cuda, "lib64"), "-lcudart",
                           "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"

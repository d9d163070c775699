"""Host-side logic of the library, tested without a GPU: the range
allocator the server admits requests with (compiled with g++ from the
library's own header)."""
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

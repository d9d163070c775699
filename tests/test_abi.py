"""The C-ABI library builds, loads and exports every symbol include/me.h
declares; argument checks that need no GPU return the documented codes."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "me.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(me_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1401_5245_gb300 import _lib
    return _lib


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for n in ("me_edges", "me_edges_batch", "me_serve_open", "me_serve_submit",
              "me_serve_poll", "me_serve_close", "me_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(me_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # the binding knows every call, and nothing the header does not declare
    assert sorted(lib.PROTOTYPES) == declared_functions()


def test_header_is_c_and_every_entry_point_links_from_c(lib, tmp_path):
    """A C11 program (strict, warnings as errors) that includes the header
    and takes the address of every declared function links against the
    library."""
    names = declared_functions()
    src = tmp_path / "uses_every_entry_point.c"
    src.write_text("#include \"me.h\"\n#include <stdio.h>\n"
                   "int main(void) {\n"
                   "    void (*fns[])(void) = {\n" +
                   "".join(f"        (void (*)(void)){n},\n" for n in names) +
                   "    };\n"
                   "    printf(\"%d\\n\", (int)(sizeof fns / sizeof fns[0]));\n"
                   "    return 0;\n}\n")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    pkg = os.path.dirname(lib.LIB_PATH)
    exe = tmp_path / "uses_every_entry_point"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-Wno-cast-function-type",
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                           str(src), "-L", pkg, "-lme", "-Wl,-rpath," + pkg, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    assert int(out.stdout) == len(names)


def test_library_links_shared_cuda_runtime(lib):
    out = subprocess.run(["readelf", "-d", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    assert "libcudart.so" in out


def test_status_strings(lib):
    L = lib.load()
    for name, code in lib.C.items():
        if name.startswith("ME_ERR_") or name in ("ME_OK", "ME_PENDING", "ME_TIMEOUT"):
            assert lib.status_string(code) == name
    assert lib.status_string(12345) == "ME_UNKNOWN_STATUS"
    assert L.me_version() >= 10000


def test_argument_errors_without_a_gpu(lib):
    L = lib.load()
    ARG, ALIAS = lib.C["ME_ERR_ARG"], lib.C["ME_ERR_ALIAS"]
    a, b = 0x10000, 0x200000
    assert L.me_edges(None, 8, 8, 1, b, 0, None) == ARG
    assert L.me_edges(a, 8, 8, 1, None, 0, None) == ARG
    assert L.me_edges(a, 0, 8, 1, b, 0, None) == ARG
    assert L.me_edges(a, 8, -1, 1, b, 0, None) == ARG
    assert L.me_edges(a, 33, 8, 1, b, 0, None) == ARG          # stride < ceil(w/32)
    assert L.me_edges(a, 8, 8, 1, b, 2, None) == ARG           # boundary
    assert L.me_edges(a + 2, 8, 8, 1, b, 0, None) == ARG       # not word aligned
    assert L.me_edges(a, 64, 100, 2, a + 400, 0, None) == ALIAS
    assert L.me_edges_staged(a, 64, 100, 2, a + 8, 0, None) == ALIAS
    assert L.me_fundamental_edges(a, 8, 8, 1, b, b, b + 64, b + 128, 0, None) == ALIAS
    assert L.me_edges_inplace(None, 8, 8, 1, 0, None) == ARG
    assert L.me_edges_inplace(a, 0, 8, 1, 0, None) == ARG             # w
    assert L.me_edges_inplace(a, 64, 8, 1, 0, None) == ARG            # stride
    assert L.me_edges_inplace(a, 8, 8, 1, 3, None) == ARG             # boundary
    assert L.me_edges_inplace(a + 2, 8, 8, 1, 0, None) == ARG         # not word aligned
    assert L.me_edges_batch(None, -1, None) == ARG
    assert L.me_edges_batch(None, 0, None) == lib.C["ME_OK"]
    bad = lib.make_descs([(a, a, 8, 8, 1, 0)])
    assert L.me_edges_batch(bad, 1, None) == ALIAS
    cfg = lib.me_tile_cfg(0, 3, 4, 256, 0, 32, 4)
    assert L.me_set_tile_cfg(0, ctypes.byref(cfg)) == ARG      # rows_per_lane 3
    cfg = lib.me_tile_cfg(1, 8, 4, 256, 0, 64, 4)
    assert L.me_set_tile_cfg(0, ctypes.byref(cfg)) == ARG      # 256 KiB of stages
    cfg = lib.me_tile_cfg(1, 8, 4, 256, 0, 32, 1)
    assert L.me_set_tile_cfg(1, ctypes.byref(cfg)) == ARG      # one stage
    assert L.me_set_tile_cfg(7, ctypes.byref(cfg)) == ARG
    for chunk in (-1, 65):                                      # tiles per chunk
        cfg = lib.me_tile_cfg(0, 4, 4, 256, 8, 32, 4, chunk)
        assert L.me_set_tile_cfg(1, ctypes.byref(cfg)) == ARG
    g = 0x300000                                                # a made-up grey image
    assert L.me_threshold_edges(None, 64, 4, 64, 128, b, 2, None, 0, None) == ARG
    assert L.me_threshold_edges(g, 64, 4, 63, 128, b, 2, None, 0, None) == ARG   # pitch < w
    assert L.me_threshold_edges(g, 64, 4, 64, 128, b, 1, None, 0, None) == ARG   # stride
    assert L.me_threshold_edges(g, 64, 4, 64, 128, b, 2, None, 2, None) == ARG   # boundary
    assert L.me_threshold_edges(g, 64, 4, 64, 128, b + 2, 2, None, 0, None) == ARG
    assert L.me_threshold_edges(g, 64, 4, 64, 128, g + 64, 2, None, 0, None) == ALIAS
    assert L.me_threshold_edges(g, 64, 4, 64, 128, b, 2, b + 4, 0, None) == ALIAS
    assert L.me_threshold_edges_otsu(None, 64, 4, 64, b, 2, None, 0, None, None) == ARG
    assert L.me_threshold_edges_otsu(g, 0, 4, 64, b, 2, None, 0, None, None) == ARG
    assert L.me_threshold_edges_otsu(g, 64, 4, 64, g + 8, 2, None, 0, None, None) == ALIAS
    assert L.me_serve_open(None, None) == ARG
    assert L.me_serve_poll(None, 1, None, 0, None) == ARG
    assert L.me_serve_close(None, 0) == ARG


def test_tile_cfg_roundtrip(lib):
    L = lib.load()
    old = lib.me_tile_cfg()
    assert L.me_get_tile_cfg(1, ctypes.byref(old)) == 0
    new = lib.me_tile_cfg(1, 16, 4, 512, 2, 48, 3, 7)
    assert L.me_set_tile_cfg(1, ctypes.byref(new)) == 0
    assert lib.me_get_tile_cfg(1).as_dict() == new.as_dict()
    assert L.me_set_tile_cfg(1, ctypes.byref(old)) == 0
    # the batch kind with narrower accesses keeps a configuration of its own
    old_any = lib.me_get_tile_cfg(lib.ME_KIND_BATCH_ANY)
    other = lib.me_tile_cfg(0, 8, 4, 256, 0, 32, 4, 3)
    assert L.me_set_tile_cfg(lib.ME_KIND_BATCH_ANY, ctypes.byref(other)) == 0
    assert lib.me_get_tile_cfg(lib.ME_KIND_BATCH_ANY).as_dict() == other.as_dict()
    assert lib.me_get_tile_cfg(1).as_dict() == old.as_dict()
    assert L.me_set_tile_cfg(lib.ME_KIND_BATCH_ANY, ctypes.byref(old_any)) == 0
    assert L.me_set_tile_cfg(3, ctypes.byref(old)) == lib.C["ME_ERR_ARG"]
    assert L.me_get_tile_cfg(3, ctypes.byref(old)) == lib.C["ME_ERR_ARG"]

"""The tile autotuner: it picks a valid configuration, leaves exact results
behind, writes its choice to the ME_TUNE_CACHE file, and a fresh process
reads that choice back."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_1401_5245_gb300 import _lib, synth as S
from tests.gpu_util import DevBuf, SENTINEL, check_output_layout

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.init()
    _lib.load()


def test_autotune_batch_writes_and_reads_cache(tmp_path, monkeypatch):
    import torch
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("ME_TUNE_CACHE", str(cache))
    saved = _lib.me_get_tile_cfg(1)
    items, keep = [], []
    for i, (w, h) in enumerate(S.batch_shapes(5, 40, 16, 600)):
        img = S.strokes(w, h, 5, i)
        words = S.pack(img, S.batch_stride(w), pad="random", seed=i)
        src, dst = DevBuf(words), DevBuf(np.zeros_like(words), fill=SENTINEL)
        keep.append((img, src, dst))
        items.append((src.ptr(), dst.ptr(), w, h, words.shape[1], 0))
    try:
        best = _lib.me_autotune(1, _lib.make_descs(items), len(items), reps=2)
        got = best.as_dict()
        assert got == _lib.me_get_tile_cfg(1).as_dict()
        assert got["engine"] in (0, 1) and got["cta_threads"] in (128, 256, 512)
        torch.cuda.synchronize()
        for img, src, dst in keep:
            ow = dst.words()
            check_output_layout(ow, img.shape[1])
            assert np.array_equal(S.unpack(ow, img.shape[1]), O.edges(img, 0))
        text = cache.read_text()
        assert "|1|" in text and len(text.strip().splitlines()) == 1
        # a fresh process picks the cached choice up
        code = ("import sys; sys.path.insert(0, %r); import torch; torch.cuda.init();"
                "from paper_1401_5245_gb300 import _lib; print(_lib.me_get_tile_cfg(1).as_dict())"
                % ROOT)
        env = dict(os.environ, ME_TUNE_CACHE=str(cache))
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           env=env, timeout=300)
        assert r.returncode == 0, r.stderr
        assert eval(r.stdout.strip().splitlines()[-1]) == got
    finally:
        _lib.load().me_set_tile_cfg(1, saved)


def test_autotune_rejects_bad_arguments():
    L = _lib.load()
    best = _lib.me_tile_cfg()
    import ctypes
    assert L.me_autotune(5, None, 0, 1, None, ctypes.byref(best)) == _lib.C["ME_ERR_ARG"]
    assert L.me_autotune(0, None, 1, 1, None, ctypes.byref(best)) == _lib.C["ME_ERR_ARG"]


def narrow_sample(seed, n=40):
    """Images with stride = ceil(w / 32), unpadded: some strides are not whole
    16-byte groups, so the batch is of the kind ME_KIND_BATCH_ANY."""
    items, keep = [], []
    for i, (w, h) in enumerate(S.batch_shapes(seed, n, 16, 600)):
        img = S.strokes(w, h, 5, i)
        words = S.pack(img, S.batch_stride(w, False), pad="random", seed=i)
        src, dst = DevBuf(words), DevBuf(np.zeros_like(words), fill=SENTINEL)
        keep.append((img, src, dst))
        items.append((src.ptr(), dst.ptr(), w, h, words.shape[1], 0))
    assert any(it[4] % 4 for it in items)
    return items, keep


def test_autotune_of_the_narrow_batch_kind():
    """Tuning ME_KIND_BATCH_ANY on a batch with narrower accesses sets that
    kind's configuration only, and the batch's edge maps stay exact."""
    import torch
    saved = (_lib.me_get_tile_cfg(_lib.ME_KIND_BATCH), _lib.me_get_tile_cfg(_lib.ME_KIND_BATCH_ANY))
    items, keep = narrow_sample(6)
    try:
        best = _lib.me_autotune(_lib.ME_KIND_BATCH_ANY, _lib.make_descs(items), len(items), reps=2)
        assert best.as_dict() == _lib.me_get_tile_cfg(_lib.ME_KIND_BATCH_ANY).as_dict()
        assert _lib.me_get_tile_cfg(_lib.ME_KIND_BATCH).as_dict() == saved[0].as_dict()
        for img, src, dst in keep:
            dst.t.fill_(int(np.uint32(SENTINEL).view(np.int32)))
        assert _lib.me_edges_batch(_lib.make_descs(items), len(items)) == 0
        torch.cuda.synchronize()
        for img, src, dst in keep:
            ow = dst.words()
            check_output_layout(ow, img.shape[1])
            assert np.array_equal(S.unpack(ow, img.shape[1]), O.edges(img, 0))
    finally:
        L = _lib.load()
        L.me_set_tile_cfg(_lib.ME_KIND_BATCH, saved[0])
        L.me_set_tile_cfg(_lib.ME_KIND_BATCH_ANY, saved[1])


def test_autotune_refuses_a_sample_of_the_other_batch_kind():
    """A sample's launches use its own kind's configuration, so tuning the
    other kind on it would time identical launches: refused."""
    import ctypes
    L = _lib.load()
    best = _lib.me_tile_cfg()
    narrow, keep = narrow_sample(7, 8)
    wide = []
    for i, (w, h) in enumerate(S.batch_shapes(8, 8, 16, 300)):
        words = S.pack(S.strokes(w, h, 3, i), S.batch_stride(w), pad="random", seed=i)
        src, dst = DevBuf(words), DevBuf(np.zeros_like(words))
        keep.append((None, src, dst))
        wide.append((src.ptr(), dst.ptr(), w, h, words.shape[1], 0))
    assert L.me_autotune(_lib.ME_KIND_BATCH, _lib.make_descs(narrow), len(narrow), 1, None,
                         ctypes.byref(best)) == _lib.C["ME_ERR_ARG"]
    assert L.me_autotune(_lib.ME_KIND_BATCH_ANY, _lib.make_descs(wide), len(wide), 1, None,
                         ctypes.byref(best)) == _lib.C["ME_ERR_ARG"]

"""me_edges_staged_static, the staged form that allocates nothing.

Some callers cannot allocate device memory once they are running: a
framework's caching allocator may own the whole device, a real-time loop
must not wait on an allocator, or device memory may be capped after
start-up.  For them the mask image of the staged form lives in a fixed
device array built into the library.  These tests call it through the C
ABI and check it against the allocating entry point (me_edges_staged) bit
for bit, over two calls in a row that share the array.
"""
import numpy as np
import pytest

from paper_1401_5245_gb300 import _lib, synth as S
from tests.gpu_util import DevBuf, SENTINEL, check_output_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.init()
    _lib.load()


def sync():
    import torch
    torch.cuda.synchronize()


def prepare(img, stride, seed):
    h, w = img.shape
    words = S.pack(img, stride, pad="random", seed=seed)
    src = DevBuf(words)
    out_static = DevBuf(np.zeros_like(words), fill=SENTINEL)
    out_ref = DevBuf(np.zeros_like(words), fill=SENTINEL)
    return (w, h, stride, src, out_static, out_ref)


def test_matches_the_allocating_entry_point_on_two_calls_in_a_row():
    L = _lib.load()
    g = np.random.default_rng(7)
    # the first call fills most of the array; the second is smaller and
    # different, so anything left from the first call would show
    first = prepare((g.random((3000, 4000)) < 0.5).astype(np.uint8), 128, 1)
    second = prepare(S.strokes(1000, 777, 40, 3), 33, 2)
    for boundary in (0, 1):
        for (w, h, stride, src, out_s, out_r) in (first, second):
            assert L.me_edges_staged_static(src.ptr(), w, h, stride, out_s.ptr(),
                                            boundary, None) == 0
        for (w, h, stride, src, out_s, out_r) in (first, second):
            assert L.me_edges_staged(src.ptr(), w, h, stride, out_r.ptr(), boundary,
                                     None) == 0
        sync()
        for (w, h, stride, src, out_s, out_r) in (first, second):
            a, b = out_s.words(), out_r.words()
            assert out_s.guards_intact()
            check_output_layout(a, w)
            assert np.array_equal(a, b), (w, h, boundary)


def test_largest_image_it_holds_and_the_next_size_up():
    L = _lib.load()
    limit = _lib.C["ME_STATIC_MASK_WORDS"]
    w, stride = 4096, 128
    h = limit // stride
    img = (np.random.default_rng(3).random((h, w)) < 0.4).astype(np.uint8)
    w_, h_, stride_, src, out_s, out_r = prepare(img, stride, 4)
    assert L.me_edges_staged_static(src.ptr(), w, h, stride, out_s.ptr(), 0, None) == 0
    assert L.me_edges_staged(src.ptr(), w, h, stride, out_r.ptr(), 0, None) == 0
    sync()
    assert np.array_equal(out_s.words(), out_r.words())
    # one row more no longer fits: a clear error and nothing written
    big = DevBuf(np.zeros((h + 1, stride), dtype=np.uint32))
    out = DevBuf(np.zeros((h + 1, stride), dtype=np.uint32), fill=SENTINEL)
    rc = L.me_edges_staged_static(big.ptr(), w, h + 1, stride, out.ptr(), 0, None)
    assert rc == _lib.C["ME_ERR_TOO_BIG"]
    assert _lib.status_string(rc) == "ME_ERR_TOO_BIG"
    sync()
    assert (out.words() == SENTINEL).all()

"""me_edges_staged_static, the staged form that allocates nothing.

Some callers cannot allocate device memory once they are running: a
framework's caching allocator may own the whole device, a real-time loop
must not wait on an allocator, or device memory may be capped after
start-up.  For them the mask image of the staged form lives in a fixed
device array built into the library.  These tests call it through the C
ABI and check it bit for bit against the allocating entry point
(me_edges_staged) and against the CPU oracle, over two calls in a row that
share the array.
"""
import numpy as np
import pytest

from oracle import oracle as O
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
    return (img, w, h, stride, src, out_static, out_ref)


def test_matches_the_allocating_entry_point_and_the_oracle_on_two_calls_in_a_row():
    L = _lib.load()
    limit = _lib.C["ME_STATIC_MASK_WORDS"]
    g = np.random.default_rng(7)
    # the first call fills the whole array (h * stride == the limit); the
    # second is smaller and different, so anything left from the first call
    # would show in it
    stride = 128
    first = prepare((g.random((limit // stride, 4000)) < 0.5).astype(np.uint8), stride, 1)
    second = prepare(S.strokes(1000, 777, 40, 3), 33, 2)
    assert first[2] * first[3] == limit
    for boundary in (0, 1):
        for (img, w, h, stride, src, out_s, out_r) in (first, second):
            assert L.me_edges_staged_static(src.ptr(), w, h, stride, out_s.ptr(),
                                            boundary, None) == 0
        for (img, w, h, stride, src, out_s, out_r) in (first, second):
            assert L.me_edges_staged(src.ptr(), w, h, stride, out_r.ptr(), boundary,
                                     None) == 0
        sync()
        for (img, w, h, stride, src, out_s, out_r) in (first, second):
            a, b = out_s.words(), out_r.words()
            assert out_s.guards_intact()
            check_output_layout(a, w)
            assert np.array_equal(a, b), (w, h, boundary)
            assert np.array_equal(S.unpack(a, w), O.edges(img, boundary)), (w, h, boundary)


def test_largest_image_it_holds_and_the_next_size_up():
    L = _lib.load()
    limit = _lib.C["ME_STATIC_MASK_WORDS"]
    w, stride = 4096, 128
    h = limit // stride
    img = (np.random.default_rng(3).random((h, w)) < 0.4).astype(np.uint8)
    _, w_, h_, stride_, src, out_s, out_r = prepare(img, stride, 4)
    assert L.me_edges_staged_static(src.ptr(), w, h, stride, out_s.ptr(), 0, None) == 0
    assert L.me_edges_staged(src.ptr(), w, h, stride, out_r.ptr(), 0, None) == 0
    sync()
    assert np.array_equal(out_s.words(), out_r.words())
    assert np.array_equal(S.unpack(out_s.words(), w), O.edges(img, 0))
    # one row more no longer fits: a clear error and nothing written
    big = DevBuf(np.zeros((h + 1, stride), dtype=np.uint32))
    out = DevBuf(np.zeros((h + 1, stride), dtype=np.uint32), fill=SENTINEL)
    rc = L.me_edges_staged_static(big.ptr(), w, h + 1, stride, out.ptr(), 0, None)
    assert rc == _lib.C["ME_ERR_TOO_BIG"]
    assert _lib.status_string(rc) == "ME_ERR_TOO_BIG"
    sync()
    assert (out.words() == SENTINEL).all()


def test_after_shutdown_the_address_is_looked_up_again():
    """me_shutdown() forgets the cached device address of the array (the
    recovery step after a device reset); the next call looks it up again
    and still matches the oracle."""
    L = _lib.load()
    img = S.strokes(300, 200, 12, 5)
    im, w, h, stride, src, out_s, _ = prepare(img, 10, 6)
    assert L.me_edges_staged_static(src.ptr(), w, h, stride, out_s.ptr(), 0, None) == 0
    sync()
    assert L.me_shutdown() == 0
    out2 = DevBuf(np.zeros((h, stride), dtype=np.uint32), fill=SENTINEL)
    assert L.me_edges_staged_static(src.ptr(), w, h, stride, out2.ptr(), 0, None) == 0
    sync()
    assert np.array_equal(out2.words(), out_s.words())
    assert np.array_equal(S.unpack(out2.words(), w), O.edges(im, 0))

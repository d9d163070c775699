"""Bit-exact parity of me_edges_inplace (the edge map written over the image)
with the CPU oracle: many widths, heights that cross several band seams,
both boundary colours, aligned and unaligned layouts, the two-columns-per-
thread path for very wide rows, and agreement with me_edges."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1401_5245_gb300 import _lib, synth as S
from tests.gpu_util import DevBuf, check_output_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.init()
    _lib.load()


@pytest.fixture(autouse=True, params=["bands", "copy"])
def route(request, monkeypatch):
    """Every case both ways: bands of rows walked in place (copy limit 0)
    and the whole-image copy (limit above every test image)."""
    monkeypatch.setenv("ME_INPLACE_COPY_MAX", "0" if request.param == "bands" else str(1 << 40))
    return request.param


def sync():
    import torch
    torch.cuda.synchronize()


def run_inplace(img, b, stride, off=0, pad="random", seed=0):
    h, w = img.shape
    words = S.pack(img, stride, pad=pad, seed=seed)
    buf = DevBuf(words, off)
    rc = _lib.me_edges_inplace(buf.ptr(), w, h, stride, b)
    assert rc == 0, _lib.status_string(rc)
    sync()
    assert buf.guards_intact()
    out = buf.words()
    check_output_layout(out, w)
    return S.unpack(out, w)


@pytest.mark.parametrize("w", [1, 2, 31, 32, 33, 63, 64, 65, 97, 127, 128, 129, 1000,
                               4095, 4096, 4097])
@pytest.mark.parametrize("b", [0, 1])
def test_widths_across_band_seams(w, b):
    """1000 rows: bands of 32 rows, 31 seams."""
    img = S.strokes(w, 1000, max(1, w // 40), w + 7 * b)
    if w % 3 == 0:
        img = (np.random.default_rng(w).random((1000, w)) < 0.5).astype(np.uint8)
    assert np.array_equal(run_inplace(img, b, S.batch_stride(w)), O.edges(img, b))


@pytest.mark.parametrize("h", [1, 2, 3, 31, 32, 33, 64, 65, 97])
def test_heights_near_band_sizes(h):
    img = (np.random.default_rng(h).random((h, 300)) < 0.4).astype(np.uint8)
    assert np.array_equal(run_inplace(img, 0, S.batch_stride(300)), O.edges(img, 0))


@pytest.mark.parametrize("stride_extra,off", [(0, 1), (1, 0), (3, 2), (5, 3)])
def test_unaligned_rows_and_buffers(stride_extra, off):
    """Strides that are not a multiple of 4 words and starts off 16 bytes:
    the 32-bit path, with its per-word stores stopping at the stride."""
    w = 777
    img = S.strokes(w, 400, 30, stride_extra * 10 + off)
    stride = (w + 31) // 32 + stride_extra
    assert np.array_equal(run_inplace(img, 1, stride, off=off), O.edges(img, 1))


def test_two_columns_per_thread():
    """Rows of 140000 pixels: 1094 groups of 4 words, more than one CTA's
    threads, so every thread takes two columns."""
    w, h = 140000, 70
    img = (np.random.default_rng(3).random((h, w)) < 0.3).astype(np.uint8)
    assert np.array_equal(run_inplace(img, 0, S.batch_stride(w)), O.edges(img, 0))


def test_large_image_against_the_oracle():
    """16384 x 8192 (512 MiB of bands and seams on the band route): the
    result over the image equals the oracle's edge map and me_edges."""
    import torch
    w, h = 16384, 8192
    words = S.bernoulli_half_packed(w, h, seed=4)
    want = O.edges(S.unpack(words, w), 0)
    x = torch.from_numpy(words.view(np.int32)).cuda()
    ref = torch.empty_like(x)
    assert _lib.me_edges(x, w, h, 512, ref, 0) == 0
    assert _lib.me_edges_inplace(x, w, h, 512, 0) == 0
    sync()
    got = x.cpu().numpy().view(np.uint32)
    assert np.array_equal(S.unpack(got, w), want)
    assert torch.equal(x, ref)


def test_rows_too_wide_and_bad_arguments(route):
    """Bands take rows of at most 2048 groups of 4 words; the whole-image
    copy has no such limit."""
    import torch
    L = _lib.load()
    x = torch.zeros(8200, dtype=torch.int32, device="cuda")
    want = _lib.C["ME_ERR_TOO_BIG"] if route == "bands" else 0
    assert L.me_edges_inplace(x.data_ptr(), 262145, 1, 8193, 0, None) == want
    assert L.me_edges_inplace(x.data_ptr(), 262144, 1, 8192, 0, None) == 0
    host = np.zeros(64, dtype=np.uint32)
    assert L.me_edges_inplace(host.ctypes.data, 32, 2, 1, 0, None) == _lib.C["ME_ERR_ARG"]

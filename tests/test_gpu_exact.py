"""Bit-exact parity of the CUDA single-image paths with the CPU oracle.

Covers the fused kernel (128-bit and 32-bit paths, every tile
configuration), the staged five-pass form, the fundamental edges, the drawn
polarity and the end-point map, on every width 1..97 and 4095..4097,
strides wider than the row, garbage in padding bits and words, misaligned
buffers, both boundary colours, the 256x256 glyph images, the 4096x4096
images of several densities and the 32768x32768 image in the launch
configuration the benchmark times.  Outputs are checked for zeroed
padding bits and words and intact guard canaries around every buffer.
"""
import itertools

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
    yield
    torch.cuda.synchronize()


def sync():
    import torch
    torch.cuda.synchronize()


def run_single(fn, img, stride=None, boundary=0, pad="random", off=0, seed=0, n_out=1):
    """Run one single-image call; returns the unpacked output(s)."""
    h, w = img.shape
    stride = S.words_per_row(w) if stride is None else stride
    words = S.pack(img, stride, pad=pad, seed=seed)
    src = DevBuf(words, off)
    outs = [DevBuf(np.zeros_like(words), off, fill=SENTINEL) for _ in range(n_out)]
    rc = fn(src.ptr(), w, h, stride, *[o.ptr() for o in outs], boundary, None)
    assert rc == 0, _lib.status_string(rc)
    sync()
    assert np.array_equal(src.words(), words), "input modified"
    res = []
    for o in outs:
        assert o.guards_intact(), "write outside the output buffer"
        ow = o.words()
        check_output_layout(ow, w)
        res.append(S.unpack(ow, w))
    return res if n_out > 1 else res[0]


def edges_fused(*a):
    return _lib.load().me_edges(*a)


def edges_staged(*a):
    return _lib.load().me_edges_staged(*a)


PATHS = {"fused": edges_fused, "staged": edges_staged}


def rand_img(seed, h, w, p_black=0.5):
    g = np.random.default_rng(seed)
    return (g.random((h, w)) >= p_black).astype(np.uint8)


# ---------------------------------------------------------------- configs
@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("boundary", [0, 1])
def test_glyph_256(path, seed, boundary):
    img = S.ellipse_glyphs(seed)
    assert np.array_equal(run_single(PATHS[path], img, boundary=boundary),
                          O.edges(img, boundary))


@pytest.mark.parametrize("path", sorted(PATHS))
def test_every_width_1_to_97(path):
    for w in range(1, 98):
        for h in (1, 2, 7, 33):
            img = rand_img(w * 100 + h, h, w, p_black=0.6)
            for boundary in (0, 1):
                got = run_single(PATHS[path], img, boundary=boundary, seed=w)
                assert np.array_equal(got, O.edges(img, boundary)), (w, h, boundary)


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("w", [4095, 4096, 4097])
def test_wide_rows(path, w):
    img = rand_img(w, 9, w, p_black=0.7)
    for boundary in (0, 1):
        assert np.array_equal(run_single(PATHS[path], img, boundary=boundary),
                              O.edges(img, boundary))


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("extra,off", [(1, 0), (3, 0), (4, 0), (0, 1), (4, 1), (5, 3)])
def test_strides_and_alignment(path, extra, off):
    """Padding words, strides that break 16-byte row alignment, and buffers
    that start off a 16-byte boundary (the 32-bit path)."""
    for w, h in [(70, 40), (129, 65), (1000, 17), (31, 300)]:
        img = rand_img(w + h, h, w, 0.5)
        stride = S.words_per_row(w) + extra
        for boundary in (0, 1):
            got = run_single(PATHS[path], img, stride=stride, boundary=boundary, off=off)
            assert np.array_equal(got, O.edges(img, boundary)), (w, h, extra, off)


@pytest.mark.parametrize("pad", [0, 1, "random"])
def test_padding_garbage_is_ignored(pad):
    img = rand_img(5, 50, 77, 0.5)
    ref = O.edges(img, 0)
    for stride in (3, 4, 7):
        assert np.array_equal(run_single(edges_fused, img, stride, 0, pad=pad), ref)


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("p_black", [0.1, 0.5, 0.9])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_4096_bernoulli(path, p_black, seed):
    img = S.bernoulli(4096, 4096, p_black, seed)
    assert np.array_equal(run_single(PATHS[path], img), O.edges(img, 0))


@pytest.mark.parametrize("path", sorted(PATHS))
def test_4096_strokes(path):
    img = S.strokes(4096, 4096, 200, 0)
    assert np.array_equal(run_single(PATHS[path], img), O.edges(img, 0))


@pytest.mark.parametrize("kind", ["bernoulli", "blocks"])
def test_32768_full_image(kind):
    """The 1-Gpixel image in the benchmark's launch configuration (the
    single-image tile configuration in force), compared in full."""
    import torch
    w = h = 32768
    words = (S.bernoulli_half_packed(w, h, seed=0) if kind == "bernoulli"
             else S.blocks_packed(w, h, seed=0))
    img = S.unpack(words, w)
    want = O.edges(img, 0)
    del img
    x = torch.from_numpy(words.view(np.int32)).cuda()
    y = torch.empty_like(x)
    assert _lib.me_edges(x, w, h, words.shape[1], y, 0) == 0
    sync()
    got = S.unpack(y.cpu().numpy().view(np.uint32), w)
    assert np.array_equal(got, want)


# ------------------------------------------------------ tile configurations
def all_single_cfgs():
    out = []
    for rows, threads, ctas, vec in itertools.product([4, 8, 16, 32], [128, 256, 512],
                                                      [0, 1, 3], [1, 4]):
        out.append((0, rows, vec, threads, ctas, 32, 4))
    for kb, st, threads, ctas in itertools.product([4, 8, 16, 32, 64], [2, 3, 4],
                                                   [128, 256, 512], [0, 1]):
        if kb * st <= 216:
            out.append((1, 8, 4, threads, ctas, kb, st))
    return out


def test_every_tile_configuration():
    """Every engine and tile shape on ragged images: whole-row bands,
    column strips (rows wider than a stage), rows of 16-byte groups, of word
    pairs (64-bit accesses) and unaligned rows (cooperative loads, 32-bit
    stores), and tiny images."""
    L = _lib.load()
    saved = _lib.me_get_tile_cfg(0)
    shapes = [(97, 45), (4100, 37), (300, 129), (33, 1000), (1, 70), (40000, 19)]
    cases = []
    for s_, (w, h) in enumerate(shapes):
        img = rand_img(s_, h, w, 0.5)
        ref = O.edges(img, 0)
        cases.append((img, ref, S.round_up(S.words_per_row(w), 4), 0))
        cases.append((img, ref, S.words_per_row(w) + 1, 1))
        # 64-bit pairs: an even stride off the 16-byte grid, and 16-byte
        # rows in buffers 8 bytes past it
        cases.append((img, ref, S.round_up(S.words_per_row(w), 4) + 2, 0))
        cases.append((img, ref, S.round_up(S.words_per_row(w), 4), 2))
    try:
        for c in all_single_cfgs():
            assert _lib.me_set_tile_cfg(0, _lib.me_tile_cfg(*c)) == 0, c
            for img, ref, stride, off in cases:
                got = run_single(edges_fused, img, stride=stride, off=off)
                assert np.array_equal(got, ref), (c, img.shape, stride, off)
        assert _lib.me_device_faults(clear=True) == 0
    finally:
        L.me_set_tile_cfg(0, saved)


@pytest.mark.parametrize("kb,stages", [(32, 4), (64, 3), (8, 2)])
def test_bulk_engine_32768(kb, stages):
    """The bulk engine on the 1-Gpixel image, compared in full."""
    import torch
    L = _lib.load()
    saved = _lib.me_get_tile_cfg(0)
    w = h = 32768
    words = S.blocks_packed(w, h, seed=1)
    want = O.edges(S.unpack(words, w), 0)
    x = torch.from_numpy(words.view(np.int32)).cuda()
    y = torch.empty_like(x)
    try:
        assert _lib.me_set_tile_cfg(0, _lib.me_tile_cfg(1, 8, 4, 512, 0, kb, stages)) == 0
        assert _lib.me_edges(x, w, h, words.shape[1], y, 0) == 0
        sync()
        assert np.array_equal(S.unpack(y.cpu().numpy().view(np.uint32), w), want)
        assert _lib.me_device_faults(clear=True) == 0
    finally:
        L.me_set_tile_cfg(0, saved)


# ------------------------------------------------------------- other outputs
def fund_call(img, w, h, stride, l, r, u, d, boundary, stream):
    return _lib.load().me_fundamental_edges(img, w, h, stride, l, r, u, d, boundary, stream)


@pytest.mark.parametrize("w,h", [(1, 5), (33, 20), (200, 64), (4097, 3)])
def test_fundamental_edges(w, h):
    img = rand_img(w * h, h, w, 0.5)
    for boundary in (0, 1):
        for stride in (S.words_per_row(w), S.round_up(S.words_per_row(w), 4),
                       S.round_up(S.words_per_row(w), 4) + 2):
            got = run_single(fund_call, img, stride=stride, boundary=boundary, n_out=4)
            want = O.fundamental(img, boundary)
            for name, g_, w_ in zip(("left", "right", "up", "down"), got, want):
                assert np.array_equal(g_, w_), (name, w, h, boundary)


def test_fundamental_fig2_types():
    """The Fig. 2 hand cases fire exactly their named edge on the GPU."""
    for name, pos in (("right", (3, 4)), ("left", (3, 2)), ("up", (2, 3)), ("down", (4, 3))):
        field = np.zeros((7, 7), dtype=np.uint8)
        field[pos] = 1
        got = run_single(fund_call, field, boundary=1, n_out=4)
        fired = [n for n, g in zip(("left", "right", "up", "down"), got) if g[3, 3]]
        assert fired == [name]


@pytest.mark.parametrize("w,h", [(1, 1), (45, 31), (300, 77), (4097, 5)])
def test_display_polarity(w, h):
    img = rand_img(w + 3 * h, h, w, 0.4)
    for boundary in (0, 1):
        got = run_single(lambda *a: _lib.load().me_edges_display(*a), img,
                         stride=S.round_up(S.words_per_row(w), 4), boundary=boundary)
        assert np.array_equal(got, 1 - O.edges(img, boundary))


@pytest.mark.parametrize("w,h", [(1, 9), (40, 33), (129, 64), (2000, 11)])
def test_end_points(w, h):
    img = rand_img(w * 7 + h, h, w, 0.35)
    for boundary in (0, 1):
        for stride in (S.words_per_row(w), S.round_up(S.words_per_row(w), 4) + 4):
            got = run_single(lambda *a: _lib.load().me_end_points(*a), img, stride=stride,
                             boundary=boundary)
            assert np.array_equal(got, O.end_points(img, boundary)), (w, h, boundary)


def test_end_points_line():
    img = np.ones((5, 70), dtype=np.uint8)
    img[2, 3:60] = 0
    got = run_single(lambda *a: _lib.load().me_end_points(*a), img)
    assert np.flatnonzero(got[2]).tolist() == [3, 59] and got.sum() == 2


# --------------------------------------------- other outputs at full size
def _big_images():
    """4096 x 4096: Bernoulli(0.5) and 200 random thick polylines."""
    return {"bernoulli": rand_img(40, 4096, 4096, 0.5),
            "strokes": S.strokes(4096, 4096, 200, 41)}


OUTPUT_KINDS = {
    "fundamental": (fund_call, 4, lambda img, b: O.fundamental(img, b)),
    "display": (lambda *a: _lib.load().me_edges_display(*a), 1,
                lambda img, b: (1 - O.edges(img, b),)),
    "end_points": (lambda *a: _lib.load().me_end_points(*a), 1,
                   lambda img, b: (O.end_points(img, b),)),
}


@pytest.fixture(scope="module")
def big_images():
    return _big_images()


@pytest.mark.parametrize("kind", sorted(OUTPUT_KINDS))
@pytest.mark.parametrize("name", ["bernoulli", "strokes"])
@pytest.mark.parametrize("boundary", [0, 1])
def test_other_outputs_4096(big_images, kind, name, boundary):
    """Tall multi-tile columns on the 128-bit path: every output of every
    pixel against the oracle."""
    fn, n_out, oracle_fn = OUTPUT_KINDS[kind]
    img = big_images[name]
    got = run_single(fn, img, stride=128, boundary=boundary, n_out=n_out)
    got = got if n_out > 1 else [got]
    for k, (g_, w_) in enumerate(zip(got, oracle_fn(img, boundary))):
        assert np.array_equal(g_, w_), (kind, name, boundary, k)


@pytest.mark.parametrize("kind", sorted(OUTPUT_KINDS))
@pytest.mark.parametrize("w,h,extra", [(4097, 1500, 3), (32768, 160, 0)])
def test_other_outputs_wide_rows(kind, w, h, extra):
    """Rows wider than 32 vector columns: overlapping warps over column
    blocks (4097: one block and a ragged one; 32768: 35 blocks), compared
    in full against the oracle, both boundaries."""
    fn, n_out, oracle_fn = OUTPUT_KINDS[kind]
    img = S.strokes(w, h, 60, w + h) if w < 32768 else rand_img(42, h, w, 0.5)
    stride = S.round_up(S.words_per_row(w), 4) + extra
    for boundary in (0, 1):
        got = run_single(fn, img, stride=stride, boundary=boundary, n_out=n_out)
        got = got if n_out > 1 else [got]
        for k, (g_, w_) in enumerate(zip(got, oracle_fn(img, boundary))):
            assert np.array_equal(g_, w_), (kind, w, h, boundary, k)


# ------------------------------------------------------------- error paths
def test_host_pointer_is_rejected():
    words = np.zeros((8, 1), dtype=np.uint32)
    out = np.zeros_like(words)
    rc = _lib.load().me_edges(words.ctypes.data, 8, 8, 1, out.ctypes.data, 0, None)
    assert rc == _lib.C["ME_ERR_ARG"]


def test_alias_is_rejected():
    import torch
    x = torch.zeros(1024, dtype=torch.int32, device="cuda")
    L = _lib.load()
    assert L.me_edges(x.data_ptr(), 32, 16, 1, x.data_ptr() + 32, 0, None) == _lib.C["ME_ERR_ALIAS"]
    assert L.me_edges_staged(x.data_ptr(), 32, 16, 1, x.data_ptr(), 0, None) == _lib.C["ME_ERR_ALIAS"]


def test_streams_are_honoured():
    import torch
    img = S.strokes(1000, 800, 30, 3)
    words = S.pack(img, 32)
    x = torch.from_numpy(words.view(np.int32)).cuda()
    s = torch.cuda.Stream()
    y = torch.zeros_like(x)
    with torch.cuda.stream(s):
        assert _lib.me_edges(x, 1000, 800, 32, y, 0, s) == 0
        assert _lib.me_edges_staged(x, 1000, 800, 32, y, 0, s) == 0
    s.synchronize()
    assert np.array_equal(S.unpack(y.cpu().numpy().view(np.uint32), 1000), O.edges(img, 0))

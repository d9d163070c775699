"""Bit-exact parity of the persistent batch kernel (me_edges_batch, batch
plans) with the CPU oracle, image by image, including the full 4096-image
uneven batch the benchmark times."""
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


def sync():
    import torch
    torch.cuda.synchronize()


def make_batch(seed, n, lo, hi, pad16=True, boundaries=None, offs=None):
    shapes = S.batch_shapes(seed, n, lo, hi)
    imgs, srcs, dsts, items = [], [], [], []
    for i, (w, h) in enumerate(shapes):
        img = S.strokes(w, h, max(1, (w * h) // 4000), seed * 977 + i)
        if i % 5 == 0:       # some dense noise too
            img = (np.random.default_rng(i).random((h, w)) < 0.5).astype(np.uint8)
        stride = S.batch_stride(w, pad16)
        words = S.pack(img, stride, pad="random", seed=i)
        off = 0 if offs is None else offs[i % len(offs)]
        src = DevBuf(words, off)
        dst = DevBuf(np.zeros_like(words), off, fill=SENTINEL)
        b = 0 if boundaries is None else boundaries[i % len(boundaries)]
        imgs.append((img, b))
        srcs.append(src)
        dsts.append(dst)
        items.append((src.ptr(), dst.ptr(), w, h, stride, b))
    return imgs, srcs, dsts, items


def check_batch(imgs, srcs, dsts):
    for (img, b), src, dst in zip(imgs, srcs, dsts):
        h, w = img.shape
        assert dst.guards_intact()
        ow = dst.words()
        check_output_layout(ow, w)
        assert np.array_equal(S.unpack(ow, w), O.edges(img, b)), (w, h, b)


def image_item(img, b, seed, pad16=True):
    h, w = img.shape
    stride = S.batch_stride(w, pad16)
    words = S.pack(img, stride, pad="random", seed=seed)
    src, dst = DevBuf(words), DevBuf(np.zeros_like(words), fill=SENTINEL)
    return (img, b), src, dst, (src.ptr(), dst.ptr(), w, h, stride, b)


def set_batch_cfg(c):
    """Give both batch kinds (every image on 128-bit accesses, and some image
    on narrower ones) the configuration c; return the previous pair."""
    saved = (_lib.me_get_tile_cfg(_lib.ME_KIND_BATCH), _lib.me_get_tile_cfg(_lib.ME_KIND_BATCH_ANY))
    for kind in (_lib.ME_KIND_BATCH, _lib.ME_KIND_BATCH_ANY):
        assert _lib.me_set_tile_cfg(kind, c) == 0, (kind, c.as_dict())
    return saved


def restore_batch_cfg(saved):
    L = _lib.load()
    L.me_set_tile_cfg(_lib.ME_KIND_BATCH, saved[0])
    L.me_set_tile_cfg(_lib.ME_KIND_BATCH_ANY, saved[1])


@pytest.mark.parametrize("chunk", [1, 4, 64])
def test_many_small_images_before_a_tall_one(chunk):
    """40 one-tile images ahead of a 4000 x 40000 image (10000 tiles): the
    tile table then holds one entry per 64 tiles and its first entry
    brackets all 40 small images, which the kernel bisects."""
    saved = None
    parts = []
    rng = np.random.default_rng(5)
    for i in range(40):
        w, h = int(rng.integers(1, 129)), int(rng.integers(1, 5))
        parts.append(image_item((rng.random((h, w)) < 0.5).astype(np.uint8), i % 2, i))
    tall = S.strokes(4000, 40000, 400, 11)
    parts.append(image_item(tall, 0, 99))
    imgs, srcs, dsts, items = (list(x) for x in zip(*parts))
    try:
        saved = set_batch_cfg(_lib.me_tile_cfg(0, 4, 4, 512, 8, 32, 4, chunk))
        assert _lib.me_edges_batch(_lib.make_descs(items), len(items)) == 0
        sync()
        check_batch(imgs, srcs, dsts)
    finally:
        if saved:
            restore_batch_cfg(saved)


@pytest.mark.parametrize("pad16", [True, False])
def test_small_uneven_batch(pad16):
    imgs, srcs, dsts, items = make_batch(1, 96, 1, 700, pad16, boundaries=[0, 1])
    descs = _lib.make_descs(items)
    assert _lib.me_edges_batch(descs, len(items)) == 0
    sync()
    check_batch(imgs, srcs, dsts)


def test_misaligned_buffers_take_the_narrower_paths():
    """Buffers 0, 1, 2 and 3 words past the 16-byte grid: 128-bit, 32-bit,
    64-bit and 32-bit accesses in one launch."""
    imgs, srcs, dsts, items = make_batch(2, 40, 1, 300, True, offs=[0, 1, 2, 3])
    assert _lib.me_edges_batch(_lib.make_descs(items), len(items)) == 0
    sync()
    check_batch(imgs, srcs, dsts)


@pytest.mark.parametrize("offs", [[0, 2], [2]])
def test_batch_of_128_and_64_bit_images_only(offs):
    """Images on the 128-bit and the 64-bit paths with none on the 32-bit
    one (buffers 0 or 2 words past the 16-byte grid, rows of 16-byte
    groups): the plan must still take the kernel form that carries the
    64-bit tile, and no image may be skipped."""
    _lib.me_device_faults(clear=True)
    imgs, srcs, dsts, items = make_batch(4, 60, 1, 500, True, offs=offs)
    assert _lib.me_edges_batch(_lib.make_descs(items), len(items)) == 0
    sync()
    check_batch(imgs, srcs, dsts)
    assert _lib.me_device_faults(clear=True) == 0


def test_repeated_calls_reuse_graphs_and_slots():
    """Many calls in a row with different batch sizes: the staging ring
    and the cached graphs are reused while earlier launches may be in
    flight; every result stays exact."""
    batches = [make_batch(10 + k, n, 1, 400) for k, n in enumerate([1, 7, 64, 300, 5, 64, 2])]
    for _ in range(3):
        for imgs, srcs, dsts, items in batches:
            for d in dsts:
                d.t.fill_(int(np.int32(np.uint32(SENTINEL).view(np.int32))))
            assert _lib.me_edges_batch(_lib.make_descs(items), len(items)) == 0
        sync()
        for imgs, srcs, dsts, items in batches:
            check_batch(imgs, srcs, dsts)


def test_the_same_batch_again_reads_its_images_anew():
    """The same descriptors submitted again launch on the plan already on the
    device: each call's edge maps still come from the images as they are at
    that call (new content written into the same buffers before every call,
    outputs reset to a sentinel), with another batch submitted in between
    and a change of one descriptor (an output moved) planned afresh."""
    import torch
    from tests.gpu_util import GUARD
    imgs, srcs, dsts, items = make_batch(21, 50, 1, 600)
    other = make_batch(22, 30, 1, 400)
    descs = _lib.make_descs(items)
    rng = np.random.default_rng(4)
    sentinel = int(np.uint32(SENTINEL).view(np.int32))
    for rep in range(5):
        fresh = []
        for (img, b), src, it in zip(imgs, srcs, items):
            new = (rng.random(img.shape) < 0.3 + 0.1 * rep).astype(np.uint8)
            words = S.pack(new, it[4], pad="random", seed=rep)
            src.t[GUARD + src.off:GUARD + src.off + src.n] = \
                torch.from_numpy(words.view(np.int32).ravel()).to(src.t.device)
            fresh.append((new, b))
        for d in dsts:
            d.t.fill_(sentinel)
        assert _lib.me_edges_batch(descs, len(items)) == 0
        if rep % 2 == 1:
            assert _lib.me_edges_batch(_lib.make_descs(other[3]), len(other[3])) == 0
        sync()
        check_batch(fresh, srcs, dsts)
        if rep % 2 == 1:
            check_batch(*other[:3])
    # one output moved: a new plan, the right buffer written
    moved = DevBuf(np.zeros_like(dsts[0].words()), fill=SENTINEL)
    items2 = list(items)
    items2[0] = (items[0][0], moved.ptr()) + tuple(items[0][2:])
    for d in dsts:
        d.t.fill_(sentinel)
    assert _lib.me_edges_batch(_lib.make_descs(items2), len(items2)) == 0
    sync()
    check_batch(fresh[:1], srcs[:1], [moved])
    check_batch(fresh[1:], srcs[1:], dsts[1:])
    assert (dsts[0].words() == np.uint32(SENTINEL)).all()


def batch_cfgs():
    out = []
    chunks = itertools.cycle([1, 3, 4, 64])
    for rows, threads, ctas, vec in itertools.product([4, 8, 16, 32], [128, 256, 512],
                                                      [0, 1, 2, 8], [1, 4]):
        out.append((0, rows, vec, threads, ctas, 32, 4, next(chunks)))
    # tiles per chunk, persistent and one chunk per warp
    for ctas, chunk in itertools.product([0, 8], [0, 1, 2, 5, 8, 16, 17, 64]):
        out.append((0, 4, 4, 512, ctas, 32, 4, chunk))
    for kb, st, threads, ctas in itertools.product([4, 16, 32, 64], [2, 3, 4],
                                                   [128, 256, 512], [0, 1, 2]):
        if kb * st <= 216:
            out.append((1, 8, 4, threads, ctas, kb, st))
    return out


def test_every_batch_configuration():
    """Every configuration on a batch of both kinds' images (buffers on and
    off the 16-byte grid), set for both batch kinds."""
    saved = set_batch_cfg(_lib.me_get_tile_cfg(_lib.ME_KIND_BATCH))
    imgs, srcs, dsts, items = make_batch(3, 50, 1, 1200, offs=[0, 0, 2, 1])
    # one very wide image forces column strips in the bulk engine
    wide = (np.random.default_rng(9).random((21, 30000)) < 0.5).astype(np.uint8)
    words = S.pack(wide, S.batch_stride(30000), pad="random", seed=3)
    src, dst = DevBuf(words), DevBuf(np.zeros_like(words), fill=SENTINEL)
    imgs.append((wide, 0)); srcs.append(src); dsts.append(dst)
    items.append((src.ptr(), dst.ptr(), 30000, 21, words.shape[1], 0))
    descs = _lib.make_descs(items)
    try:
        for c in batch_cfgs():
            set_batch_cfg(_lib.me_tile_cfg(*c))
            for d in dsts:
                d.t.fill_(int(np.uint32(SENTINEL).view(np.int32)))
            assert _lib.me_edges_batch(descs, len(items)) == 0
            sync()
            check_batch(imgs, srcs, dsts)
        assert _lib.me_device_faults(clear=True) == 0
    finally:
        restore_batch_cfg(saved)


def test_plan_replays():
    imgs, srcs, dsts, items = make_batch(4, 80, 1, 900, boundaries=[1, 0, 0])
    plan = _lib.BatchPlan(_lib.make_descs(items), len(items))
    want = sum(2 * it[3] * it[4] * 4 for it in items)
    assert plan.bytes == want
    for _ in range(5):
        assert plan.run() == 0
    sync()
    check_batch(imgs, srcs, dsts)
    plan.close()


def test_batch_matches_single_calls():
    import torch
    imgs, srcs, dsts, items = make_batch(5, 64, 16, 2000)
    assert _lib.me_edges_batch(_lib.make_descs(items), len(items)) == 0
    for (img, b), src, dst, it in zip(imgs, srcs, dsts, items):
        ref = torch.empty_like(dst.t)
        off = (dst.ptr() - dst.t.data_ptr())
        assert _lib.me_edges(it[0], it[2], it[3], it[4], ref.data_ptr() + off, it[5]) == 0
        sync()
        a = dst.t.cpu().numpy()
        r = ref.cpu().numpy()
        n = it[3] * it[4]
        lo = off // 4
        nw = S.words_per_row(it[2])
        aa = a[lo:lo + n].reshape(it[3], it[4])[:, :nw]
        rr = r[lo:lo + n].reshape(it[3], it[4])[:, :nw]
        assert np.array_equal(aa, rr)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_full_uneven_batch_4096(seed):
    """The benchmark's batch (seed 0) and two more draws of it: 4096 images,
    log-uniform 16..4096 per side, glyph strokes, rows padded to 16 bytes;
    every image against the oracle."""
    import torch
    batch = S.batch(seed, workers=8)
    srcs, dsts, items = [], [], []
    for im in batch:
        x = torch.from_numpy(im.words.view(np.int32)).cuda()
        y = torch.full_like(x, int(np.uint32(SENTINEL).view(np.int32)))
        srcs.append(x)
        dsts.append(y)
        items.append((x, y, im.w, im.h, im.stride_words, 0))
    assert _lib.me_edges_batch(_lib.make_descs(items), len(items)) == 0
    sync()
    for im, y in zip(batch, dsts):
        ow = y.cpu().numpy().view(np.uint32)
        check_output_layout(ow, im.w)
        img = S.unpack(im.words, im.w)
        assert np.array_equal(S.unpack(ow, im.w), O.edges(img, 0)), (im.w, im.h)


def test_zero_and_bad_batches():
    L = _lib.load()
    assert L.me_edges_batch(None, 0, None) == 0
    imgs, srcs, dsts, items = make_batch(6, 3, 16, 64)
    bad = list(items)
    bad[1] = (bad[1][0], bad[1][1], bad[1][2], bad[1][3], 0, 0)   # stride 0
    assert _lib.me_edges_batch(_lib.make_descs(bad), 3) == _lib.C["ME_ERR_ARG"]


# ------------------------------------------------------- batch in host memory
def host_batch(seed, n, lo, hi, gap_words=0, align4=True):
    """Images packed one after another in one host buffer (optionally with
    gaps), as me_edges_batch_host takes them."""
    shapes = S.batch_shapes(seed, n, lo, hi)
    imgs, items, off = [], [], 0
    for i, (w, h) in enumerate(shapes):
        img = S.strokes(w, h, max(1, (w * h) // 3000), seed * 31 + i)
        stride = S.batch_stride(w, pad16=align4)
        words = S.pack(img, stride, pad="random", seed=i)
        imgs.append((img, words, off))
        items.append((off, w, h, stride, i % 2))
        off += words.size + gap_words
        if align4:
            off = (off + 3) // 4 * 4
    buf = np.full(off + 16, SENTINEL, dtype=np.uint32)
    for img, words, o in imgs:
        buf[o:o + words.size] = words.ravel()
    return imgs, items, buf


def check_host(imgs, items, out):
    covered = np.zeros(out.size, dtype=bool)
    for (img, words, o), it in zip(imgs, items):
        h, w = img.shape
        ow = out[o:o + words.size].reshape(words.shape)
        check_output_layout(ow, w)
        assert np.array_equal(S.unpack(ow, w), O.edges(img, it[4])), (w, h)
        covered[o:o + words.size] = True
    assert (out[~covered] == SENTINEL).all(), "bytes between images were written"


@pytest.mark.parametrize("chunk", [0, 1 << 20, 64 << 10])
def test_host_batch_chunks(chunk):
    imgs, items, buf = host_batch(20, 120, 1, 1500)
    out = np.full_like(buf, SENTINEL)
    rc = _lib.me_edges_batch_host(buf, out, _lib.make_host_images(items), len(items), chunk)
    assert rc == 0, _lib.status_string(rc)
    check_host(imgs, items, out)


def test_host_batch_gaps_unaligned_and_pinned():
    import torch
    imgs, items, buf = host_batch(21, 60, 1, 900, gap_words=5, align4=False)
    pin_in = torch.from_numpy(buf.view(np.int32)).pin_memory()
    pin_out = torch.full_like(pin_in, int(np.uint32(SENTINEL).view(np.int32))).pin_memory()
    rc = _lib.me_edges_batch_host(pin_in, pin_out, _lib.make_host_images(items), len(items),
                                  256 << 10)
    assert rc == 0, _lib.status_string(rc)
    check_host(imgs, items, pin_out.numpy().view(np.uint32))
    assert _lib.me_device_faults(clear=True) == 0


def at_page_offset(a, offset):
    """A copy of `a` whose first byte sits `offset` bytes past a 4 KiB page."""
    raw = np.empty(a.size + 2048, dtype=np.uint32)
    skip = ((offset - raw.ctypes.data) % 4096) // 4
    out = raw[skip:skip + a.size]
    out[:] = a
    assert out.ctypes.data % 4096 == offset
    return out


@pytest.mark.parametrize("in_off,out_off", [(48, 2064), (4080, 16), (4, 4092)])
def test_host_batch_page_offsets(in_off, out_off):
    """Copies are split at host page boundaries and the first chunk's upload
    cannot start below the input buffer: buffers that start part way into a
    page, small chunks so most chunks start mid-page, gaps between images."""
    imgs, items, buf = host_batch(23, 80, 1, 700, gap_words=3, align4=in_off % 16 == 0)
    src = at_page_offset(buf, in_off)
    out = at_page_offset(np.full_like(buf, SENTINEL), out_off)
    rc = _lib.me_edges_batch_host(src, out, _lib.make_host_images(items), len(items), 64 << 10)
    assert rc == 0, _lib.status_string(rc)
    check_host(imgs, items, out)


def test_host_batch_errors():
    imgs, items, buf = host_batch(22, 4, 16, 64)
    L = _lib.load()
    descs = _lib.make_host_images(items)
    assert L.me_edges_batch_host(buf.ctypes.data, buf.ctypes.data, descs, 4, 0, None) == \
        _lib.C["ME_ERR_ALIAS"]
    bad = _lib.make_host_images([(-4,) + tuple(items[0][1:])])
    out = np.empty_like(buf)
    assert L.me_edges_batch_host(buf.ctypes.data, out.ctypes.data, bad, 1, 0, None) == \
        _lib.C["ME_ERR_ARG"]
    assert L.me_edges_batch_host(None, None, None, 0, 0, None) == 0

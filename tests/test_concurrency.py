"""Thread safety of the C ABI: several host threads, each on its own CUDA
stream, call me_edges_batch, me_edges and me_edges_batch_host at the same
time (the ctypes calls release the GIL); every result is checked against
the oracle."""
import threading

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


def make_batch(seed, n, lo, hi):
    imgs, srcs, dsts, items = [], [], [], []
    for i, (w, h) in enumerate(S.batch_shapes(seed, n, lo, hi)):
        img = S.strokes(w, h, max(1, (w * h) // 4000), seed * 131 + i)
        stride = S.batch_stride(w)
        words = S.pack(img, stride, pad="random", seed=i)
        src, dst = DevBuf(words), DevBuf(np.zeros_like(words), fill=SENTINEL)
        imgs.append(img)
        srcs.append(src)
        dsts.append(dst)
        items.append((src.ptr(), dst.ptr(), w, h, stride, 0))
    return imgs, srcs, dsts, items


def check(imgs, dsts):
    for img, dst in zip(imgs, dsts):
        h, w = img.shape
        assert dst.guards_intact()
        out = dst.words()
        check_output_layout(out, w)
        assert np.array_equal(S.unpack(out, w), O.edges(img, 0)), (w, h)


def test_threads_on_their_own_streams():
    import torch
    work = [make_batch(40 + k, n, 1, 900) for k, n in enumerate([3, 50, 17, 120])]
    torch.cuda.synchronize()            # uploads done before other streams use them
    errors = []

    def worker(k):
        try:
            imgs, srcs, dsts, items = work[k]
            s = torch.cuda.Stream()
            descs = _lib.make_descs(items)
            for r in range(8):
                with torch.cuda.stream(s):
                    for d in dsts:
                        d.t.fill_(int(np.uint32(SENTINEL).view(np.int32)))
                if r % 2 == 0:
                    rc = _lib.me_edges_batch(descs, len(items), s)
                    if rc != 0:
                        raise _lib.MeError(rc, "me_edges_batch")
                else:
                    for img_p, edge_p, w, h, stride, b in items:
                        rc = _lib.me_edges(img_p, w, h, stride, edge_p, b, s)
                        if rc != 0:
                            raise _lib.MeError(rc, "me_edges")
                s.synchronize()
                check(imgs, dsts)
        except Exception as e:          # reported in the main thread
            errors.append((k, repr(e)))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(len(work))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors


def test_host_batches_from_two_threads():
    """me_edges_batch_host keeps one pipeline per device; two threads share
    it (calls are serialised inside) and both results stay exact."""
    errors = []

    def worker(k):
        try:
            shapes = S.batch_shapes(60 + k, 80, 1, 700)
            imgs, items, off = [], [], 0
            for i, (w, h) in enumerate(shapes):
                img = S.strokes(w, h, 3, k * 97 + i)
                stride = S.batch_stride(w)
                words = S.pack(img, stride, pad="random", seed=i)
                imgs.append((img, words, off))
                items.append((off, w, h, stride, 0))
                off += words.size
            buf = np.zeros(off, dtype=np.uint32)
            for img, words, o in imgs:
                buf[o:o + words.size] = words.ravel()
            for _ in range(4):
                out = np.full_like(buf, SENTINEL)
                rc = _lib.me_edges_batch_host(buf, out, _lib.make_host_images(items),
                                              len(items), 64 << 10)
                if rc != 0:
                    raise _lib.MeError(rc, "me_edges_batch_host")
                for img, words, o in imgs:
                    h, w = img.shape
                    got = S.unpack(out[o:o + words.size].reshape(words.shape), w)
                    if not np.array_equal(got, O.edges(img, 0)):
                        raise AssertionError(f"host batch {k}: image {w}x{h} differs")
        except Exception as e:
            errors.append((k, repr(e)))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors

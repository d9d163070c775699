"""Bit-exact parity of me_threshold_edges (grey image thresholded and its
edges found in one pass) with the oracle's threshold followed by its edge
map: widths across word boundaries, tight and 16-byte pitches, thresholds
at both ends, both boundary colours, with and without the binary output."""
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


def grey_image(w, h, seed):
    """Smooth ramps plus noise, so every threshold cuts shapes out of it."""
    g = np.random.default_rng(seed)
    y, x = np.mgrid[0:h, 0:w]
    base = (np.sin(x / (3 + seed)) + np.cos(y / (5 + seed))) * 60 + 128
    return np.clip(base + g.normal(0, 25, (h, w)), 0, 255).astype(np.uint8)


def run(grey, t, b, pitch, stride, with_binary, grey_off=0):
    import torch
    h, w = grey.shape
    buf = np.full(h * pitch + 64, 7, dtype=np.uint8)
    for y in range(h):
        buf[grey_off + y * pitch:grey_off + y * pitch + w] = grey[y]
    dgrey = torch.from_numpy(buf).cuda()
    zero = np.zeros((h, stride), dtype=np.uint32)
    edge = DevBuf(zero, fill=SENTINEL)
    binary = DevBuf(zero, fill=SENTINEL) if with_binary else None
    rc = _lib.me_threshold_edges(dgrey.data_ptr() + grey_off, w, h, pitch, t, edge.ptr(), stride,
                                 binary.ptr() if binary else None, b)
    assert rc == 0, _lib.status_string(rc)
    torch.cuda.synchronize()
    bw = O.threshold(grey, t)
    for out, want in ((edge, O.edges(bw, b)), (binary, bw)):
        if out is None:
            continue
        assert out.guards_intact()
        words = out.words()
        check_output_layout(words, w)
        assert np.array_equal(S.unpack(words, w), want), (w, h, t, b, pitch)


WIDTHS = [1, 2, 31, 32, 33, 63, 64, 65, 100, 959, 960, 961, 1000, 4095, 4096, 4097]


@pytest.mark.parametrize("w", WIDTHS)
def test_widths_pitches_thresholds(w):
    cases = itertools.cycle(itertools.product([0, 1, 100, 128, 255, 256], [0, 1], [False, True]))
    for k, pitch in enumerate([w, (w + 15) // 16 * 16, (w + 15) // 16 * 16 + 48]):
        t, b, with_binary = next(cases)
        h = [1, 17, 300][k]
        grey = grey_image(w, h, w + k)
        stride = S.batch_stride(w) + (k == 2)
        run(grey, t, b, pitch, stride, with_binary)


@pytest.mark.parametrize("t", [0, 1, 64, 127, 128, 200, 255, 256, 1000, -5])
def test_thresholds_on_one_image(t):
    grey = grey_image(777, 333, 3)
    run(grey, t, 0, 784, S.batch_stride(777), True)


def test_unaligned_grey_start():
    grey = grey_image(500, 120, 5)
    run(grey, 128, 1, 512, S.batch_stride(500), True, grey_off=3)


@pytest.mark.parametrize("pitch", [2000, 2003])
def test_tall_image_long_bands(pitch):
    """A tall image in few column blocks: each warp walks a band of many rows
    (rows pass through the row ring several times; the last band is partly
    filled), on the 16-byte path (pitch 2000) and the byte path (2003).
    Every row is compared."""
    grey = np.tile(grey_image(2000, 667, 11), (30, 1))[:20001]
    run(grey, 128, 1, pitch, S.batch_stride(2000), True)


def test_large_image_sampled_rows():
    """8192 x 8192 (64 MiB of grey): whole rows compared at the top, the
    bottom and every 512th row in between."""
    import torch
    w = h = 8192
    grey = grey_image(w, 256, 9)
    big = np.tile(grey, (h // 256, 1))
    dgrey = torch.from_numpy(big).cuda()
    edge = torch.empty((h, w // 32), dtype=torch.int32, device="cuda")
    assert _lib.me_threshold_edges(dgrey, w, h, w, 128, edge, w // 32) == 0
    torch.cuda.synchronize()
    out = edge.cpu().numpy().view(np.uint32)
    want = O.edges(O.threshold(big, 128), 0)
    for y in list(range(0, h, 512)) + [h - 1]:
        assert np.array_equal(S.unpack(out[y:y + 1], w)[0], want[y]), y


def test_bad_arguments():
    import torch
    L = _lib.load()
    g = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    e = torch.zeros(1024, dtype=torch.int32, device="cuda")
    ARG, ALIAS = _lib.C["ME_ERR_ARG"], _lib.C["ME_ERR_ALIAS"]
    assert L.me_threshold_edges(g.data_ptr(), 64, 4, 63, 128, e.data_ptr(), 2, None, 0, None) == ARG
    assert L.me_threshold_edges(g.data_ptr(), 64, 4, 64, 128, e.data_ptr(), 1, None, 0, None) == ARG
    assert L.me_threshold_edges(g.data_ptr(), 64, 4, 64, 128, e.data_ptr(), 2, None, 2, None) == ARG
    assert L.me_threshold_edges(g.data_ptr(), 64, 4, 64, 128, g.data_ptr() + 64, 2, None, 0,
                                None) == ALIAS
    assert L.me_threshold_edges(g.data_ptr(), 64, 4, 64, 128, e.data_ptr(), 2, e.data_ptr(), 0,
                                None) == ALIAS


# ---------------------------------------------------------------------------
# Otsu's threshold chosen on the device (me_threshold_edges_otsu)
# ---------------------------------------------------------------------------

def mixture(seed, h, w, mus=(60, 180), sigmas=(15, 20), weights=(0.5, 0.5)):
    g = np.random.default_rng(seed)
    k = g.choice(len(mus), size=(h, w), p=weights)
    v = g.normal(np.asarray(mus)[k], np.asarray(sigmas)[k])
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


def run_otsu(grey, b, pitch, stride, with_binary, grey_off=0, t_out=True):
    """me_threshold_edges_otsu against the oracle: the threshold equals the
    oracle's Otsu threshold, and edge (and binary) equal the oracle's edge
    map of the image thresholded there.  Padding bytes of each grey row hold
    7s, which must not enter the histogram."""
    import torch
    h, w = grey.shape
    buf = np.full(h * pitch + 64, 7, dtype=np.uint8)
    for y in range(h):
        buf[grey_off + y * pitch:grey_off + y * pitch + w] = grey[y]
    dgrey = torch.from_numpy(buf).cuda()
    zero = np.zeros((h, stride), dtype=np.uint32)
    edge = DevBuf(zero, fill=SENTINEL)
    binary = DevBuf(zero, fill=SENTINEL) if with_binary else None
    tdev = torch.full((4,), -7, dtype=torch.int32, device="cuda") if t_out else None
    rc = _lib.me_threshold_edges_otsu(dgrey.data_ptr() + grey_off, w, h, pitch, edge.ptr(),
                                      stride, binary.ptr() if binary else None, b,
                                      tdev[1:2] if t_out else None)
    assert rc == 0, _lib.status_string(rc)
    torch.cuda.synchronize()
    t = O.otsu_threshold(grey)
    if t_out:
        got = tdev.cpu().numpy()
        assert got[1] == t, (w, h, got[1], t)
        assert got[0] == -7 and got[2] == -7          # nothing else written
    bw = O.threshold(grey, t)
    for out, want in ((edge, O.edges(bw, b)), (binary, bw)):
        if out is None:
            continue
        assert out.guards_intact()
        words = out.words()
        check_output_layout(words, w)
        assert np.array_equal(S.unpack(words, w), want), (w, h, t, b, pitch)
    return t


@pytest.mark.parametrize("w", [1, 2, 31, 32, 33, 100, 961, 4096, 4097])
def test_otsu_widths_and_pitches(w):
    for k, pitch in enumerate([w, (w + 15) // 16 * 16, (w + 15) // 16 * 16 + 48]):
        h = [1, 17, 300][k]
        run_otsu(mixture(w + k, h, w), k % 2, pitch, S.batch_stride(w) + (k == 2), k != 1)


def test_otsu_image_kinds():
    # bimodal photo-like, three modes, smooth ramps, a dark image with few
    # bright pixels, two grey levels, constant images, one pixel
    run_otsu(mixture(1, 333, 777), 0, 784, S.batch_stride(777), True)
    run_otsu(mixture(2, 200, 640, (40, 120, 220), (10, 10, 10), (0.3, 0.4, 0.3)), 1, 640, 20, True)
    run_otsu(grey_image(500, 120, 4), 0, 512, S.batch_stride(500), False)
    run_otsu(mixture(3, 64, 96, (20, 235), (5, 5), (0.95, 0.05)), 0, 96, 4, True)
    assert run_otsu(np.array([[50] * 10 + [200] * 30] * 3, dtype=np.uint8), 0, 48, 4, True) == 51
    for v in (0, 1, 77, 255):
        assert run_otsu(np.full((9, 40), v, dtype=np.uint8), 0, 48, 4, True) == v
    run_otsu(np.array([[9]], dtype=np.uint8), 0, 16, 4, True)


def test_otsu_unaligned_start_and_no_threshold_out():
    run_otsu(mixture(5, 120, 500), 1, 512, S.batch_stride(500), True, grey_off=3)
    run_otsu(mixture(6, 150, 1000), 0, 1008, S.batch_stride(1000), True, t_out=False)


def test_otsu_large_image():
    """4096 x 8192 (32 MiB of grey), every row compared."""
    run_otsu(np.tile(mixture(7, 512, 4096), (16, 1)), 0, 4096, 128, False)


def test_otsu_bad_arguments():
    import torch
    L = _lib.load()
    g = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    e = torch.zeros(1024, dtype=torch.int32, device="cuda")
    t = torch.zeros(4, dtype=torch.int32, device="cuda")
    ARG, ALIAS = _lib.C["ME_ERR_ARG"], _lib.C["ME_ERR_ALIAS"]
    assert L.me_threshold_edges_otsu(g.data_ptr(), 64, 4, 63, e.data_ptr(), 2, None, 0,
                                     t.data_ptr(), None) == ARG
    assert L.me_threshold_edges_otsu(g.data_ptr(), 64, 4, 64, e.data_ptr(), 2, None, 0,
                                     t.data_ptr() + 2, None) == ARG
    assert L.me_threshold_edges_otsu(g.data_ptr(), 64, 4, 64, e.data_ptr(), 2, None, 0,
                                     e.data_ptr() + 4, None) == ALIAS
    assert L.me_threshold_edges_otsu(g.data_ptr(), 64, 4, 64, e.data_ptr(), 2, None, 0,
                                     g.data_ptr() + 8, None) == ALIAS
    assert L.me_threshold_edges_otsu(g.data_ptr(), 64, 4, 64, g.data_ptr() + 64, 2, None, 0,
                                     None, None) == ALIAS

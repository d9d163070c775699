"""Packed layout and seeded generators (no edge arithmetic here)."""
import os

import numpy as np
import pytest

from paper_1401_5245_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_layout():
    rows = []
    with open(os.path.join(GOLDEN, "pack_layout.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w, stride, white, *words = line.split()
            cols = [] if white == "-" else [int(c) for c in white.split(",")]
            rows.append((int(w), int(stride), cols, [int(x, 16) for x in words]))
    return rows


@pytest.mark.parametrize("w,stride,white,words", load_layout())
def test_pack_layout_fixture(w, stride, white, words):
    img = np.zeros((1, w), dtype=np.uint8)
    img[0, white] = 1
    packed = S.pack(img, stride, pad=0)
    assert packed.dtype == np.uint32 and packed.shape == (1, stride)
    assert packed[0].tolist() == words
    assert np.array_equal(S.unpack(packed, w), img)


@pytest.mark.parametrize("seed", range(5))
def test_roundtrip_with_garbage_padding(seed):
    g = np.random.default_rng(seed)
    h, w = int(g.integers(1, 50)), int(g.integers(1, 200))
    img = (g.random((h, w)) < 0.5).astype(np.uint8)
    nw = S.words_per_row(w)
    for stride in (nw, nw + 3):
        for pad in (0, 1, "random"):
            packed = S.pack(img, stride, pad=pad, seed=seed)
            assert np.array_equal(S.unpack(packed, w), img)


def test_generators_are_seeded():
    assert np.array_equal(S.ellipse_glyphs(3), S.ellipse_glyphs(3))
    assert not np.array_equal(S.ellipse_glyphs(3), S.ellipse_glyphs(4))
    a = S.strokes(300, 200, 20, 7)
    assert a.shape == (200, 300) and 0.3 < a.mean() < 1.0
    assert np.array_equal(a, S.strokes(300, 200, 20, 7))
    b = S.bernoulli(128, 64, 0.9, 1)
    assert abs((b == 0).mean() - 0.9) < 0.02


def test_packed_generators():
    w, h = 256, 130
    bp = S.blocks_packed(w, h, seed=1, block=64)
    img = S.unpack(bp, w)
    # every 64x64 block is a single colour
    for by in range(0, h, 64):
        for bx in range(0, w, 64):
            blk = img[by:by + 64, bx:bx + 64]
            assert blk.min() == blk.max()
    rp = S.bernoulli_half_packed(100, 50, seed=2, stride_words=8)
    assert rp.shape == (50, 8)
    assert 0.45 < S.unpack(rp, 100).mean() < 0.55


def test_capsule_is_the_distance_set():
    """The stroke rasteriser marks exactly the pixel centres within t/2 of
    the segment (checked by brute-force distance on a small canvas)."""
    g = np.random.default_rng(0)
    for _ in range(20):
        w, h = 40, 30
        ax, ay, bx, by = g.uniform(-5, 45), g.uniform(-5, 35), g.uniform(-5, 45), g.uniform(-5, 35)
        r = float(g.uniform(0.5, 4))
        c = S._Canvas(w, h)
        c.capsule(ax, ay, bx, by, r)
        got = c.render() == 0
        yy, xx = np.mgrid[0:h, 0:w].astype(float)
        vx, vy = bx - ax, by - ay
        L2 = vx * vx + vy * vy
        t = np.clip(((xx - ax) * vx + (yy - ay) * vy) / L2, 0, 1) if L2 > 0 else 0
        d = np.hypot(xx - (ax + t * vx), yy - (ay + t * vy))
        want = d <= r
        # allow disagreement only for centres within 1e-6 of the boundary
        diff = got != want
        assert np.all(np.abs(d[diff] - r) < 1e-6)


def test_batch_shapes_and_strides():
    shapes = S.batch_shapes(0, n=4096)
    ws = np.array([w for w, _ in shapes])
    hs = np.array([h for _, h in shapes])
    assert ws.min() >= 16 and ws.max() <= 4096 and hs.min() >= 16
    assert (ws % 32 != 0).mean() > 0.9
    for w in (16, 33, 100, 4096):
        assert S.batch_stride(w) % 4 == 0 and S.batch_stride(w) >= S.words_per_row(w)
        assert S.batch_stride(w, pad16=False) == S.words_per_row(w)
    imgs = S.batch(0, n=8)
    assert [(i.w, i.h) for i in imgs] == S.batch_shapes(0, n=8)


def test_serve_trace():
    t, cls = S.serve_trace(0, 5000, rate_hz=1000.0)
    assert np.all(np.diff(t) >= 0)
    frac = np.bincount(cls, minlength=3) / len(cls)
    assert abs(frac[0] - 0.70) < 0.03 and abs(frac[1] - 0.25) < 0.03

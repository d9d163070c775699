"""Seeded synthetic binary images and the packed 1-bit row layout.

This module draws inputs and converts between two storage forms of the same
bitmap. It holds none of the edge arithmetic (no mask, no shift, no AND/OR of
neighbours), so both the CUDA path and the CPU oracle can take their inputs
from it without sharing any of the method.

Pixel convention (Section 2 of the paper: a monochrome bitmap holds one bit
per pixel, 0 for black and 1 for white):

* byte image  ``u8[h, w]``: one byte per pixel, 0 = black, 1 = white.
* packed rows ``uint32[h, stride_words]``: pixel (x, y) is bit ``x % 32`` of
  word ``y * stride_words + x // 32``; the least significant bit is the
  leftmost pixel and row 0 is the top row.  Bits at ``x >= w`` of the last
  word of a row, and words ``>= ceil(w / 32)``, are padding.

Shapes are rasterised from their exact definitions at integer pixel centres:
a stroke of width ``t`` is every pixel centre within ``t / 2`` of a segment
(a capsule), an ellipse is every centre inside the rotated ellipse.  All
random draws come from numpy's PCG64 seeded with the caller's seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

WHITE = 1
BLACK = 0


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def words_per_row(w: int) -> int:
    return (int(w) + 31) // 32


def round_up(v: int, m: int) -> int:
    return (int(v) + m - 1) // m * m


# ----------------------------------------------------------------------------
# packed layout
# ----------------------------------------------------------------------------

def pack(img: np.ndarray, stride_words: int | None = None,
         pad: str | int = 0, seed: int = 0) -> np.ndarray:
    """Pack a byte image ``u8[h, w]`` into ``uint32[h, stride_words]`` rows.

    ``pad`` chooses what goes into padding bits and padding words: an integer
    bit value (0 or 1) for all of them, or ``"random"`` for seeded garbage,
    which a correct consumer must ignore.
    """
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if img.ndim != 2:
        raise ValueError("pack expects a 2-D byte image")
    h, w = img.shape
    nw = words_per_row(w)
    if stride_words is None:
        stride_words = nw
    if stride_words < nw:
        raise ValueError("stride_words < ceil(w/32)")
    if pad == "random":
        out = rng(seed).integers(0, 2 ** 32, size=(h, stride_words),
                                 dtype=np.uint64).astype(np.uint32)
        pad_bit = None
    else:
        pad_bit = 1 if int(pad) else 0
        out = np.full((h, stride_words), 0xFFFFFFFF if pad_bit else 0,
                      dtype=np.uint32)
    if h == 0 or w == 0:
        return out
    wpad = nw * 32
    bits = np.empty((h, wpad), dtype=np.uint8)
    bits[:, :w] = img != 0
    if wpad > w:
        if pad_bit is None:
            bits[:, w:] = rng(seed + 1).integers(0, 2, size=(h, wpad - w),
                                                 dtype=np.uint8)
        else:
            bits[:, w:] = pad_bit
    packed = np.packbits(bits, axis=1, bitorder="little")
    out[:, :nw] = packed.view("<u4").reshape(h, nw)
    return out


def unpack(words: np.ndarray, w: int) -> np.ndarray:
    """Inverse of :func:`pack` for the first ``w`` pixels of every row."""
    words = np.ascontiguousarray(words, dtype=np.uint32)
    h = words.shape[0]
    nw = words_per_row(w)
    if h == 0 or w == 0:
        return np.zeros((h, w), dtype=np.uint8)
    as_bytes = words[:, :nw].astype("<u4").view(np.uint8).reshape(h, nw * 4)
    bits = np.unpackbits(as_bytes, axis=1, bitorder="little")
    return np.ascontiguousarray(bits[:, :w])


# ----------------------------------------------------------------------------
# shape rasterisers
# ----------------------------------------------------------------------------

def _capsule_rows(ax, ay, bx, by, r, w, h):
    """Rows ``ys`` and closed column ranges ``[xl, xr]`` of the pixel centres
    within distance ``r`` of segment AB, clipped to the image."""
    y0 = max(0, int(math.ceil(min(ay, by) - r)))
    y1 = min(h - 1, int(math.floor(max(ay, by) + r)))
    if y1 < y0:
        e = np.zeros(0, dtype=np.int64)
        return e, e, e
    ys = np.arange(y0, y1 + 1, dtype=np.float64)
    lo = np.full(ys.shape, np.inf)
    hi = np.full(ys.shape, -np.inf)
    # the two end discs
    for cx, cy in ((ax, ay), (bx, by)):
        dy = ys - cy
        inside = np.abs(dy) <= r
        half = np.sqrt(np.maximum(r * r - dy * dy, 0.0))
        lo = np.where(inside, np.minimum(lo, cx - half), lo)
        hi = np.where(inside, np.maximum(hi, cx + half), hi)
    # the slab between them: 0 <= (p-A).d <= L and |(p-A) x d| <= r
    L = math.hypot(bx - ax, by - ay)
    if L > 0:
        dx, dy = (bx - ax) / L, (by - ay) / L
        slo = np.full(ys.shape, -np.inf)
        shi = np.full(ys.shape, np.inf)
        ok = np.ones(ys.shape, dtype=bool)
        ry = ys - ay
        # (x-ax)*c + const must lie in [lim_lo, lim_hi]: first the position
        # along the axis, then the signed distance across it
        for c, const, lim_lo, lim_hi in ((dx, ry * dy, 0.0, L),
                                         (dy, -ry * dx, -r, r)):
            if abs(c) < 1e-12:
                ok &= (const >= lim_lo) & (const <= lim_hi)
            else:
                a = (lim_lo - const) / c + ax
                b = (lim_hi - const) / c + ax
                slo = np.maximum(slo, np.minimum(a, b))
                shi = np.minimum(shi, np.maximum(a, b))
        ok &= slo <= shi
        lo = np.where(ok, np.minimum(lo, slo), lo)
        hi = np.where(ok, np.maximum(hi, shi), hi)
    xl = np.maximum(np.ceil(lo - 1e-9), 0)
    xr = np.minimum(np.floor(hi + 1e-9), w - 1)
    keep = np.isfinite(lo) & (xl <= xr)
    return (ys[keep].astype(np.int64), xl[keep].astype(np.int64),
            xr[keep].astype(np.int64))


class _Canvas:
    """White canvas that accumulates black row intervals, then renders."""

    def __init__(self, w: int, h: int):
        self.w, self.h = int(w), int(h)
        self.ys, self.xl, self.xr = [], [], []

    def capsule(self, ax, ay, bx, by, r):
        ys, xl, xr = _capsule_rows(ax, ay, bx, by, r, self.w, self.h)
        if ys.size:
            self.ys.append(ys)
            self.xl.append(xl)
            self.xr.append(xr)

    def polyline(self, pts, r):
        for (ax, ay), (bx, by) in zip(pts[:-1], pts[1:]):
            self.capsule(ax, ay, bx, by, r)

    def render(self) -> np.ndarray:
        w, h = self.w, self.h
        if not self.ys:
            return np.ones((h, w), dtype=np.uint8)
        ys = np.concatenate(self.ys)
        xl = np.concatenate(self.xl)
        xr = np.concatenate(self.xr)
        width = w + 1
        n = h * width
        diff = np.bincount(ys * width + xl, minlength=n)[:n]
        diff -= np.bincount(ys * width + xr + 1, minlength=n)[:n]
        cover = np.cumsum(diff.reshape(h, width), axis=1)[:, :w]
        return (cover <= 0).astype(np.uint8)


def ellipse_glyphs(seed: int, w: int = 256, h: int = 256, n_shapes: int = 40,
                   rmin: int = 2, rmax: int = 20, flip: float = 0.02) -> np.ndarray:
    """White page with ``n_shapes`` filled black ellipses or thick strokes
    (size parameter r uniform in [rmin, rmax] px), then every pixel flipped
    independently with probability ``flip`` (salt-and-pepper noise)."""
    g = rng(seed)
    img = np.ones((h, w), dtype=np.uint8)
    yy, xx = np.mgrid[0:h, 0:w]
    canvas = _Canvas(w, h)
    for _ in range(n_shapes):
        r = int(g.integers(rmin, rmax + 1))
        cx, cy = g.uniform(0, w), g.uniform(0, h)
        if g.random() < 0.5:
            a = float(r)
            b = float(g.integers(rmin, r + 1))
            th = g.uniform(0, math.pi)
            c, s = math.cos(th), math.sin(th)
            u = (xx - cx) * c + (yy - cy) * s
            v = -(xx - cx) * s + (yy - cy) * c
            img[(u / a) ** 2 + (v / b) ** 2 <= 1.0] = BLACK
        else:
            th = g.uniform(0, 2 * math.pi)
            length = g.uniform(2 * r, 4 * r)
            bx, by = cx + length * math.cos(th), cy + length * math.sin(th)
            canvas.capsule(cx, cy, bx, by, max(1.0, r / 4.0))
    img &= canvas.render()
    if flip > 0:
        img ^= (g.random((h, w)) < flip).astype(np.uint8)
    return img


def bernoulli(w: int, h: int, p_black: float, seed: int) -> np.ndarray:
    """Every pixel black independently with probability ``p_black``."""
    g = rng(seed)
    return (g.random((h, w)) >= p_black).astype(np.uint8)


def bernoulli_half_packed(w: int, h: int, seed: int,
                          stride_words: int | None = None) -> np.ndarray:
    """Bernoulli(0.5) image generated directly in packed form (uniform random
    words), for images too large to draw byte by byte.  Padding bits and
    padding words carry random garbage."""
    nw = words_per_row(w)
    stride_words = nw if stride_words is None else stride_words
    g = rng(seed)
    return g.integers(0, 2 ** 32, size=(h, stride_words),
                      dtype=np.uint64).astype(np.uint32)


def blocks_packed(w: int, h: int, seed: int, block: int = 64,
                  p_black: float = 0.5,
                  stride_words: int | None = None) -> np.ndarray:
    """Solid ``block`` x ``block`` squares, each black with ``p_black``,
    in packed form.  ``block`` must be a multiple of 32 and divide ``w``."""
    if block % 32 or w % block:
        raise ValueError("blocks_packed wants block % 32 == 0 and w % block == 0")
    nw = words_per_row(w)
    stride_words = nw if stride_words is None else stride_words
    g = rng(seed)
    nbx, nby = w // block, (h + block - 1) // block
    black = g.random((nby, nbx)) < p_black
    word = np.where(black, np.uint32(0), np.uint32(0xFFFFFFFF))
    row_words = np.repeat(word, block // 32, axis=1)          # [nby, nw]
    out = np.zeros((h, stride_words), dtype=np.uint32)
    out[:, :nw] = np.repeat(row_words, block, axis=0)[:h]
    return out


def strokes(w: int, h: int, n_lines: int, seed: int, width_lo: int = 1,
            width_hi: int = 6, verts_lo: int = 2, verts_hi: int = 8) -> np.ndarray:
    """White image with ``n_lines`` black polylines; each has U{verts_lo..
    verts_hi} vertices uniform in the image and width U{width_lo..width_hi}."""
    g = rng(seed)
    canvas = _Canvas(w, h)
    for _ in range(n_lines):
        nv = int(g.integers(verts_lo, verts_hi + 1))
        width = int(g.integers(width_lo, width_hi + 1))
        pts = np.stack([g.uniform(0, w, nv), g.uniform(0, h, nv)], axis=1)
        canvas.polyline(pts, width / 2.0)
    return canvas.render()


def glyph_cell(g: np.random.Generator, canvas: _Canvas, x0: float, y0: float,
               size: float = 48.0):
    """A glyph-like blob: 2-4 strokes of width 2-5 inside a size x size cell."""
    for _ in range(int(g.integers(2, 5))):
        nv = int(g.integers(2, 4))
        width = int(g.integers(2, 6))
        pts = np.stack([x0 + g.uniform(0.15, 0.85, nv) * size,
                        y0 + g.uniform(0.15, 0.85, nv) * size], axis=1)
        canvas.polyline(pts, width / 2.0)


def glyph(seed: int, size: int = 48) -> np.ndarray:
    g = rng(seed)
    canvas = _Canvas(size, size)
    glyph_cell(g, canvas, 0.0, 0.0, float(size))
    return canvas.render()


def page(seed: int, w: int = 2480, h: int = 3508, cell: int = 48,
         margin: int = 120, line_gap: int = 16) -> np.ndarray:
    """A text page: lines of ``cell``-px glyph blobs inside the margins."""
    g = rng(seed)
    canvas = _Canvas(w, h)
    y = float(margin)
    while y + cell < h - margin:
        x = float(margin)
        while x + cell < w - margin:
            if g.random() < 0.85:          # word gaps
                glyph_cell(g, canvas, x, y, float(cell))
            x += cell * g.uniform(0.8, 1.1)
        y += cell + line_gap
    return canvas.render()


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclass
class Image:
    """One packed image plus the facts a caller needs about it."""
    words: np.ndarray          # uint32[h, stride_words]
    w: int
    h: int
    boundary: int = 0          # 0 = outside is white, 1 = outside is black

    @property
    def stride_words(self) -> int:
        return int(self.words.shape[1])

    @property
    def pixels(self) -> int:
        return self.w * self.h

    @property
    def packed_bytes(self) -> int:
        return self.h * self.stride_words * 4


def batch_shapes(seed: int, n: int = 4096, lo: int = 16, hi: int = 4096):
    """``n`` (w, h) pairs, each drawn independently log-uniform on [lo, hi]."""
    g = rng(seed)
    ws = np.exp(g.uniform(math.log(lo), math.log(hi), n))
    hs = np.exp(g.uniform(math.log(lo), math.log(hi), n))
    ws = np.clip(np.rint(ws), lo, hi).astype(np.int64)
    hs = np.clip(np.rint(hs), lo, hi).astype(np.int64)
    return list(zip(ws.tolist(), hs.tolist()))


def batch_stride(w: int, pad16: bool = True) -> int:
    nw = words_per_row(w)
    return round_up(nw, 4) if pad16 else nw


def batch_image(seed: int, index: int, w: int, h: int, pad16: bool = True,
                ref_area: int = 4096 * 4096, ref_lines: int = 200) -> Image:
    """Image ``index`` of the uneven glyph-stroke batch: max(1, round(
    ref_lines * w * h / ref_area)) polylines of width U{1..6}."""
    n_lines = max(1, int(round(ref_lines * w * h / ref_area)))
    img = strokes(w, h, n_lines, seed * 1_000_003 + index)
    words = pack(img, batch_stride(w, pad16), pad="random",
                 seed=seed * 7919 + index)
    return Image(words, w, h)


def _batch_part(args):
    seed, items, pad16 = args
    return [batch_image(seed, i, w, h, pad16) for i, w, h in items]


def batch(seed: int, n: int = 4096, lo: int = 16, hi: int = 4096,
          pad16: bool = True, workers: int = 1) -> list[Image]:
    """The uneven glyph-stroke batch.  ``workers > 1`` draws it in a pool of
    spawned processes (safe to start after CUDA is initialised); the result
    does not depend on the worker count."""
    items = [(i, w, h) for i, (w, h) in enumerate(batch_shapes(seed, n, lo, hi))]
    if workers <= 1 or n < 64:
        return _batch_part((seed, items, pad16))
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    chunks = [items[k::workers * 4] for k in range(workers * 4)]
    out: list = [None] * n
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        for chunk, imgs in zip(chunks, ex.map(_batch_part,
                                              [(seed, c, pad16) for c in chunks])):
            for (i, _, _), im in zip(chunk, imgs):
                out[i] = im
    return out


SERVE_MIX = ((48, 48, 0.70), (1024, 1024, 0.25), (2480, 3508, 0.05))


def serve_trace(seed: int, n_requests: int, rate_hz: float):
    """Poisson arrivals: returns (arrival times in s, size-class indices)."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    probs = np.array([p for _, _, p in SERVE_MIX])
    cls = g.choice(len(SERVE_MIX), size=n_requests, p=probs / probs.sum())
    return t, cls


def serve_pool(seed: int, per_class=(16, 4, 2)) -> list[list[Image]]:
    """A few images of each serving size class; requests reuse them."""
    out = []
    for ci, ((w, h, _), k) in enumerate(zip(SERVE_MIX, per_class)):
        imgs = []
        for j in range(k):
            s = seed * 10_007 + ci * 101 + j
            if (w, h) == (48, 48):
                im = glyph(s, 48)
            elif (w, h) == (2480, 3508):
                im = page(s, w, h)
            else:
                im = strokes(w, h, max(1, int(round(200 * w * h / 4096 ** 2))) * 8, s)
            imgs.append(Image(pack(im, words_per_row(w)), w, h))
        out.append(imgs)
    return out

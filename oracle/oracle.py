"""CPU oracle for edge detection of binary images by the method of masks.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only code allowed to import this
module.  It shares no code with the CUDA library and never imports it.

Two independent statements of what the path computes, both on byte images
``u8[h, w]`` with 0 = black and 1 = white (Section 2):

* ``edges``/``fundamental``/``mask``/``end_points`` call the plain C loops
  in ``me_oracle.c`` (Sections 1, 3 and 4; Fig. 1 numbering).
* ``definition_*`` evaluate the binary edge-point definition of Section 1
  with BOTH of its clauses -- a black point with at least one white
  4-neighbour, or a black point with at most one black 8-neighbour -- by
  brute force, in Python loops for tiny inputs and with numpy over stacks
  of images.  They pin the C oracle: the paper asserts (Section 1) that the
  second clause adds no edge point beyond the first, so both must agree.

A neighbour outside the image takes the boundary colour: ``boundary=0``
reads outside pixels as white (the default reading), ``boundary=1`` as black.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "me_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libme_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/_build``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-Wextra",
                               "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.c_void_p
            i32 = ctypes.c_int
            lib.me_oracle_mask.argtypes = [u8p, i32, i32, u8p]
            lib.me_oracle_edges.argtypes = [u8p, i32, i32, i32, u8p]
            lib.me_oracle_edges_many.argtypes = [u8p, i32, i32, i32, i32, u8p]
            lib.me_oracle_fundamental.argtypes = [u8p, i32, i32, i32, u8p, u8p,
                                                  u8p, u8p]
            lib.me_oracle_end_points.argtypes = [u8p, i32, i32, i32, u8p]
            lib.me_oracle_threshold.argtypes = [u8p, i32, i32, i32, i32, u8p]
            for f in (lib.me_oracle_mask, lib.me_oracle_edges,
                      lib.me_oracle_edges_many, lib.me_oracle_fundamental,
                      lib.me_oracle_end_points, lib.me_oracle_threshold):
                f.restype = i32
            _lib = lib
    return _lib


def _as_img(img) -> np.ndarray:
    a = np.ascontiguousarray(img, dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("expected a 2-D byte image")
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int):
    if rc != 0:
        raise ValueError("oracle rejected its arguments")


def mask(img) -> np.ndarray:
    """Section 3: the negative image (1 where the image is black)."""
    a = _as_img(img)
    out = np.empty_like(a)
    _check(_load().me_oracle_mask(_ptr(a), a.shape[1], a.shape[0], _ptr(out)))
    return out


def edges(img, boundary: int = 0) -> np.ndarray:
    """Section 1, Edge(p) per pixel: 1 marks an edge point."""
    a = _as_img(img)
    out = np.empty_like(a)
    _check(_load().me_oracle_edges(_ptr(a), a.shape[1], a.shape[0],
                                   int(boundary), _ptr(out)))
    return out


def edges_many(imgs, boundary: int = 0) -> np.ndarray:
    """``edges`` over a stack ``u8[n, h, w]`` of same-sized images."""
    a = np.ascontiguousarray(imgs, dtype=np.uint8)
    n, h, w = a.shape
    out = np.empty_like(a)
    _check(_load().me_oracle_edges_many(_ptr(a), n, w, h, int(boundary),
                                        _ptr(out)))
    return out


def fundamental(img, boundary: int = 0):
    """Section 4: the (left, right, up, down) fundamental edges."""
    a = _as_img(img)
    outs = [np.empty_like(a) for _ in range(4)]
    _check(_load().me_oracle_fundamental(_ptr(a), a.shape[1], a.shape[0],
                                         int(boundary), *[_ptr(o) for o in outs]))
    return tuple(outs)


def end_points(img, boundary: int = 0) -> np.ndarray:
    """Section 1, second clause alone: black points with at most one black
    8-neighbour."""
    a = _as_img(img)
    out = np.empty_like(a)
    _check(_load().me_oracle_end_points(_ptr(a), a.shape[1], a.shape[0],
                                        int(boundary), _ptr(out)))
    return out


def threshold(grey, t: int) -> np.ndarray:
    """Section 7's grey photograph made binary (the paper names no rule):
    1 (white) where grey >= t, 0 (black) below."""
    a = np.ascontiguousarray(grey, dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("expected a 2-D grey image")
    out = np.empty_like(a)
    _check(_load().me_oracle_threshold(_ptr(a), a.shape[1], a.shape[0], a.shape[1],
                                       int(t), _ptr(out)))
    return out


def otsu_threshold(grey) -> int:
    """Otsu's rule for the threshold of Section 7's grey photograph (the paper
    names none; N. Otsu, "A threshold selection method from gray-level
    histograms", IEEE Trans. SMC 9(1), 1979): the t in 1..255 whose classes
    grey < t and grey >= t have the largest between-class variance
    w0 w1 (mu1 - mu0)^2.  With N pixels, S the sum of all grey values, n0
    pixels and s0 grey sum below t, that variance is
    (S n0 - s0 N)^2 / (N^2 n0 (N - n0)); N^2 is common to every t, so
    D(t) = x^2 / (n0 (N - n0)), x = S n0 - s0 N, is compared, for t with
    0 < n0 < N.  The comparison is taken in IEEE double arithmetic in exactly
    this order (x = S*n0 - s0*N, then x*x / (n0 * (N - n0)), every operand an
    exact integer converted to double), the first largest t wins, and an
    image of one grey value v takes t = v (every pixel white)."""
    a = np.asarray(grey, dtype=np.uint8)
    if a.size == 0:
        raise ValueError("empty image")
    hist = np.bincount(a.ravel(), minlength=256)
    N = int(a.size)
    S = sum(i * int(hist[i]) for i in range(256))
    best_t, best_d = None, None
    n0 = s0 = 0
    for t in range(1, 256):
        n0 += int(hist[t - 1])
        s0 += (t - 1) * int(hist[t - 1])
        if n0 == 0 or n0 == N:
            continue
        x = float(S) * float(n0) - float(s0) * float(N)
        d = (x * x) / (float(n0) * float(N - n0))
        if best_d is None or d > best_d:
            best_t, best_d = t, d
    if best_t is None:
        return int(a.flat[0])
    return best_t


# ----------------------------------------------------------------------------
# brute force over the full definition of Section 1
# ----------------------------------------------------------------------------

# Fig. 1: neighbour k sits at (dx, dy) from P, with y growing downwards.
FIG1_OFFSETS = {1: (1, -1), 2: (0, -1), 3: (-1, -1), 4: (-1, 0),
                5: (-1, 1), 6: (0, 1), 7: (1, 1), 8: (1, 0)}
FOUR_NEIGHBOURS = (2, 4, 6, 8)


def definition_point(img, x: int, y: int, boundary: int = 0) -> int:
    """Both clauses of the Section 1 definition at one pixel, in plain Python."""
    h, w = len(img), len(img[0])
    outside = 0 if boundary else 1

    def colour(i, j):
        if 0 <= i < w and 0 <= j < h:
            return 1 if img[j][i] else 0
        return outside

    if colour(x, y) != 0:
        return 0
    nb = {k: colour(x + dx, y + dy) for k, (dx, dy) in FIG1_OFFSETS.items()}
    white_4 = any(nb[k] == 1 for k in FOUR_NEIGHBOURS)
    black_8 = sum(1 for k in nb if nb[k] == 0)
    return 1 if (white_4 or black_8 <= 1) else 0


def definition_edges_loops(img, boundary: int = 0) -> np.ndarray:
    a = _as_img(img)
    h, w = a.shape
    rows = a.tolist()
    return np.array([[definition_point(rows, x, y, boundary) for x in range(w)]
                     for y in range(h)], dtype=np.uint8).reshape(h, w)


def definition_edges_stack(imgs, boundary: int = 0) -> np.ndarray:
    """Both clauses of the Section 1 definition over a stack ``u8[n, h, w]``,
    evaluated by explicit neighbour enumeration on boundary-padded copies."""
    a = (np.asarray(imgs) != 0).astype(np.int16)
    n, h, w = a.shape
    outside = 0 if boundary else 1
    padded = np.full((n, h + 2, w + 2), outside, dtype=np.int16)
    padded[:, 1:h + 1, 1:w + 1] = a

    def nbr(k):
        dx, dy = FIG1_OFFSETS[k]
        return padded[:, 1 + dy:1 + dy + h, 1 + dx:1 + dx + w]

    black = a == 0
    white_4 = np.zeros_like(black)
    for k in FOUR_NEIGHBOURS:
        white_4 |= nbr(k) == 1
    black_8 = np.zeros(a.shape, dtype=np.int16)
    for k in FIG1_OFFSETS:
        black_8 += (nbr(k) == 0)
    return (black & (white_4 | (black_8 <= 1))).astype(np.uint8)

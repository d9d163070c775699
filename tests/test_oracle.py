"""Pins for the CPU oracle: it is checked against things other than itself.

* brute force over the full two-clause definition of Section 1 (every 3x3
  neighbourhood, every image with w*h <= 16, random images);
* the four edge-point types of Fig. 2 (golden fixture);
* hand-built cases and invariants (edge = black AND NOT erode4(black) with
  scipy's binary erosion, flips, transposes, all-white, all-black);
* the end-point map (second clause) against a scipy neighbour count;
* Otsu's threshold: a closed form for two grey levels, constant images, the
  within-class form computed from the class pixels, shift and inversion;
* planted mistakes in a copy of the C source must fail at least one pin.
"""
import ctypes
import itertools
import os
import re
import subprocess

import numpy as np
import pytest
from scipy import ndimage

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")
CROSS = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]], dtype=bool)


def rand_img(seed, h, w, p_black=0.5):
    g = np.random.default_rng(seed)
    return (g.random((h, w)) >= p_black).astype(np.uint8)


def all_images(w, h):
    """Every binary image of size h x w, as u8[2**(w*h), h, w]."""
    n = w * h
    codes = np.arange(2 ** n, dtype=np.int64)
    bits = (codes[:, None] >> np.arange(n)[None, :]) & 1
    return bits.astype(np.uint8).reshape(-1, h, w)


# ---------------------------------------------------------------------------
# brute force over the full definition
# ---------------------------------------------------------------------------

def test_lemma_every_3x3_neighbourhood():
    """Section 1 claims the two-clause definition reduces to the four
    edge-point types: a black point with <= 1 black 8-neighbour always has a
    white 4-neighbour.  Check it, and the oracle, on all 512 neighbourhoods."""
    extra = 0
    for code in range(512):
        img = np.array([(code >> k) & 1 for k in range(9)],
                       dtype=np.uint8).reshape(3, 3)
        d = O.definition_point(img.tolist(), 1, 1)
        for b in (0, 1):
            assert O.edges(img, b)[1, 1] == d, (code, b)
        if img[1, 1] == 0:
            nb = [img[1 + dy, 1 + dx] for dx, dy in O.FIG1_OFFSETS.values()]
            four = [img[1 + O.FIG1_OFFSETS[k][1], 1 + O.FIG1_OFFSETS[k][0]]
                    for k in O.FOUR_NEIGHBOURS]
            if nb.count(0) <= 1 and not any(four):
                extra += 1
    assert extra == 0


@pytest.mark.parametrize("boundary", [0, 1])
def test_every_image_up_to_16_pixels(boundary):
    for w in range(1, 17):
        for h in range(1, 16 // w + 1):
            imgs = all_images(w, h)
            got = O.edges_many(imgs, boundary)
            want = O.definition_edges_stack(imgs, boundary)
            assert np.array_equal(got, want), (w, h, boundary)


@pytest.mark.parametrize("seed", range(4))
def test_random_small_images_against_python_loops(seed):
    g = np.random.default_rng(100 + seed)
    h, w = int(g.integers(1, 12)), int(g.integers(1, 12))
    img = rand_img(seed, h, w, p_black=float(g.uniform(0.2, 0.9)))
    for b in (0, 1):
        assert np.array_equal(O.edges(img, b), O.definition_edges_loops(img, b))


@pytest.mark.parametrize("p_black", [0.1, 0.5, 0.9])
def test_random_64x64_against_definition(p_black):
    imgs = np.stack([rand_img(s, 64, 64, p_black) for s in range(8)])
    for b in (0, 1):
        assert np.array_equal(O.edges_many(imgs, b),
                              O.definition_edges_stack(imgs, b))


# ---------------------------------------------------------------------------
# Fig. 2: the four types of edge point
# ---------------------------------------------------------------------------

def load_fig2():
    cases = []
    with open(os.path.join(GOLDEN, "fig2_edge_types.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            panel, name, *rows = line.split()
            cases.append((panel, name, rows))
    return cases


FUND_INDEX = {"left": 0, "right": 1, "up": 2, "down": 3}


@pytest.mark.parametrize("panel,name,rows", load_fig2())
def test_fig2_edge_types(panel, name, rows):
    free = [(r, c) for r in range(3) for c in range(3) if rows[r][c] == "x"]
    for fill in itertools.product((0, 1), repeat=len(free)):
        patch = np.zeros((3, 3), dtype=np.uint8)
        for r in range(3):
            for c in range(3):
                if rows[r][c] == "1":
                    patch[r, c] = 1
        for (r, c), v in zip(free, fill):
            patch[r, c] = v
        # embed in a black field with a black outside, so nothing else is white
        field = np.zeros((7, 7), dtype=np.uint8)
        field[2:5, 2:5] = patch
        fund = O.fundamental(field, boundary=1)
        assert O.edges(field, 1)[3, 3] == 1
        assert fund[FUND_INDEX[name]][3, 3] == 1
        if not any(fill):
            fired = [k for k, f in FUND_INDEX.items() if fund[f][3, 3]]
            assert fired == [name]


# ---------------------------------------------------------------------------
# hand-built cases
# ---------------------------------------------------------------------------

def test_isolated_black_pixel_fires_all_four():
    img = np.ones((5, 5), dtype=np.uint8)
    img[2, 2] = 0
    fund = O.fundamental(img)
    assert all(f[2, 2] == 1 for f in fund)
    assert O.edges(img).sum() == 1 and O.end_points(img)[2, 2] == 1


def test_solid_block_interior_is_not_edge():
    img = np.ones((9, 9), dtype=np.uint8)
    img[2:7, 2:7] = 0
    e = O.edges(img)
    assert e[3:6, 3:6].sum() == 0
    ring = np.zeros_like(e)
    ring[2:7, 2:7] = 1
    ring[3:6, 3:6] = 0
    assert np.array_equal(e, ring)


def test_horizontal_line_fires_up_and_down_only_inside():
    img = np.ones((5, 9), dtype=np.uint8)
    img[2, 1:8] = 0
    left, right, up, down = O.fundamental(img)
    assert up[2, 1:8].all() and down[2, 1:8].all()
    assert left[2, 1] == 1 and left[2, 2:8].sum() == 0
    assert right[2, 7] == 1 and right[2, 1:7].sum() == 0


def test_diagonal_only_white_neighbour_is_not_edge():
    img = np.zeros((5, 5), dtype=np.uint8)
    img[1, 3] = 1                    # neighbour 1 of (2, 2) is white
    assert O.edges(img, 1)[2, 2] == 0


def test_one_pixel_wide_images():
    col = np.zeros((7, 1), dtype=np.uint8)
    assert O.edges(col, 0).all()                 # white outside
    assert O.edges(col, 1).sum() == 0            # black outside
    row = np.array([[0, 1, 0, 0, 0]], dtype=np.uint8)
    assert O.edges(row, 0).tolist() == [[1, 0, 1, 1, 1]]
    assert O.edges(row, 1).tolist() == [[1, 0, 1, 0, 0]]


def test_empty_image_and_bad_args():
    assert O.edges(np.zeros((0, 5), dtype=np.uint8)).shape == (0, 5)
    with pytest.raises(ValueError):
        O.edges(np.zeros((3, 3), dtype=np.uint8), boundary=2)


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_invariants_random(seed):
    g = np.random.default_rng(seed)
    h, w = int(g.integers(1, 90)), int(g.integers(1, 90))
    img = rand_img(seed, h, w, float(g.uniform(0.05, 0.95)))
    black = img == 0
    for b in (0, 1):
        e = O.edges(img, b)
        assert not (e.astype(bool) & ~black).any()             # edge within black
        assert e.sum() <= black.sum()
        eroded = ndimage.binary_erosion(black, structure=CROSS,
                                        border_value=1 if b else 0)
        assert np.array_equal(e.astype(bool), black & ~eroded)
        fl, fr, fu, fd = O.fundamental(img, b)
        assert np.array_equal(e, fl | fr | fu | fd)
        assert np.array_equal(O.edges(img[:, ::-1], b), e[:, ::-1])
        assert np.array_equal(O.edges(img[::-1, :], b), e[::-1, :])
        assert np.array_equal(O.edges(img.T.copy(), b), e.T)
        # a horizontal flip swaps the left and right edges
        fl2, fr2, fu2, fd2 = O.fundamental(img[:, ::-1], b)
        assert np.array_equal(fl2, fr[:, ::-1]) and np.array_equal(fr2, fl[:, ::-1])
        assert np.array_equal(fu2, fu[:, ::-1])
        fl3, fr3, fu3, fd3 = O.fundamental(img[::-1, :], b)
        assert np.array_equal(fu3, fd[::-1, :]) and np.array_equal(fd3, fu[::-1, :])
    assert np.array_equal(O.mask(img), 1 - img)


def test_all_white_and_all_black():
    white = np.ones((6, 11), dtype=np.uint8)
    assert O.edges(white, 0).sum() == 0 and O.edges(white, 1).sum() == 0
    black = np.zeros((6, 11), dtype=np.uint8)
    ring = np.ones_like(black)
    ring[1:-1, 1:-1] = 0
    assert np.array_equal(O.edges(black, 0), ring)
    assert O.edges(black, 1).sum() == 0


def test_shift_direction_of_left_edge():
    """Section 4: the left edge is the mask ANDed with the image moved one
    pixel to the right, i.e. black pixels whose LEFT neighbour is white."""
    img = np.array([[1, 0, 0, 1]], dtype=np.uint8)
    left, right, _, _ = O.fundamental(img, boundary=1)
    assert left.tolist() == [[0, 1, 0, 0]]
    assert right.tolist() == [[0, 0, 1, 0]]
    moved_right = np.concatenate([[[0]], img[:, :-1]], axis=1)  # outside black
    assert np.array_equal(left, (1 - img) & moved_right)


# ---------------------------------------------------------------------------
# second clause alone: end points
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_end_points_against_neighbour_count(seed):
    img = rand_img(seed, 40, 33, p_black=0.3 + 0.15 * seed)
    kernel = np.ones((3, 3), dtype=np.int32)
    kernel[1, 1] = 0
    for b in (0, 1):
        black = (img == 0).astype(np.int32)
        count = ndimage.convolve(black, kernel, mode="constant", cval=b)
        want = (black == 1) & (count <= 1)
        assert np.array_equal(O.end_points(img, b).astype(bool), want)
        # and the second clause never adds a point the first misses
        assert not (O.end_points(img, b) & (1 - O.edges(img, b))).any()


def test_end_points_hand_cases():
    img = np.ones((5, 9), dtype=np.uint8)
    img[2, 1:8] = 0                      # a one-pixel line
    ep = O.end_points(img)
    assert ep[2].tolist() == [0, 1, 0, 0, 0, 0, 0, 1, 0]


# ---------------------------------------------------------------------------
# thresholding ahead of the method (Section 7)
# ---------------------------------------------------------------------------

def test_threshold_extremes_and_hand_case():
    grey = np.array([[0, 127, 128, 255]], dtype=np.uint8)
    assert O.threshold(grey, 128).tolist() == [[0, 0, 1, 1]]
    assert O.threshold(grey, 0).tolist() == [[1, 1, 1, 1]]
    assert O.threshold(grey, 256).tolist() == [[0, 0, 0, 0]]
    assert O.threshold(grey, 255).tolist() == [[0, 0, 0, 1]]


@pytest.mark.parametrize("seed", range(3))
def test_threshold_counts_match_the_histogram(seed):
    """White pixels at threshold t = the histogram's mass at t and above,
    for every t; whites only shrink as t grows."""
    g = np.random.default_rng(seed)
    grey = g.integers(0, 256, (37, 53), dtype=np.uint8)
    tail = np.cumsum(np.bincount(grey.ravel(), minlength=256)[::-1])[::-1]
    prev = None
    for t in range(0, 257):
        b = O.threshold(grey, t)
        assert b.sum() == (tail[t] if t < 256 else 0)
        if prev is not None:
            assert not (b & (1 - prev)).any()
        prev = b


# ---------------------------------------------------------------------------
# Otsu's threshold for Section 7's photograph (the paper names no rule)
# ---------------------------------------------------------------------------

def mixture(seed, h, w, mus, sigmas, weights):
    """Grey pixels drawn from a mixture of clipped normals."""
    g = np.random.default_rng(seed)
    k = g.choice(len(mus), size=(h, w), p=weights)
    v = g.normal(np.asarray(mus)[k], np.asarray(sigmas)[k])
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


def within_class_argmin(grey):
    """Otsu's criterion in its other form, from the pixels themselves: the t
    in 1..255 with the least within-class variance w0 var0 + w1 var1 of the
    classes grey < t and grey >= t (Otsu 1979: within- plus between-class
    variance is the total variance, so the least of one is the largest of
    the other), each class's variance by numpy's var on its pixels.  Returns
    t and the relative margin to the best t with another split."""
    v = grey.ravel().astype(np.float64)
    best = {}
    for t in range(1, 256):
        lo, hi = v[v < t], v[v >= t]
        if lo.size == 0 or hi.size == 0:
            continue
        score = (lo.size * lo.var() + hi.size * hi.var()) / v.size
        key = lo.size                       # thresholds with the same split tie
        if key not in best or score < best[key][0]:
            best[key] = (score, t)
    ranked = sorted(best.values())
    (s1, t1), (s2, _) = ranked[0], ranked[1]
    return t1, (s2 - s1) / max(s1, 1e-300)


MIXTURES = [
    (0, 48, 64, (60, 180), (15, 20), (0.5, 0.5)),
    (1, 40, 70, (40, 140), (10, 30), (0.7, 0.3)),
    (2, 64, 64, (100, 130, 220), (12, 8, 10), (0.4, 0.3, 0.3)),
    (3, 33, 97, (20, 235), (5, 5), (0.9, 0.1)),
    (4, 50, 50, (128,), (40,), (1.0,)),
]


def otsu_pins(otsu):
    """Every check that pins an Otsu threshold function."""
    # two grey levels a < b: every t in a+1..b makes the same two classes,
    # and the first of the tied t wins
    for a, b, na, nb in ((50, 200, 10, 30), (0, 255, 1, 1), (7, 8, 5, 100), (100, 101, 3, 2)):
        grey = np.array([[a] * na + [b] * nb], dtype=np.uint8)
        assert otsu(grey) == a + 1, (a, b, na, nb)
    # one grey value: every pixel white
    for v in (0, 1, 77, 255):
        assert otsu(np.full((3, 5), v, dtype=np.uint8)) == v
    # the within-class form, computed from the class pixels
    for seed, h, w, mus, sig, wts in MIXTURES:
        grey = mixture(seed, h, w, mus, sig, wts)
        t_ref, gap = within_class_argmin(grey)
        assert gap > 1e-9, "ambiguous case"
        assert otsu(grey) == t_ref, (seed, otsu(grey), t_ref)
    # shifting every grey value by c shifts t by c; inverting the grey
    # scale (255 - grey) swaps the two classes, so the split is the same
    # (t itself may move within a run of empty bins: the first t wins)
    for seed, h, w, mus, sig, wts in MIXTURES[:3]:
        grey = np.clip(mixture(seed, h, w, mus, sig, wts), 10, 200)
        t = otsu(grey)
        assert otsu(grey + 40) == t + 40
        inv = 255 - grey
        assert np.array_equal(grey >= t, inv < otsu(inv))


def test_otsu_pins():
    otsu_pins(O.otsu_threshold)


OTSU_MUTATIONS = {
    "grey sum off by one": ("s0 += (t - 1) * int(hist[t - 1])", "s0 += t * int(hist[t - 1])"),
    "one class size": ("(float(n0) * float(N - n0))", "(float(n0) * float(N))"),
    "square dropped": ("d = (x * x) /", "d = abs(x) /"),
    "last tie wins": ("d > best_d", "d >= best_d"),
}


@pytest.mark.parametrize("name", sorted(OTSU_MUTATIONS))
def test_otsu_planted_mistake_is_caught(name):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(O.otsu_threshold))
    old, new = OTSU_MUTATIONS[name]
    assert old in src
    ns = {"np": np}
    exec(src.replace(old, new), ns)
    with pytest.raises(AssertionError):
        otsu_pins(ns["otsu_threshold"])


# ---------------------------------------------------------------------------
# planted mistakes must fail a pin
# ---------------------------------------------------------------------------

MUTATIONS = {
    "dropped down term": ("(n2 || n4 || n6 || n8)", "(n2 || n4 || n8)"),
    "wrong left index": ("int n4 = pixel(img, w, h, x - 1, y, o);",
                         "int n4 = pixel(img, w, h, x + 1, y, o);"),
    "outside colour flipped": ("return boundary ? 0 : 1;", "return boundary ? 1 : 0;"),
    "transposed store": ("out[(size_t)y * w + x] = (uint8_t)(!p &&",
                         "out[(size_t)x * h + y] = (uint8_t)(!p &&"),
    "mask not inverted": ("(uint8_t)(!p && (n2", "(uint8_t)(p && (n2"),
    "left/right swapped": ("left[i]  = (uint8_t)(m && pixel(img, w, h, x - 1, y, o));",
                           "left[i]  = (uint8_t)(m && pixel(img, w, h, x + 1, y, o));"),
    "threshold strict": ("(int)grey[(size_t)y * pitch + x] >= t", "(int)grey[(size_t)y * pitch + x] > t"),
    "threshold pitch ignored": ("grey[(size_t)y * pitch + x]", "grey[(size_t)y * w + x]"),
}


def _compile_mutant(tmp_path, old, new):
    src = open(os.path.join(ROOT, "oracle", "me_oracle.c")).read()
    assert old in src, old
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", str(so), str(path)])
    lib = ctypes.CDLL(str(so))
    return lib


def _pins_pass(lib):
    """The cheap subset of the pins above, run against a loaded library."""
    def edges(img, b):
        a = np.ascontiguousarray(img, dtype=np.uint8)
        out = np.zeros_like(a)
        lib.me_oracle_edges(ctypes.c_void_p(a.ctypes.data), a.shape[1], a.shape[0],
                            b, ctypes.c_void_p(out.ctypes.data))
        return out

    def left(img, b):
        a = np.ascontiguousarray(img, dtype=np.uint8)
        outs = [np.zeros_like(a) for _ in range(4)]
        lib.me_oracle_fundamental(ctypes.c_void_p(a.ctypes.data), a.shape[1],
                                  a.shape[0], b,
                                  *[ctypes.c_void_p(o.ctypes.data) for o in outs])
        return outs[0]

    for code in range(512):
        img = np.array([(code >> k) & 1 for k in range(9)], np.uint8).reshape(3, 3)
        if edges(img, 0)[1, 1] != O.definition_point(img.tolist(), 1, 1):
            return False
    for seed in range(3):
        img = rand_img(seed, 7, 12, 0.6)
        for b in (0, 1):
            if not np.array_equal(edges(img, b), O.definition_edges_stack(img[None], b)[0]):
                return False
    img = np.array([[1, 0, 0, 1]], dtype=np.uint8)
    if left(img, 1).tolist() != [[0, 1, 0, 0]]:
        return False
    # thresholding: the hand case, and a pitch wider than the row
    grey = np.array([[0, 127, 128, 255, 9, 9], [200, 3, 128, 127, 9, 9]], dtype=np.uint8)
    out = np.zeros((2, 4), dtype=np.uint8)
    lib.me_oracle_threshold(ctypes.c_void_p(grey.ctypes.data), 4, 2, 6, 128,
                            ctypes.c_void_p(out.ctypes.data))
    if out.tolist() != [[0, 0, 1, 1], [1, 0, 1, 0]]:
        return False
    return True


def test_pins_pass_on_real_oracle(tmp_path):
    lib = ctypes.CDLL(O.build())
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    assert not _pins_pass(_compile_mutant(tmp_path, old, new)), name

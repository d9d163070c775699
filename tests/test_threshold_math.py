"""The packed compare that the grey front end uses, checked on the CPU for
every threshold: with c = 256 - t in every byte, grey >= t is the majority
of a's bit 7, c's bit 7 and the carry out of the low seven bits of a + c
(one add per four bytes, never crossing a byte); a multiply by 0x00204081
moves the four carries to bits 28..31, and appending nibbles from the top
builds the word with bit k = byte k.  The arithmetic is restated here in
numpy (32-bit wrap-around) and compared with the plain byte comparison
grey >= t; the GPU parity tests check that the kernel computes it."""
import numpy as np
import pytest

M7 = np.uint32(0x7F7F7F7F)
H = np.uint32(0x80808080)


def carries(a, t):
    """The carry word of four grey bytes a (uint32) for threshold t."""
    c4 = np.uint32((256 - t) * 0x01010101)
    s = (a & M7) + (c4 & M7)                     # never carries across a byte
    if t <= 128:                                 # c's bit 7 set: majority = a7 | s7
        return (a | s) & H
    return a & s & H                             # c's bit 7 clear: majority = a7 & s7


def gather(carry):
    """Bits 7, 15, 23, 31 of carry to bits 0..3 (through bits 28..31 of the
    32-bit product)."""
    with np.errstate(over="ignore"):             # the product wraps at 32 bits
        return (np.uint32(carry) * np.uint32(0x00204081)) >> np.uint32(28)


def pack32(grey32, t):
    """32 grey bytes (uint8[..., 32]) to one word, nibbles appended from the
    top as the kernel's funnel shift does: out = (out << 4) | nibble."""
    words = grey32.reshape(grey32.shape[:-1] + (8, 4)).astype(np.uint32)
    words = words[..., 0] | (words[..., 1] << 8) | (words[..., 2] << 16) | (words[..., 3] << 24)
    out = np.zeros(grey32.shape[:-1], dtype=np.uint32)
    for k in range(7, -1, -1):
        out = ((out << np.uint32(4)) | gather(carries(words[..., k], t))) & np.uint32(0xFFFFFFFF)
    return out


def test_gather_every_carry_pattern():
    for p in range(16):
        carry = np.uint32(sum(((p >> b) & 1) << (8 * b + 7) for b in range(4)))
        assert int(gather(carry)) == p, p


@pytest.mark.parametrize("t", range(1, 256))
def test_every_byte_value_in_every_position(t):
    """All 256 values of one byte with the other three bytes random (so a
    carry leaking across bytes would show), for every threshold."""
    g = np.random.default_rng(t)
    for pos in range(4):
        others = g.integers(0, 256, size=(256, 4), dtype=np.uint32)
        others[:, pos] = np.arange(256, dtype=np.uint32)
        a = others[:, 0] | (others[:, 1] << 8) | (others[:, 2] << 16) | (others[:, 3] << 24)
        got = gather(carries(a.astype(np.uint32), t))
        want = sum((others[:, b] >= t).astype(np.uint32) << np.uint32(b) for b in range(4))
        assert np.array_equal(got, want), (t, pos)


@pytest.mark.parametrize("t", [1, 2, 64, 127, 128, 129, 200, 254, 255])
def test_whole_words(t):
    g = np.random.default_rng(1000 + t)
    grey = g.integers(0, 256, size=(4096, 32), dtype=np.uint8)
    grey[0] = t                  # exactly at the threshold
    grey[1] = t - 1              # just below
    got = pack32(grey, t)
    bits = (grey >= t).astype(np.uint64)
    want = (bits << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    assert np.array_equal(got, want)

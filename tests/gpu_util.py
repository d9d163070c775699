"""Helpers for the GPU parity tests: device buffers with guard canaries and
zeroed-padding checks around the packed images."""
import numpy as np

SENTINEL = 0xA5A5A5A5
GUARD = 64          # canary words before and after every buffer


def torch_dev():
    import torch
    return torch.device("cuda:0")


class DevBuf:
    """A device buffer of h*stride words inside a larger canary-filled
    allocation; `off` words of extra misalignment move the start."""

    def __init__(self, words: np.ndarray, off: int = 0, fill: int | None = None):
        import torch
        words = np.ascontiguousarray(words, dtype=np.uint32)
        self.shape = words.shape
        n = words.size
        total = GUARD + off + n + GUARD
        host = np.full(total, SENTINEL, dtype=np.uint32)
        if fill is None:
            host[GUARD + off:GUARD + off + n] = words.ravel()
        else:
            host[GUARD + off:GUARD + off + n] = np.uint32(fill)
        self.off = off
        self.n = n
        self.t = torch.from_numpy(host.view(np.int32)).to(torch_dev())

    def ptr(self) -> int:
        return self.t.data_ptr() + 4 * (GUARD + self.off)

    def host_all(self) -> np.ndarray:
        return self.t.cpu().numpy().view(np.uint32)

    def words(self) -> np.ndarray:
        a = self.host_all()
        return a[GUARD + self.off:GUARD + self.off + self.n].reshape(self.shape)

    def guards_intact(self) -> bool:
        a = self.host_all()
        return bool((a[:GUARD + self.off] == SENTINEL).all() and
                    (a[GUARD + self.off + self.n:] == SENTINEL).all())


def check_output_layout(out_words: np.ndarray, w: int):
    """Output padding bits of word nw-1 and padding words >= nw are all 0."""
    nw = (w + 31) // 32
    if w % 32:
        assert (out_words[:, nw - 1] >> np.uint32(w % 32) == 0).all(), "padding bits set"
    if out_words.shape[1] > nw:
        assert (out_words[:, nw:] == 0).all(), "padding words not zeroed"

"""ctypes binding of libme (C ABI in include/me.h).

Argument marshalling only: every computation runs in the CUDA kernels of
libme.so.  Functions keep the C names and return the C status code; the
``*_checked`` helpers and :func:`check` raise :class:`MeError` instead.
Tensors may be passed wherever the C call takes a device pointer (their
``data_ptr()`` is used); streams may be a ``torch.cuda.Stream``, a raw
``cudaStream_t`` integer, or None for the current torch stream.

There is no fallback: if libme.so is missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB_PATH = os.path.join(PKG, "libme.so")
HEADER = os.path.join(ROOT, "include", "me.h")

c_i32, c_i64, c_u64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p


def _constants():
    """#define constants of me.h, read from the header itself."""
    out = {}
    with open(HEADER) as f:
        for m in re.finditer(r"^#define\s+(ME_[A-Z0-9_]+)\s+(-?\d+)", f.read(), re.M):
            out[m.group(1)] = int(m.group(2))
    return out


C = _constants()
globals().update(C)


class MeError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = status_string(status) if _lib is not None else str(status)
        extra = ""
        if status == C["ME_ERR_CUDA"] and _lib is not None:
            extra = f" (cudaError {_lib.me_last_cuda_error()})"
        super().__init__(f"{what}: {name}{extra}" if what else name + extra)


class me_desc(ctypes.Structure):
    _fields_ = [("img", c_vp), ("edge", c_vp), ("w", c_i32), ("h", c_i32),
                ("stride_words", c_i32), ("boundary", c_i32)]


class me_tile_cfg(ctypes.Structure):
    _fields_ = [("engine", c_i32), ("rows_per_lane", c_i32), ("vec_words", c_i32),
                ("cta_threads", c_i32), ("ctas_per_sm", c_i32), ("stage_kb", c_i32),
                ("stages", c_i32), ("chunk_tiles", c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class me_host_image(ctypes.Structure):
    _fields_ = [("offset_words", c_i64), ("w", c_i32), ("h", c_i32),
                ("stride_words", c_i32), ("boundary", c_i32)]


class me_serve_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_i64), ("staging_bytes", c_i64),
                ("max_inflight", c_i32), ("max_batch", c_i32), ("tick_us", c_i32),
                ("device", c_i32)]


class me_timing(ctypes.Structure):
    _fields_ = [("queue_us", ctypes.c_double), ("device_us", ctypes.c_double),
                ("total_us", ctypes.c_double)]


# name -> (restype, argtypes)
PROTOTYPES = {
    "me_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "me_last_cuda_error": (ctypes.c_int, []),
    "me_version": (ctypes.c_int, []),
    "me_edges": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_vp, c_i32, c_vp]),
    "me_edges_staged": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_vp, c_i32, c_vp]),
    "me_edges_staged_static": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_vp, c_i32,
                                              c_vp]),
    "me_fundamental_edges": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_vp, c_vp,
                                            c_vp, c_vp, c_i32, c_vp]),
    "me_edges_display": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_vp, c_i32, c_vp]),
    "me_end_points": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_vp, c_i32, c_vp]),
    "me_edges_inplace": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_i32, c_vp]),
    "me_threshold_edges": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_i32, c_vp, c_i32,
                                          c_vp, c_i32, c_vp]),
    "me_threshold_edges_otsu": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_vp, c_i32, c_vp,
                                               c_i32, c_vp, c_vp]),
    "me_edges_batch": (ctypes.c_int, [ctypes.POINTER(me_desc), c_i32, c_vp]),
    "me_batch_plan_create": (ctypes.c_int, [ctypes.POINTER(me_desc), c_i32, c_vp,
                                            ctypes.POINTER(c_vp)]),
    "me_batch_run": (ctypes.c_int, [c_vp, c_vp]),
    "me_batch_plan_bytes": (c_i64, [c_vp]),
    "me_batch_plan_destroy": (ctypes.c_int, [c_vp]),
    "me_edges_batch_host": (ctypes.c_int, [c_vp, c_vp, ctypes.POINTER(me_host_image), c_i32,
                                           c_i64, c_vp]),
    "me_get_tile_cfg": (ctypes.c_int, [c_i32, ctypes.POINTER(me_tile_cfg)]),
    "me_set_tile_cfg": (ctypes.c_int, [c_i32, ctypes.POINTER(me_tile_cfg)]),
    "me_autotune": (ctypes.c_int, [c_i32, ctypes.POINTER(me_desc), c_i32, c_i32, c_vp,
                                   ctypes.POINTER(me_tile_cfg)]),
    "me_serve_open": (ctypes.c_int, [ctypes.POINTER(me_serve_cfg), ctypes.POINTER(c_vp)]),
    "me_serve_submit": (ctypes.c_int, [c_vp, c_vp, c_i32, c_i32, c_i32, c_i32,
                                       ctypes.POINTER(c_u64)]),
    "me_serve_poll": (ctypes.c_int, [c_vp, c_u64, c_vp, c_i64, ctypes.POINTER(me_timing)]),
    "me_serve_cancel": (ctypes.c_int, [c_vp, c_u64]),
    "me_serve_submit_direct": (ctypes.c_int, [c_vp, c_vp, c_vp, c_i32, c_i32, c_i32, c_i32,
                                              ctypes.POINTER(c_u64)]),
    "me_serve_reserve": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_i32, ctypes.POINTER(c_u64),
                                        ctypes.POINTER(c_vp)]),
    "me_serve_commit": (ctypes.c_int, [c_vp, c_u64]),
    "me_serve_poll_view": (ctypes.c_int, [c_vp, c_u64, c_i64, ctypes.POINTER(c_vp),
                                          ctypes.POINTER(me_timing)]),
    "me_serve_release": (ctypes.c_int, [c_vp, c_u64]),
    "me_serve_stats": (ctypes.c_int, [c_vp, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64),
                                      ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    "me_serve_copies": (ctypes.c_int, [c_vp, ctypes.POINTER(c_i64)]),
    "me_serve_close": (ctypes.c_int, [c_vp, c_i64]),
    "me_device_faults": (ctypes.c_int, [c_i32, ctypes.POINTER(ctypes.c_uint32)]),
    "me_shutdown": (ctypes.c_int, []),
}

_lib = None
_lock = threading.Lock()


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libme.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise MeError(C["ME_ERR_UNSUPPORTED"],
                              f"libme.so not built at {p}; run __graft_entry__.build()")
            lib = ctypes.CDLL(p)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().me_status_string(int(status)).decode()


def check(status: int, what: str = "") -> int:
    if status < 0:
        raise MeError(status, what)
    return status


def ptr(x) -> int | None:
    """Device pointer of a tensor, or an integer pointer as is."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------- the C calls
def me_edges(img, w, h, stride_words, edge, boundary=0, stream=None) -> int:
    return load().me_edges(ptr(img), w, h, stride_words, ptr(edge), boundary,
                           stream_handle(stream))


def me_edges_staged(img, w, h, stride_words, edge, boundary=0, stream=None) -> int:
    return load().me_edges_staged(ptr(img), w, h, stride_words, ptr(edge), boundary,
                                  stream_handle(stream))


def me_edges_inplace(img, w, h, stride_words, boundary=0, stream=None) -> int:
    return load().me_edges_inplace(ptr(img), w, h, stride_words, boundary,
                                   stream_handle(stream))


def me_threshold_edges(grey, w, h, pitch_bytes, threshold, edge, stride_words, binary=None,
                       boundary=0, stream=None) -> int:
    return load().me_threshold_edges(ptr(grey), w, h, pitch_bytes, threshold, ptr(edge),
                                     stride_words, ptr(binary), boundary, stream_handle(stream))


def me_threshold_edges_otsu(grey, w, h, pitch_bytes, edge, stride_words, binary=None,
                            boundary=0, threshold_out=None, stream=None) -> int:
    return load().me_threshold_edges_otsu(ptr(grey), w, h, pitch_bytes, ptr(edge), stride_words,
                                          ptr(binary), boundary, ptr(threshold_out),
                                          stream_handle(stream))


def me_edges_staged_static(img, w, h, stride_words, edge, boundary=0, stream=None) -> int:
    return load().me_edges_staged_static(ptr(img), w, h, stride_words, ptr(edge), boundary,
                                         stream_handle(stream))


def me_fundamental_edges(img, w, h, stride_words, left, right, up, down, boundary=0,
                         stream=None) -> int:
    return load().me_fundamental_edges(ptr(img), w, h, stride_words, ptr(left),
                                       ptr(right), ptr(up), ptr(down), boundary,
                                       stream_handle(stream))


def me_edges_display(img, w, h, stride_words, out, boundary=0, stream=None) -> int:
    return load().me_edges_display(ptr(img), w, h, stride_words, ptr(out), boundary,
                                   stream_handle(stream))


def me_end_points(img, w, h, stride_words, out, boundary=0, stream=None) -> int:
    return load().me_end_points(ptr(img), w, h, stride_words, ptr(out), boundary,
                                stream_handle(stream))


def make_descs(items) -> ctypes.Array:
    """items: iterable of (img, edge, w, h, stride_words, boundary)."""
    items = list(items)
    arr = (me_desc * max(1, len(items)))()
    for i, (img, edge, w, h, stride, boundary) in enumerate(items):
        arr[i] = me_desc(ptr(img), ptr(edge), w, h, stride, boundary)
    return arr


def me_edges_batch(descs, n=None, stream=None) -> int:
    n = len(descs) if n is None else n
    return load().me_edges_batch(descs, n, stream_handle(stream))


def make_host_images(items) -> ctypes.Array:
    """items: iterable of (offset_words, w, h, stride_words, boundary)."""
    items = list(items)
    arr = (me_host_image * max(1, len(items)))()
    for i, (off, w, h, stride, boundary) in enumerate(items):
        arr[i] = me_host_image(off, w, h, stride, boundary)
    return arr


def me_edges_batch_host(host_in, host_out, imgs, n=None, chunk_bytes=0, stream=None) -> int:
    """host_in / host_out: numpy arrays, pinned torch CPU tensors or pointers."""
    def hptr(x):
        if hasattr(x, "ctypes"):
            return x.ctypes.data
        if hasattr(x, "data_ptr"):
            return x.data_ptr()
        return int(x)
    n = len(imgs) if n is None else n
    return load().me_edges_batch_host(hptr(host_in), hptr(host_out), imgs, n, chunk_bytes,
                                      stream_handle(stream))


class BatchPlan:
    """me_batch_plan_create / me_batch_run / me_batch_plan_destroy."""

    def __init__(self, descs, n=None, stream=None):
        n = len(descs) if n is None else n
        self._h = c_vp()
        check(load().me_batch_plan_create(descs, n, stream_handle(stream),
                                          ctypes.byref(self._h)), "me_batch_plan_create")

    def run(self, stream=None) -> int:
        return load().me_batch_run(self._h, stream_handle(stream))

    @property
    def bytes(self) -> int:
        return load().me_batch_plan_bytes(self._h)

    def close(self):
        if self._h:
            load().me_batch_plan_destroy(self._h)
            self._h = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def me_get_tile_cfg(kind) -> me_tile_cfg:
    c = me_tile_cfg()
    check(load().me_get_tile_cfg(kind, ctypes.byref(c)), "me_get_tile_cfg")
    return c


def me_set_tile_cfg(kind, cfg: me_tile_cfg) -> int:
    return load().me_set_tile_cfg(kind, ctypes.byref(cfg))


def me_autotune(kind, descs, n=None, reps=10, stream=None) -> me_tile_cfg:
    n = len(descs) if n is None else n
    best = me_tile_cfg()
    check(load().me_autotune(kind, descs, n, reps, stream_handle(stream),
                             ctypes.byref(best)), "me_autotune")
    return best


def me_device_faults(clear=True) -> int:
    v = ctypes.c_uint32()
    check(load().me_device_faults(1 if clear else 0, ctypes.byref(v)), "me_device_faults")
    return v.value


def me_shutdown() -> int:
    return load().me_shutdown()


# ---------------------------------------------------------------- serving
class Server:
    """me_serve_open / submit / poll / stats / close."""

    def __init__(self, hbm_budget_bytes=8 << 30, staging_bytes=0, max_inflight=4,
                 max_batch=256, tick_us=50, device=0):
        cfg = me_serve_cfg(hbm_budget_bytes, staging_bytes, max_inflight, max_batch,
                           tick_us, device)
        self._h = c_vp()
        check(load().me_serve_open(ctypes.byref(cfg), ctypes.byref(self._h)),
              "me_serve_open")

    def submit(self, host_img, w, h, stride_words, boundary=0) -> tuple[int, int]:
        """host_img: a C-contiguous numpy uint32 array (or a pointer)."""
        t = c_u64()
        p = host_img.ctypes.data if hasattr(host_img, "ctypes") else int(host_img)
        rc = load().me_serve_submit(self._h, p, w, h, stride_words, boundary,
                                    ctypes.byref(t))
        return rc, t.value

    def poll(self, ticket, host_edge, timeout_us=-1):
        tm = me_timing()
        p = host_edge.ctypes.data if hasattr(host_edge, "ctypes") else int(host_edge)
        rc = load().me_serve_poll(self._h, ticket, p, timeout_us, ctypes.byref(tm))
        return rc, tm

    def cancel(self, ticket) -> int:
        return load().me_serve_cancel(self._h, ticket)

    def submit_direct(self, host_img, host_edge, w, h, stride_words, boundary=0):
        """Direct submit: host_img and host_edge are pinned host buffers (numpy
        views of pinned tensors, or pointers) the kernel reads and writes."""
        t = c_u64()
        pi = host_img.ctypes.data if hasattr(host_img, "ctypes") else int(host_img)
        po = host_edge.ctypes.data if hasattr(host_edge, "ctypes") else int(host_edge)
        rc = load().me_serve_submit_direct(self._h, pi, po, w, h, stride_words, boundary,
                                           ctypes.byref(t))
        return rc, t.value

    def poll_direct(self, ticket, timeout_us=-1):
        """Collect a direct ticket (its edge map is in its own buffer)."""
        tm = me_timing()
        rc = load().me_serve_poll(self._h, ticket, None, timeout_us, ctypes.byref(tm))
        return rc, tm

    def reserve(self, w, h, stride_words, boundary=0):
        """Zero-copy submit, step 1: (status, ticket, numpy view of the
        staging to write the h x stride_words image into)."""
        import numpy as np
        t, p = c_u64(), c_vp()
        rc = load().me_serve_reserve(self._h, w, h, stride_words, boundary, ctypes.byref(t),
                                     ctypes.byref(p))
        if rc != 0:
            return rc, 0, None
        buf = (ctypes.c_uint32 * (h * stride_words)).from_address(p.value)
        return rc, t.value, np.ctypeslib.as_array(buf).reshape(h, stride_words)

    def commit(self, ticket) -> int:
        return load().me_serve_commit(self._h, ticket)

    def poll_view(self, ticket, h, stride_words, timeout_us=-1):
        """Zero-copy collect: (status, timing, read-only numpy view of the
        edge map in the server's staging, valid until release)."""
        import numpy as np
        tm, p = me_timing(), c_vp()
        rc = load().me_serve_poll_view(self._h, ticket, timeout_us, ctypes.byref(p),
                                       ctypes.byref(tm))
        if rc != 0:
            return rc, tm, None
        buf = (ctypes.c_uint32 * (h * stride_words)).from_address(p.value)
        v = np.ctypeslib.as_array(buf).reshape(h, stride_words)
        v.flags.writeable = False
        return rc, tm, v

    def release(self, ticket) -> int:
        return load().me_serve_release(self._h, ticket)

    def stats(self):
        v = [c_i64() for _ in range(5)]
        check(load().me_serve_stats(self._h, *[ctypes.byref(x) for x in v[:4]]),
              "me_serve_stats")
        check(load().me_serve_copies(self._h, ctypes.byref(v[4])), "me_serve_copies")
        return dict(zip(("submitted", "completed", "batches", "peak_bytes", "copies"),
                        [x.value for x in v]))

    @property
    def handle(self):
        return self._h

    def close(self, drain_timeout_us=-1) -> int:
        rc = C["ME_OK"]
        if self._h:
            rc = load().me_serve_close(self._h, drain_timeout_us)
            self._h = c_vp()
        return rc

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------ serving load generator
LOADGEN_PATH = os.path.join(PKG, "libme_loadgen.so")


class me_load_item(ctypes.Structure):
    _fields_ = [("img", c_vp), ("expect", c_vp), ("w", c_i32), ("h", c_i32),
                ("stride_words", c_i32), ("boundary", c_i32)]


class me_load_result(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("mismatches", c_i64), ("errors", c_i64),
                ("first_error", c_i32), ("pad", c_i32)]


_loadgen = None


def load_loadgen() -> ctypes.CDLL:
    """libme_loadgen.so (built beside libme.so; raises if missing)."""
    global _loadgen
    load()
    with _lock:
        if _loadgen is None:
            if not os.path.exists(LOADGEN_PATH):
                raise OSError(f"{LOADGEN_PATH} not built: run paper_1401_5245_gb300.build")
            lg = ctypes.CDLL(LOADGEN_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lg.me_load_run.restype = ctypes.c_int
            lg.me_load_run.argtypes = [c_vp, ctypes.POINTER(me_load_item), c_i64, dp, c_i32,
                                       c_i32, c_i32, c_vp, c_i64, c_i32, dp, dp,
                                       ctypes.POINTER(me_load_result)]
            _loadgen = lg
    return _loadgen


def load_run(server: "Server", reqs, expect=None, arrival_s=None, clients=4, window=32,
             zero_copy=False, direct=None):
    """Drive `server` with the requests `reqs` (objects with .words, .w, .h,
    .stride_words, .boundary) from C threads (me_load_run).  expect: None or
    one edge-map array per request to compare with.  arrival_s: None for a
    closed loop of `window` outstanding requests per client, else the
    arrival times in seconds (open loop).  zero_copy: the clients write into
    reserved staging and read results in place.  direct: (out_ring, slot_words,
    slots) -- the requests' images are pinned and the kernel writes each
    edge map into a slot of the pinned out_ring (`slots` per client).
    Returns wall_s, mismatches,
    errors, first_error and the per-request latency_us / server_us arrays."""
    import numpy as np
    n = len(reqs)
    items = (me_load_item * n)()
    for i, im in enumerate(reqs):
        items[i].img = im.words.ctypes.data
        items[i].expect = expect[i].ctypes.data if expect is not None else None
        items[i].w, items[i].h = im.w, im.h
        items[i].stride_words, items[i].boundary = im.stride_words, im.boundary
    lat = np.full(n, np.nan)
    srv_us = np.full(n, np.nan)
    dp = ctypes.POINTER(ctypes.c_double)
    arr = None
    if arrival_s is not None:
        arr = np.ascontiguousarray(np.asarray(arrival_s, dtype=np.float64) * 1e6)
    res = me_load_result()
    check(load_loadgen().me_load_run(
        server.handle, items, n, arr.ctypes.data_as(dp) if arr is not None else None,
        clients, window, 2 if direct else 1 if zero_copy else 0,
        direct[0] if direct else None, direct[1] if direct else 0, direct[2] if direct else 0,
        lat.ctypes.data_as(dp), srv_us.ctypes.data_as(dp),
        ctypes.byref(res)), "me_load_run")
    return {"wall_s": res.wall_s, "mismatches": res.mismatches, "errors": res.errors,
            "first_error": res.first_error, "latency_us": lat, "server_us": srv_us}

"""The serving engine: every served edge map equals the one computed alone,
under concurrent submitters, a budget small enough to force queuing, heap
fallback when staging is full, cancellation, timeouts and budget refusal.
All failures are made on the host (no GPU fault is ever provoked)."""
import ctypes
import threading

import numpy as np
import pytest

from oracle import oracle as O
from paper_1401_5245_gb300 import _lib, synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.init()
    _lib.load()


@pytest.fixture(scope="module")
def pool():
    """A few images of each serving size class (48x48 glyphs, 1024x1024
    crops, 2480x3508 pages), plus odd shapes and black boundaries."""
    p = S.serve_pool(0, per_class=(8, 3, 2))
    items = [im for cls in p for im in cls]
    g = np.random.default_rng(1)
    for w, h in [(1, 1), (33, 7), (100, 1), (5000, 3)]:
        img = (g.random((h, w)) < 0.5).astype(np.uint8)
        items.append(S.Image(S.pack(img, S.words_per_row(w) + 1, pad="random"), w, h, 1))
    return items


def alone(im):
    """The same image through me_edges on the device, alone."""
    import torch
    x = torch.from_numpy(im.words.view(np.int32)).cuda()
    y = torch.zeros_like(x)
    assert _lib.me_edges(x, im.w, im.h, im.stride_words, y, im.boundary) == 0
    torch.cuda.synchronize()
    return y.cpu().numpy().view(np.uint32)


def serve_all(srv, ims, threads=1):
    out = [None] * len(ims)
    errs = []

    def worker(idx):
        try:
            tickets = []
            for i in idx:
                im = ims[i]
                rc, t = srv.submit(np.ascontiguousarray(im.words), im.w, im.h,
                                   im.stride_words, im.boundary)
                assert rc == 0, _lib.status_string(rc)
                tickets.append((i, t))
            for i, t in tickets:
                res = np.empty_like(ims[i].words)
                rc, tm = srv.poll(t, res, -1)
                assert rc == 0, _lib.status_string(rc)
                assert tm.total_us >= tm.device_us >= 0 and tm.queue_us >= 0
                out[i] = res
        except Exception as e:   # noqa: BLE001
            errs.append(e)

    ths = [threading.Thread(target=worker, args=(list(range(k, len(ims), threads)),))
           for k in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errs, errs
    return out


def test_served_equals_alone_with_concurrent_submitters(pool):
    ims = [pool[i % len(pool)] for i in range(120)]
    refs = {id(im): alone(im) for im in pool}
    srv = _lib.Server(hbm_budget_bytes=256 << 20, staging_bytes=256 << 20,
                      max_inflight=3, max_batch=16, tick_us=20)
    try:
        out = serve_all(srv, ims, threads=4)
        for im, res in zip(ims, out):
            assert np.array_equal(res, refs[id(im)])
        st = srv.stats()
        assert st["submitted"] == st["completed"] == len(ims)
        assert st["batches"] >= 1 and 0 < st["peak_bytes"] <= 256 << 20
    finally:
        assert srv.close() == 0
    # every served shape (glyphs, crops, pages, odd shapes, black boundary)
    # is also the oracle's edge map
    for im in pool:
        want = O.edges(S.unpack(im.words, im.w), im.boundary)
        assert np.array_equal(S.unpack(refs[id(im)], im.w), want), (im.w, im.h)


def test_small_budget_forces_queueing(pool):
    """Room for little more than one page at a time: requests wait for
    memory, are admitted as batches retire, and every result is exact."""
    page = max(pool, key=lambda im: im.packed_bytes)
    budget = 2 * page.packed_bytes + (1 << 16)
    ims = [pool[i % len(pool)] for i in range(60)]
    refs = {id(im): alone(im) for im in pool}
    srv = _lib.Server(hbm_budget_bytes=budget, staging_bytes=64 << 20, max_inflight=2,
                      max_batch=4, tick_us=10)
    try:
        out = serve_all(srv, ims, threads=2)
        for im, res in zip(ims, out):
            assert np.array_equal(res, refs[id(im)])
        st = srv.stats()
        assert st["peak_bytes"] <= budget
        assert st["batches"] >= len(ims) // 4
    finally:
        srv.close()


def test_budget_refusal(pool):
    page = max(pool, key=lambda im: im.packed_bytes)
    srv = _lib.Server(hbm_budget_bytes=page.packed_bytes, staging_bytes=8 << 20)
    try:
        rc, _ = srv.submit(page.words, page.w, page.h, page.stride_words)
        assert rc == _lib.C["ME_ERR_BUDGET"]
        small = pool[0]
        rc, t = srv.submit(small.words, small.w, small.h, small.stride_words)
        assert rc == 0
        res = np.empty_like(small.words)
        assert srv.poll(t, res, -1)[0] == 0
        assert np.array_equal(res, alone(small))
    finally:
        srv.close()


def test_staging_full_timeout_cancel_and_unknown_ticket(pool):
    """Staging for one request only: the second waits in heap memory until
    the first is collected, so its poll times out deterministically; a
    cancelled request is forgotten; unknown tickets are refused."""
    a = pool[-5]                         # a 1024 x 1024 crop or a page
    span = (a.packed_bytes + 255) // 256 * 256
    srv = _lib.Server(hbm_budget_bytes=64 << 20, staging_bytes=2 * span,
                      max_inflight=1, max_batch=1)
    try:
        rc, ta = srv.submit(a.words, a.w, a.h, a.stride_words)
        assert rc == 0
        rc, tb = srv.submit(a.words, a.w, a.h, a.stride_words)
        assert rc == 0
        rc, tc = srv.submit(a.words, a.w, a.h, a.stride_words)
        assert rc == 0
        res = np.empty_like(a.words)
        rc, _ = srv.poll(tb, res, 2000)
        assert rc in (_lib.C["ME_TIMEOUT"], _lib.C["ME_PENDING"])
        assert srv.poll(tb, res, 0)[0] == _lib.C["ME_PENDING"]
        assert srv.cancel(tc) == 0
        assert srv.poll(tc, res, 0)[0] == _lib.C["ME_ERR_TICKET"]
        assert srv.poll(ta, res, -1)[0] == 0
        ref = alone(a)
        assert np.array_equal(res, ref)
        res2 = np.empty_like(a.words)
        assert srv.poll(tb, res2, -1)[0] == 0
        assert np.array_equal(res2, ref)
        assert srv.poll(ta, res, 0)[0] == _lib.C["ME_ERR_TICKET"]     # collected
        assert srv.poll(123456789, res, 0)[0] == _lib.C["ME_ERR_TICKET"]
        assert srv.cancel(987654321) == _lib.C["ME_ERR_TICKET"]
    finally:
        srv.close()


def test_close_drops_uncollected_and_bad_args(pool):
    srv = _lib.Server(hbm_budget_bytes=64 << 20, staging_bytes=64 << 20)
    for im in pool[:6]:
        assert srv.submit(im.words, im.w, im.h, im.stride_words)[0] == 0
    assert srv.submit(pool[0].words, 0, 5, 1)[0] == _lib.C["ME_ERR_ARG"]
    assert srv.submit(pool[0].words, 100, 5, 1)[0] == _lib.C["ME_ERR_ARG"]   # stride
    assert srv.close(-1) == 0
    L = _lib.load()
    cfg = _lib.me_serve_cfg(0, 0, 1, 1, 10, 0)
    h = _lib.c_vp()
    import ctypes
    assert L.me_serve_open(ctypes.byref(cfg), ctypes.byref(h)) == _lib.C["ME_ERR_ARG"]


# ------------------------------------------------- the C load generator
def oracle_words(im):
    """The oracle's edge map of a pool image, packed in the image's layout."""
    e = O.edges(S.unpack(im.words, im.w), im.boundary)
    return S.pack(e, im.stride_words)


def test_load_generator_closed_loop_every_result_is_the_oracles(pool):
    """Many clients in a closed loop through the C load generator: every
    result equals the oracle's edge map, requests share launches (continuous
    batching) and neighbouring requests share copies."""
    want = {id(im): oracle_words(im) for im in pool}
    g = np.random.default_rng(5)
    reqs = [pool[int(i)] for i in g.integers(0, len(pool), 3000)]
    srv = _lib.Server(hbm_budget_bytes=1 << 30, staging_bytes=512 << 20, max_inflight=1,
                      max_batch=512, tick_us=0)
    try:
        r = _lib.load_run(srv, reqs, expect=[want[id(im)] for im in reqs], clients=4,
                          window=32)
        st = srv.stats()
    finally:
        assert srv.close() == 0
    assert r["errors"] == 0 and r["first_error"] == 0
    assert r["mismatches"] == 0
    assert st["completed"] == len(reqs)
    assert not np.isnan(r["latency_us"]).any()
    assert (r["server_us"] <= r["latency_us"] + 1e-3).all()
    # one batch on the GPU at a time and 128 requests outstanding: the
    # requests that arrive meanwhile share the next launch
    assert st["completed"] / st["batches"] > 2, st
    # copies: far fewer than two per request
    assert st["copies"] < st["completed"], st


def test_load_generator_open_loop_and_black_boundary(pool):
    """Poisson arrivals (open loop) with black-boundary requests mixed in:
    every result is the oracle's and the latencies are measured from the
    scheduled arrivals."""
    items = []
    for im in pool:
        items.append(im)
        items.append(S.Image(im.words, im.w, im.h, 1 - im.boundary))
    want = {id(im): oracle_words(im) for im in items}
    g = np.random.default_rng(6)
    reqs = [items[int(i)] for i in g.integers(0, len(items), 600)]
    t = np.cumsum(g.exponential(1 / 20000.0, len(reqs)))
    srv = _lib.Server(hbm_budget_bytes=256 << 20, staging_bytes=256 << 20, max_inflight=2,
                      max_batch=64, tick_us=0)
    try:
        r = _lib.load_run(srv, reqs, expect=[want[id(im)] for im in reqs], arrival_s=t,
                          clients=2)
    finally:
        assert srv.close() == 0
    assert r["errors"] == 0 and r["mismatches"] == 0
    assert (r["latency_us"] > 0).all()
    assert r["wall_s"] >= t[-1] * 0.99


def test_load_generator_refuses_bad_arguments():
    lg = _lib.load_loadgen()
    res = _lib.me_load_result()
    assert lg.me_load_run(None, None, 0, None, 1, 1, 0, None, 0, 0, None, None,
                          ctypes.byref(res)) == _lib.C["ME_ERR_ARG"]


# ------------------------------------------------------------- zero copy
def test_zero_copy_reserve_commit_view_release(pool):
    """Images written straight into reserved staging and edge maps read
    where the server leaves them: every one is the oracle's; a reserved
    request can be cancelled; release refuses unfinished tickets; commit
    refuses tickets that are not open."""
    srv = _lib.Server(hbm_budget_bytes=256 << 20, staging_bytes=256 << 20, max_inflight=2,
                      max_batch=8, tick_us=0)
    try:
        tickets = []
        for im in pool:
            rc, t, dst = srv.reserve(im.w, im.h, im.stride_words, im.boundary)
            assert rc == 0
            dst[...] = im.words
            tickets.append((im, t))
        # one more, reserved and cancelled before it is committed
        rc, tx, _ = srv.reserve(40, 3, 2)
        assert rc == 0
        assert srv.release(tickets[0][1]) == _lib.C["ME_ERR_ARG"]     # not finished
        assert srv.cancel(tx) == 0
        for im, t in tickets:
            assert srv.commit(t) == 0
        assert srv.commit(tickets[0][1]) == _lib.C["ME_ERR_ARG"]      # committed already
        for im, t in tickets:
            rc, tm, view = srv.poll_view(t, im.h, im.stride_words)
            assert rc == 0 and tm.total_us >= tm.device_us >= 0
            assert np.array_equal(S.unpack(view, im.w),
                                  O.edges(S.unpack(im.words, im.w), im.boundary)), (im.w, im.h)
            assert srv.release(t) == 0
            assert srv.release(t) == _lib.C["ME_ERR_TICKET"]
        st = srv.stats()
        assert st["completed"] == len(pool)
    finally:
        assert srv.close() == 0


def test_zero_copy_staging_full_is_pending(pool):
    """Staging for one request: a second reservation reports ME_PENDING
    (nothing reserved) until the first is released."""
    a = max(pool, key=lambda im: im.packed_bytes)
    span = (a.packed_bytes + 255) // 256 * 256
    srv = _lib.Server(hbm_budget_bytes=64 << 20, staging_bytes=2 * span, max_inflight=1,
                      max_batch=1, tick_us=0)
    try:
        rc, t, dst = srv.reserve(a.w, a.h, a.stride_words)
        assert rc == 0
        dst[...] = a.words
        assert srv.reserve(a.w, a.h, a.stride_words)[0] == _lib.C["ME_PENDING"]
        assert srv.commit(t) == 0
        rc, _, view = srv.poll_view(t, a.h, a.stride_words)
        assert rc == 0
        assert srv.reserve(a.w, a.h, a.stride_words)[0] == _lib.C["ME_PENDING"]
        assert srv.release(t) == 0
        rc, t2, dst2 = srv.reserve(a.w, a.h, a.stride_words)
        assert rc == 0
        assert srv.cancel(t2) == 0
    finally:
        assert srv.close() == 0


def test_load_generator_zero_copy_every_result_is_the_oracles(pool):
    want = {id(im): oracle_words(im) for im in pool}
    g = np.random.default_rng(8)
    reqs = [pool[int(i)] for i in g.integers(0, len(pool), 3000)]
    srv = _lib.Server(hbm_budget_bytes=1 << 30, staging_bytes=256 << 20, max_inflight=2,
                      max_batch=512, tick_us=0)
    try:
        r = _lib.load_run(srv, reqs, expect=[want[id(im)] for im in reqs], clients=4,
                          window=32, zero_copy=True)
        r2 = _lib.load_run(srv, reqs, arrival_s=np.cumsum(g.exponential(1e-5, len(reqs))),
                           clients=3, zero_copy=True)
        st = srv.stats()
    finally:
        assert srv.close() == 0
    assert r["errors"] == 0 and r["mismatches"] == 0
    assert r2["errors"] == 0
    assert st["completed"] == 2 * len(reqs)


def test_random_interleaving_of_every_call(pool):
    """Six threads each run a random mix of copying, zero-copy and direct
    submits, polls with random timeouts (0, short, unlimited), views and
    releases, and cancels of their own requests, against a budget and a
    staging pool small enough that requests queue for memory and spill into
    heap memory.  Every result collected equals the oracle's; the server's
    counters add up; close drains what is left.  Direct requests' pinned
    buffers stay alive until close (a cancelled one may still be written)."""
    import torch
    want = {id(im): oracle_words(im) for im in pool}
    small = [im for im in pool if im.packed_bytes <= 200_000]
    pinned_in = {id(im): pinned_copy(im.words) for im in small}
    outs = []              # every direct output buffer, kept until close
    page = max(pool, key=lambda im: im.packed_bytes)
    span = (page.packed_bytes + 255) // 256 * 256
    srv = _lib.Server(hbm_budget_bytes=6 * span, staging_bytes=8 * span, max_inflight=2,
                      max_batch=5, tick_us=0)
    errs, counts = [], []

    def worker(seed):
        g = np.random.default_rng(seed)
        live = []          # (ticket, image, zero_copy, direct output or None)
        done = cancelled = 0
        try:
            for _ in range(150):
                op = g.random()
                if op < 0.45 or not live:
                    im = pool[int(g.integers(0, len(pool)))]
                    if id(im) in pinned_in and g.random() < 0.35:
                        t_out = torch.empty(im.words.size, dtype=torch.int32).pin_memory()
                        outs.append(t_out)
                        out = t_out.numpy().view(np.uint32).reshape(im.words.shape)
                        rc, t = srv.submit_direct(pinned_in[id(im)][1], out, im.w, im.h,
                                                  im.stride_words, im.boundary)
                        assert rc == 0, _lib.status_string(rc)
                        live.append((t, im, False, out))
                    elif g.random() < 0.5:
                        rc, t = srv.submit(im.words, im.w, im.h, im.stride_words, im.boundary)
                        assert rc == 0, _lib.status_string(rc)
                        live.append((t, im, False, None))
                    else:
                        rc, t, dst = srv.reserve(im.w, im.h, im.stride_words, im.boundary)
                        if rc == _lib.C["ME_PENDING"]:
                            continue
                        assert rc == 0, _lib.status_string(rc)
                        dst[...] = im.words
                        assert srv.commit(t) == 0
                        live.append((t, im, True, None))
                elif op < 0.9:
                    k = int(g.integers(0, len(live)))
                    t, im, zc, out = live[k]
                    # no unlimited wait here: a request in heap memory waits
                    # for staging that other threads' uncollected results hold
                    timeout = int(g.choice([0, 200, 5000]))
                    if out is not None and g.random() < 0.5:
                        rc, tm = srv.poll_direct(t, timeout)
                        if rc in (_lib.C["ME_PENDING"], _lib.C["ME_TIMEOUT"]):
                            continue
                        assert rc == 0, _lib.status_string(rc)
                        assert np.array_equal(out, want[id(im)])
                    elif zc or g.random() < 0.3:
                        rc, tm, view = srv.poll_view(t, im.h, im.stride_words, timeout)
                        if rc in (_lib.C["ME_PENDING"], _lib.C["ME_TIMEOUT"]):
                            continue
                        assert rc == 0, _lib.status_string(rc)
                        assert np.array_equal(view, want[id(im)])
                        assert srv.release(t) == 0
                    else:
                        res = np.empty_like(im.words)
                        rc, tm = srv.poll(t, res, timeout)
                        if rc in (_lib.C["ME_PENDING"], _lib.C["ME_TIMEOUT"]):
                            continue
                        assert rc == 0, _lib.status_string(rc)
                        assert np.array_equal(res, want[id(im)])
                    live.pop(k)
                    done += 1
                else:
                    k = int(g.integers(0, len(live)))
                    assert srv.cancel(live[k][0]) == 0
                    live.pop(k)
                    cancelled += 1
            # collect the rest, whatever is ready first, so that the staging
            # of collected results lets the waiting requests in
            import time
            deadline = time.monotonic() + 60
            while live:
                assert time.monotonic() < deadline, "requests never finished"
                keep = []
                for t, im, zc, out in live:
                    res = np.empty_like(im.words)
                    rc, _ = srv.poll(t, res, 0)
                    if rc == _lib.C["ME_PENDING"]:
                        keep.append((t, im, zc, out))
                        continue
                    assert rc == 0, _lib.status_string(rc)
                    assert np.array_equal(res, want[id(im)])
                    done += 1
                if len(keep) == len(live):
                    time.sleep(1e-4)
                live = keep
            counts.append((done, cancelled))
        except Exception as e:   # noqa: BLE001
            errs.append(e)

    ths = [threading.Thread(target=worker, args=(100 + k,)) for k in range(6)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    try:
        assert not errs, errs
        st = srv.stats()
        assert st["submitted"] == sum(d + c for d, c in counts)
        assert st["peak_bytes"] <= 6 * span
    finally:
        assert srv.close(-1) == 0
        del outs


# ------------------------------------------------------------ direct submit
def pinned_copy(words):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(words).view(np.int32)).pin_memory()
    return t, t.numpy().view(np.uint32)


def test_direct_submit_reads_and_writes_the_callers_pinned_buffers(pool):
    """The kernel reads each image from the caller's pinned buffer and
    writes the edge map into the caller's pinned output: every one is the
    oracle's, with copying requests mixed in; unpinned buffers and
    overlapping ones are refused."""
    import torch
    srv = _lib.Server(hbm_budget_bytes=64 << 20, staging_bytes=64 << 20, max_inflight=2,
                      max_batch=8, tick_us=0)
    keep = []
    try:
        tickets = []
        for k, im in enumerate(pool):
            ti, src = pinned_copy(im.words)
            to, dst = pinned_copy(np.full_like(im.words, 0xA5A5A5A5))
            keep += [ti, to]
            rc, t = srv.submit_direct(src, dst, im.w, im.h, im.stride_words, im.boundary)
            assert rc == 0, _lib.status_string(rc)
            tickets.append((t, im, dst, True))
            if k % 3 == 0:       # a copying request in between
                rc, t2 = srv.submit(im.words, im.w, im.h, im.stride_words, im.boundary)
                assert rc == 0
                tickets.append((t2, im, None, False))
        for t, im, dst, direct in tickets:
            if direct:
                rc, tm = srv.poll_direct(t)
                got = dst
            else:
                got = np.empty_like(im.words)
                rc, tm = srv.poll(t, got, -1)
            assert rc == 0, _lib.status_string(rc)
            assert np.array_equal(got, oracle_words(im)), (im.w, im.h, direct)
        # refused: unpinned memory, overlap
        im = pool[0]
        _, src = pinned_copy(im.words)
        plain = np.empty_like(im.words)
        assert srv.submit_direct(src, plain, im.w, im.h, im.stride_words)[0] == \
            _lib.C["ME_ERR_ARG"]
        assert srv.submit_direct(src, src, im.w, im.h, im.stride_words)[0] == \
            _lib.C["ME_ERR_ALIAS"]
    finally:
        assert srv.close() == 0


def test_load_generator_direct_every_result_is_the_oracles(pool):
    """Direct mode of the load generator: the clients submit pinned images
    and the kernel writes each edge map into the client's slot of a pinned
    ring; every result is the oracle's, closed and open loop."""
    import torch
    want = [oracle_words(im) for im in pool]
    pinned = [pinned_copy(im.words) for im in pool]
    g = np.random.default_rng(9)
    idx = [int(i) for i in g.integers(0, len(pool), 3000)]
    reqs = [S.Image(pinned[i][1], pool[i].w, pool[i].h, pool[i].boundary) for i in idx]
    slot_words = max(im.words.size for im in pool)
    clients, slots = 4, 8
    ring = torch.empty(clients * slots * slot_words, dtype=torch.int32).pin_memory()
    srv = _lib.Server(hbm_budget_bytes=256 << 20, staging_bytes=64 << 20, max_inflight=2,
                      max_batch=64, tick_us=0)
    try:
        r = _lib.load_run(srv, reqs, expect=[want[i] for i in idx], clients=clients,
                          window=8, direct=(ring.data_ptr(), slot_words, slots))
        t = np.cumsum(g.exponential(1e-5, len(reqs)))
        r2 = _lib.load_run(srv, reqs, arrival_s=t, clients=3,
                           direct=(ring.data_ptr(), slot_words, slots))
        st = srv.stats()
    finally:
        assert srv.close() == 0
    assert r["errors"] == 0 and r["mismatches"] == 0, r["first_error"]
    assert r2["errors"] == 0, r2["first_error"]
    assert st["completed"] == 2 * len(reqs)
    assert st["copies"] == 0, st        # no staging copy in direct mode

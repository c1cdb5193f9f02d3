"""Server scheduling logic on the host (no GPU): the server's fake executor runs a
batch for fake_ms_per_view x views milliseconds instead of launching kernels.

Covers latest-wins supersession, admission by the output pool (FVV_EBUSY),
continuous batching over several slots, latency accounting and release."""
import threading
import time

import pytest

import paper_2112_10603_b300 as fvv
from paper_2112_10603_b300 import build as fvv_build


@pytest.fixture(scope="module", autouse=True)
def _built():
    fvv_build.build()


def _server(**kw):
    cfg = fvv.fvv_serve_default_cfg(fake_ms_per_view=kw.pop("fake", 2.0), n_res=1, res_h=[64], res_w=[64],
                                    n_cams=5, **kw)
    return fvv.fvv_serve_create(None, cfg)


def _wait(s, tk, timeout=5.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        st, ptr, lat = fvv.fvv_serve_poll(s, tk)
        if st == 0:
            return lat
        time.sleep(0.001)
    raise TimeoutError(tk)


def test_latest_wins_per_user():
    s = _server(slots_per_res=1, max_batch=4, pool_views=8)
    try:
        # no frames yet: nothing can launch, so the user's earlier requests wait
        a = fvv.fvv_serve_submit(s, 7, 0, 0.1, 0)
        b = fvv.fvv_serve_submit(s, 7, 1, 0.2, 0)
        c = fvv.fvv_serve_submit(s, 8, 2, 0.3, 0)
        d = fvv.fvv_serve_submit(s, 7, 3, 0.4, 0)
        for tk in (a, b):
            with pytest.raises(fvv.FvvError) as e:
                fvv.fvv_serve_poll(s, tk)
            assert e.value.code == fvv.FVV_ESUPERSEDED
        fvv.fvv_serve_set_frames(s, 0, 0, [0] * 5)
        _wait(s, c)
        _wait(s, d)
        st = fvv.fvv_serve_stats_get(s)
        assert st["submitted"] == 4 and st["superseded"] == 2 and st["completed"] == 2
    finally:
        fvv.fvv_serve_destroy(s)


def test_admission_by_output_pool():
    s = _server(slots_per_res=1, max_batch=2, pool_views=2)
    try:
        t1 = fvv.fvv_serve_submit(s, 1, 0, 0.5, 0)
        t2 = fvv.fvv_serve_submit(s, 2, 0, 0.5, 0)
        with pytest.raises(fvv.FvvError) as e:
            fvv.fvv_serve_submit(s, 3, 0, 0.5, 0)
        assert e.value.code == fvv.FVV_EBUSY
        fvv.fvv_serve_set_frames(s, 0, 0, [0] * 5)
        _wait(s, t1)
        assert fvv.fvv_serve_release(s, t1) == 0          # buffer back to the pool
        t3 = fvv.fvv_serve_submit(s, 3, 0, 0.5, 0)
        _wait(s, t3)
        assert fvv.fvv_serve_stats_get(s)["rejected"] == 1
        with pytest.raises(fvv.FvvError) as e:
            fvv.fvv_serve_poll(s, t1)
        assert e.value.code == fvv.FVV_ENOTFOUND
        _wait(s, t2)
    finally:
        fvv.fvv_serve_destroy(s)


def test_continuous_batching_and_latency():
    # 2 slots, batches of up to 4, 5 ms per view; 24 requests from 24 users arrive
    # over ~60 ms from two threads: batches overlap and every request completes
    s = _server(slots_per_res=2, max_batch=4, pool_views=64, fake=5.0)
    fvv.fvv_serve_set_frames(s, 0, 0, [0] * 5)
    tickets = []
    lock = threading.Lock()

    def client(base):
        for k in range(12):
            tk = fvv.fvv_serve_submit(s, base + k, k % 4, 0.5, 0)
            with lock:
                tickets.append(tk)
            time.sleep(0.005)

    th = [threading.Thread(target=client, args=(b,)) for b in (0, 100)]
    [t.start() for t in th]
    [t.join() for t in th]
    try:
        lats = [_wait(s, tk) for tk in tickets]
        st = fvv.fvv_serve_stats_get(s)
        assert st["completed"] == 24 and st["superseded"] == 0
        assert st["batches"] < 24                         # requests were batched
        assert min(lats) >= 5.0 - 0.5                      # at least one view's time
        assert st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        fvv.fvv_serve_destroy(s)


def test_bad_requests():
    s = _server()
    try:
        for args in ((1, 4, 0.5, 0), (1, 0, 1.5, 0), (1, 0, 0.5, 3)):
            with pytest.raises(fvv.FvvError) as e:
                fvv.fvv_serve_submit(s, *args)
            assert e.value.code == fvv.FVV_EINVAL
    finally:
        fvv.fvv_serve_destroy(s)


def test_dense_mode_renders_once_per_instant_and_snaps():
    # 5 cameras -> 4 pairs; n = 2 levels -> 3 views per pair (t = 1/4, 1/2, 3/4);
    # max_batch 6 -> two pairs per render batch
    s = _server(slots_per_res=2, max_batch=6, dense_levels=2, fake=1.0)
    view_bytes = 64 * 64 * 3 * 4
    cams = [0x1000 * (i + 1) for i in range(5)]
    try:
        fvv.fvv_serve_set_frames(s, 0, 0, cams)
        rng = __import__("numpy").random.default_rng(4)
        reqs = []
        for u in range(40):                       # many users, one render
            p, t = int(rng.integers(0, 4)), float(rng.uniform(0, 1))
            reqs.append((fvv.fvv_serve_submit(s, u, p, t, 0), p, t))
        for tk, p, t in reqs:
            _wait(s, tk)
            st, ptr, lat = fvv.fvv_serve_poll(s, tk)
            k = min(4, max(0, round(t * 4)))
            if k == 0:
                assert ptr == cams[p]
            elif k == 4:
                assert ptr == cams[p + 1]
            else:                                  # first store, layout [pair][k - 1]
                assert ptr == (1 << 40) + (p * 3 + k - 1) * view_bytes
        st = fvv.fvv_serve_stats_get(s)
        assert st["dense_instants"] == 1 and st["batches"] == 2 and st["batched_views"] == 12
        assert st["completed"] == 40
        # a new instant renders into the other store; later requests are answered from it
        fvv.fvv_serve_set_frames(s, 1, 0, cams)
        time.sleep(0.05)
        tk = fvv.fvv_serve_submit(s, 99, 2, 0.5, 0)
        _wait(s, tk)
        st2, ptr, lat = fvv.fvv_serve_poll(s, tk)
        assert ptr == (2 << 40) + (2 * 3 + 1) * view_bytes
        st = fvv.fvv_serve_stats_get(s)
        assert st["dense_instants"] == 2 and st["batches"] == 4
    finally:
        fvv.fvv_serve_destroy(s)


def test_dense_mode_needs_whole_pairs_per_batch():
    cfg = fvv.fvv_serve_default_cfg(fake_ms_per_view=1.0, n_res=1, res_h=[64], res_w=[64], n_cams=5,
                                    max_batch=4, dense_levels=3)     # 7 views per pair > 4
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_serve_create(None, cfg)
    assert e.value.code == fvv.FVV_EINVAL


def test_dense_immediate_answers_from_newest_set_with_staleness():
    """dense_immediate: while the newest frames render, requests are answered at once
    from the newest complete set (the older instant), and the stats count how stale
    that content is; once the new set completes, answers come from it (staleness 0)."""
    s = _server(slots_per_res=2, max_batch=6, dense_levels=2, fake=10.0, dense_immediate=1)
    view_bytes = 64 * 64 * 3 * 4
    cams = [0x1000 * (i + 1) for i in range(5)]
    try:
        fvv.fvv_serve_set_frames(s, 0, 0, cams)
        tk = fvv.fvv_serve_submit(s, 1, 0, 0.5, 0)       # no set yet: waits for the first one
        _wait(s, tk)
        assert fvv.fvv_serve_stats_get(s)["dense_instants"] == 1
        fvv.fvv_serve_set_frames(s, 1, 0, cams)           # renders for ~2 x 60 ms
        time.sleep(0.01)
        t0 = time.time()
        tks = [fvv.fvv_serve_submit(s, 10 + u, 1, 0.5, 0) for u in range(8)]
        for tk in tks:
            st, ptr, lat = fvv.fvv_serve_poll(s, tk)      # answered at submit: no waiting
            assert st == 0 and lat < 5.0
            assert ptr == (1 << 40) + (1 * 3 + 1) * view_bytes   # the first store (instant 0)
        assert time.time() - t0 < 0.05
        st = fvv.fvv_serve_stats_get(s)
        assert st["stale_max"] == 1 and st["dense_instants"] == 1
        t1 = time.time()
        while fvv.fvv_serve_stats_get(s)["dense_instants"] < 2:
            assert time.time() - t1 < 5
            time.sleep(0.005)
        tk = fvv.fvv_serve_submit(s, 50, 1, 0.5, 0)
        st, ptr, lat = fvv.fvv_serve_poll(s, tk)
        assert st == 0 and ptr == (2 << 40) + (1 * 3 + 1) * view_bytes
        st = fvv.fvv_serve_stats_get(s)
        assert 0 < st["stale_mean"] < 1 and st["age_p99_ms"] > 0
    finally:
        fvv.fvv_serve_destroy(s)

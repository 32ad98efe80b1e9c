"""Host logic of the single-host elastic schedule (Sec. 5, Alg. 2) with fake
render functions: the camera queue's threshold and timeout, display order
and stale-frame discard, growing and shrinking the worker pool with the
frame rate, and host-made faults (a worker that raises, one that stalls)."""
import threading
import time

import numpy as np

from paper_2502_14938_b300.sched import CameraQueue, DisplaySink, ElasticPool


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def test_queue_threshold_order_and_timeout():
    clk = FakeClock()
    q = CameraQueue(timeout_s=1.0, pose_threshold=0.5, distance=lambda a, b: abs(a - b), clock=clk)
    assert q.put("c0", pose=0.0)
    assert not q.put("c1", pose=0.3)       # moved 0.3 <= 0.5: not queued
    assert q.put("c2", pose=0.9)
    clk.t = 0.5
    assert q.put("c3", pose=2.0)
    assert q.skipped_still == 1 and len(q) == 3
    ts, seq, cam = q.get(0)
    assert cam == "c0" and ts == 0.0        # oldest first
    clk.t = 1.2                             # c2 (t = 0) is now 1.2 s old: dropped
    ts, seq, cam = q.get(0)
    assert cam == "c3" and q.dropped_timeout == 1
    assert q.get(0) is None
    q.close()
    assert q.get(1.0) is None               # closed: returns at once


def test_sink_writes_in_order_and_discards_stale_frames():
    got = []
    s = DisplaySink(write=lambda ts, seq, f: got.append(seq))
    assert s.offer(1.0, 0, "a")
    assert s.offer(3.0, 2, "c")
    assert not s.offer(2.0, 1, "b")         # older than the last written: discarded
    assert s.offer(3.0, 3, "d")             # equal timestamps are written
    assert got == [0, 2, 3] and s.discarded == 1
    ts = [t for t, _ in s.written]
    assert ts == sorted(ts)


def producer(q, rate_hz, seconds, stop):
    dt = 1.0 / rate_hz
    t_end = time.monotonic() + seconds
    i = 0
    while time.monotonic() < t_end and not stop.is_set():
        q.put(i)
        i += 1
        time.sleep(dt)


def sleeper(ms):
    def make(wid):
        def render(cam):
            time.sleep(ms / 1e3)
            return cam
        return render
    return make


def test_pool_grows_below_min_fps():
    """Each worker renders 40 frames/s; cameras arrive at 200/s; min 100 fps
    needs at least 3 workers."""
    q = CameraQueue(timeout_s=0.2)
    s = DisplaySink()
    pool = ElasticPool(sleeper(25), q, s, min_fps=100, max_fps=400, max_workers=6, window_s=0.3, period_s=0.05)
    stop = threading.Event()
    producer(q, 200, 2.5, stop)
    grown = pool.n_workers
    pool.close()
    assert grown >= 3, pool.events
    assert [e for e in pool.events if e[1] == "start"][-1][2] >= 3
    ts = [t for t, _ in s.written]
    assert ts == sorted(ts) and len(ts) > 150
    assert pool.failed == 0


def test_pool_shrinks_above_max_fps():
    """Fast workers (2 ms) and cameras at 100/s: the displayed rate (~100)
    stays above max_fps (1 + 1/N) = 40 (1 + 1/N) for N >= 2, so the pool
    shrinks to one worker."""
    q = CameraQueue(timeout_s=0.2)
    s = DisplaySink()
    pool = ElasticPool(sleeper(2), q, s, min_fps=10, max_fps=40, max_workers=4, start_workers=4,
                       window_s=0.3, period_s=0.05)
    stop = threading.Event()
    producer(q, 100, 2.5, stop)
    n = pool.n_workers
    pool.close()
    assert n == 1, pool.events
    assert sum(1 for e in pool.events if e[1] == "stop") == 3


def test_pool_survives_a_failing_and_a_stalling_worker():
    """Worker 0 raises on its 5th frame (it is retired); worker 1 stalls 0.3 s
    on its 3rd frame, so the frame it then offers is older than frames the
    others wrote meanwhile and is discarded; frames keep being displayed."""
    calls = {}

    def make(wid):
        calls[wid] = 0

        def render(cam):
            calls[wid] += 1
            if wid == 0 and calls[wid] == 5:
                raise RuntimeError("host-made fault")
            if wid == 1 and calls[wid] == 3:
                time.sleep(0.3)
            time.sleep(0.01)
            return cam
        return render

    q = CameraQueue(timeout_s=1.0)
    s = DisplaySink()
    pool = ElasticPool(make, q, s, min_fps=1, max_fps=1000, max_workers=3, start_workers=3,
                       window_s=0.3, period_s=0.05)
    stop = threading.Event()
    producer(q, 150, 1.5, stop)
    pool.close()
    assert pool.failed == 1 and any(e[1] == "fail" for e in pool.events)
    assert s.discarded >= 1
    ts = [t for t, _ in s.written]
    assert ts == sorted(ts) and len(ts) > 60


def test_pool_restarts_when_every_worker_failed():
    def make(wid):
        def render(cam):
            if wid == 0:
                raise RuntimeError("host-made fault")
            return cam
        return render

    q = CameraQueue(timeout_s=1.0)
    s = DisplaySink()
    pool = ElasticPool(make, q, s, min_fps=1, max_fps=1000, max_workers=2, window_s=0.2, period_s=0.02)
    stop = threading.Event()
    producer(q, 100, 0.8, stop)
    pool.close()
    assert pool.failed == 1 and len(s.written) > 20
    assert [e[1] for e in pool.events][:3] == ["start", "fail", "start"]

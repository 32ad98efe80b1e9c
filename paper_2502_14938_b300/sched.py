"""Single-host form of the paper's elastic rendering schedule (Sec. 5, Alg. 2).

The paper runs rendering worker processes on several GPUs behind a shared
camera queue and starts or stops workers as the frame rate drifts.  Here the
workers are threads of one process, each owning its own renderer (its own
library context and CUDA stream on the one GPU), so their frames overlap on
the device; the library releases the GIL inside every call.

- CameraQueue: cameras enter with a timestamp when the pose has moved more
  than a threshold since the last one queued; a worker takes the oldest
  camera that is not older than the timeout (older ones are dropped).
- DisplaySink: frames are written in timestamp order; a frame older than the
  last one written is discarded (Alg. 2, "Timestamp < Last_written").
- ElasticPool: the scheduler measures the displayed frame rate over a
  window; below min_fps it starts a worker (up to max_workers), above
  max_fps (1 + 1/N) it stops one (N = workers running).  A worker whose
  render call raises is retired and counted; the scheduler may start
  another in its place.

Render functions are plain callables (camera -> image), so the host logic is
tested without a GPU; `renderer_worker` builds one from a Renderer.
"""
from __future__ import annotations

import collections
import threading
import time
from typing import Any, Callable, Deque, Dict, List, Optional, Tuple

Clock = Callable[[], float]


class CameraQueue:
    """Timestamped cameras with a pose-change threshold and a timeout."""

    def __init__(self, timeout_s: float, pose_threshold: float = 0.0,
                 distance: Optional[Callable[[Any, Any], float]] = None, clock: Clock = time.monotonic):
        self.timeout = float(timeout_s)
        self.threshold = float(pose_threshold)
        self.distance = distance
        self.clock = clock
        self._q: Deque[Tuple[float, int, Any]] = collections.deque()
        self._cv = threading.Condition()
        self._last_pose = None
        self._seq = 0
        self.dropped_timeout = 0
        self.skipped_still = 0
        self.closed = False

    def put(self, camera: Any, pose: Any = None) -> bool:
        """Queue the camera (stamped now) unless its pose moved no more than the
        threshold since the last queued one.  Returns whether it was queued."""
        with self._cv:
            if self.threshold > 0 and self._last_pose is not None and pose is not None:
                if self.distance(self._last_pose, pose) <= self.threshold:
                    self.skipped_still += 1
                    return False
            if pose is not None:
                self._last_pose = pose
            self._q.append((self.clock(), self._seq, camera))
            self._seq += 1
            self._cv.notify()
            return True

    def get(self, wait_s: float = 0.05) -> Optional[Tuple[float, int, Any]]:
        """(timestamp, sequence, camera) of the oldest camera within the
        timeout, dropping expired ones; None if nothing arrives within wait_s
        or the queue is closed."""
        deadline = time.monotonic() + wait_s
        with self._cv:
            while True:
                now = self.clock()
                while self._q and now - self._q[0][0] > self.timeout:
                    self._q.popleft()
                    self.dropped_timeout += 1
                if self._q:
                    return self._q.popleft()
                if self.closed:
                    return None
                left = deadline - time.monotonic()
                if left <= 0:
                    return None
                self._cv.wait(left)

    def close(self) -> None:
        with self._cv:
            self.closed = True
            self._cv.notify_all()

    def __len__(self) -> int:
        with self._cv:
            return len(self._q)


class DisplaySink:
    """Writes frames in timestamp order; discards frames older than the last
    one written.  write(frame) is called under the sink's lock."""

    def __init__(self, write: Optional[Callable[[float, int, Any], None]] = None, clock: Clock = time.monotonic):
        self.write = write
        self.clock = clock
        self._lock = threading.Lock()
        self.last_ts = float("-inf")
        self.written: List[Tuple[float, int]] = []
        self.write_times: List[float] = []
        self.discarded = 0

    def offer(self, ts: float, seq: int, frame: Any) -> bool:
        with self._lock:
            if ts < self.last_ts:
                self.discarded += 1
                return False
            if self.write is not None:
                self.write(ts, seq, frame)
            self.last_ts = ts
            self.written.append((ts, seq))
            self.write_times.append(self.clock())
            return True

    def fps(self, window_s: float) -> float:
        """Frames written per second over the last window_s seconds."""
        with self._lock:
            now = self.clock()
            n = sum(1 for t in self.write_times if now - t <= window_s)
        return n / window_s


class ElasticPool:
    """Render workers over a CameraQueue into a DisplaySink, grown and shrunk
    by the displayed frame rate (Alg. 2)."""

    def __init__(self, make_render: Callable[[int], Callable[[Any], Any]], queue: CameraQueue, sink: DisplaySink,
                 min_fps: float, max_fps: float, max_workers: int, start_workers: int = 1,
                 window_s: float = 0.5, period_s: float = 0.1):
        assert 0 < min_fps <= max_fps and max_workers >= 1 and 1 <= start_workers <= max_workers
        self.make_render = make_render
        self.queue, self.sink = queue, sink
        self.min_fps, self.max_fps = float(min_fps), float(max_fps)
        self.max_workers = int(max_workers)
        self.window, self.period = float(window_s), float(period_s)
        self._lock = threading.Lock()
        self._workers: Dict[int, Tuple[threading.Thread, threading.Event]] = {}
        self._next_id = 0
        self.failed = 0
        self.events: List[Tuple[float, str, int]] = []  # (time, "start" | "stop" | "fail", workers after)
        self._stop = threading.Event()
        for _ in range(start_workers):
            self._start_worker()
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._sched.start()

    # -- workers
    def _start_worker(self) -> None:
        with self._lock:
            wid = self._next_id
            self._next_id += 1
            stop = threading.Event()
            t = threading.Thread(target=self._work, args=(wid, stop), daemon=True)
            self._workers[wid] = (t, stop)
            self.events.append((time.monotonic(), "start", len(self._workers)))
        t.start()

    def _stop_one(self) -> None:
        with self._lock:
            if len(self._workers) <= 1:
                return
            wid = max(self._workers)  # the newest
            self._workers[wid][1].set()
            del self._workers[wid]
            self.events.append((time.monotonic(), "stop", len(self._workers)))

    def _work(self, wid: int, stop: threading.Event) -> None:
        try:
            render = self.make_render(wid)
            while not stop.is_set() and not self._stop.is_set():
                item = self.queue.get(wait_s=0.05)
                if item is None:
                    if self.queue.closed:
                        break
                    continue
                ts, seq, cam = item
                frame = render(cam)
                self.sink.offer(ts, seq, frame)
        except Exception:
            with self._lock:
                self.failed += 1
                self._workers.pop(wid, None)
                self.events.append((time.monotonic(), "fail", len(self._workers)))

    @property
    def n_workers(self) -> int:
        with self._lock:
            return len(self._workers)

    # -- scheduler
    def _schedule(self) -> None:
        t0 = time.monotonic()
        while not self._stop.wait(self.period):
            n = self.n_workers
            if n == 0 and self.max_workers > 0:  # every worker failed: start one again
                self._start_worker()
                continue
            if time.monotonic() - t0 < self.window:
                continue  # the first window has no rate yet
            fps = self.sink.fps(self.window)
            if fps < self.min_fps and n < self.max_workers:
                self._start_worker()
                t0 = time.monotonic()
            elif fps > self.max_fps * (1.0 + 1.0 / max(n, 1)) and n > 1:
                self._stop_one()
                t0 = time.monotonic()

    def close(self, join_s: float = 5.0) -> None:
        self._stop.set()
        self.queue.close()
        self._sched.join(join_s)
        with self._lock:
            threads = [t for t, _ in self._workers.values()]
        for t in threads:
            t.join(join_s)


def renderer_worker(make_renderer: Callable[[], Any], out_shapes: List[Tuple[int, ...]], dtype=None):
    """make_render for ElasticPool from a Renderer factory: each worker owns a
    renderer and pinned host buffers; a camera item is the list of
    gsc cameras (to_camera) of one frame; the frame is a list of arrays."""
    import numpy as np

    def make(wid: int):
        r = make_renderer()
        bufs = [np.empty(s, dtype or np.float32) for s in out_shapes]

        def render(cams):
            r.set_cameras(cams)
            r.render_frame_host(bufs, stats=False)
            return [b.copy() for b in bufs]
        return render
    return make

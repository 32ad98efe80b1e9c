"""The single-host elastic schedule (Sec. 5, Alg. 2) with real renderers:
worker threads, each with its own context and stream on the one GPU, render
queued cameras; the display receives frames in timestamp order, and every
displayed frame is the image a direct render of its camera gives."""
import threading
import time

import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def orbit(i, w=128, h=96):
    a = 0.01 * i
    R = np.array([[np.cos(a), 0, -np.sin(a)], [0, 1, 0], [np.sin(a), 0, np.cos(a)]])
    return gen.pinhole(R, np.array([0.0, 0.0, -15.0]), w, h, 60.0)


def test_two_workers_display_in_order_and_match_direct_renders():
    import paper_2502_14938_b300 as pkg
    from paper_2502_14938_b300.sched import CameraQueue, DisplaySink, ElasticPool, renderer_worker
    m = gen.tiny_scene()
    made = []

    def make_renderer():
        r = pkg.Renderer(max_views=1, use_graph=True)
        mid = r.load_model(m)
        made.append((r, mid))
        return r

    shown = {}
    q = CameraQueue(timeout_s=0.5)
    sink = DisplaySink(write=lambda ts, seq, frame: shown.__setitem__(seq, frame[0]))
    pool = ElasticPool(renderer_worker(make_renderer, [(96, 128, 3)]), q, sink, min_fps=1, max_fps=1e6,
                       max_workers=2, start_workers=2, window_s=0.3, period_s=0.05)
    cams = {}
    t_end = time.monotonic() + 1.5
    i = 0
    while time.monotonic() < t_end:
        c = orbit(i)
        cams[i] = c
        q.put([pkg.to_camera(c, model_id=0)])
        i += 1
        time.sleep(0.004)
    pool.close()
    assert pool.failed == 0
    ts = [t for t, _ in sink.written]
    assert ts == sorted(ts) and len(ts) > 50
    direct = pkg.Renderer(max_views=1)
    direct.load_model(m)
    for seq in list(shown)[:: max(1, len(shown) // 8)]:
        direct.set_cameras([pkg.to_camera(cams[seq], model_id=0)])
        out = [np.zeros((96, 128, 3), np.float32)]
        direct.render_frame_host(out, stats=False)
        assert np.array_equal(out[0], shown[seq]), f"frame {seq}"
    direct.close()
    for r, _ in made:
        r.close()

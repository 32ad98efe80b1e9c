"""Output formats and pipelined host frames through the C ABI.

RGBA8: every channel is the round-to-nearest-even of 255 x the float32 value
the F32 format would hold (clamped to [0, 1]), alpha that of 1 - T; against
the float64 oracle it is within one level where the oracle's value is not
near a rounding midpoint.  Pipelined host frames (render n+1 while n is
copied) deliver exactly the images of synchronous frames, and report a
deferred overflow."""
import numpy as np
import pytest

import gen
import oracle
from test_gpu_parity import MARGIN, make_renderer

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def quantise_f32(img):
    """The RGBA8 rule applied to a float32 image on the host (float32 multiply, ties to even)."""
    v = np.clip(img.astype(np.float32), np.float32(0), np.float32(1)) * np.float32(255)
    return np.rint(v).astype(np.uint8)


def render_fmt(r, cams, fmt):
    if fmt == "f32":
        outs = [torch.zeros((c.height, c.width, 3), dtype=torch.float32, device="cuda") for c in cams]
    else:
        outs = [torch.zeros((c.height, c.width, 4), dtype=torch.uint8, device="cuda") for c in cams]
    st = r.render_frame(outs)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], st


def test_rgba8_is_the_quantised_f32_image():
    import paper_2502_14938_b300 as pkg
    m, cam = gen.tiny_scene(), gen.tiny_camera()
    rf = make_renderer(m, [cam], flags=pkg.FLAG_DEBUG_T)
    (img,), _ = render_fmt(rf, [cam], "f32")
    T = rf.debug_final_T(0).reshape(cam.height, cam.width)
    r8 = make_renderer(m, [cam], out_format="rgba8")
    (q,), _ = render_fmt(r8, [cam], "rgba8")
    assert q.shape == (cam.height, cam.width, 4)
    assert np.array_equal(q[..., :3], quantise_f32(img))
    assert np.array_equal(q[..., 3], quantise_f32(np.float32(1) - T))
    rf.close()
    r8.close()


@pytest.mark.parametrize("frame", [0, 150])
def test_rgba8_city_within_one_level_of_the_oracle(frame):
    model, frames = gen.city_workload(n_frames=300)
    L, R = frames[frame]
    r = make_renderer(model, [L, R], partners=[1, 0], out_format="rgba8")
    imgs, _ = render_fmt(r, [L, R], "rgba8")
    rs = np.random.default_rng(frame)
    for v, cam in enumerate((L, R)):
        px = rs.integers(0, cam.width, 20000)
        py = rs.integers(0, cam.height, 20000)
        vr = oracle.view_gaussians(model, cam)
        ref, T, mg, _ = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, True, px, py)
        want = np.rint(np.clip(ref, 0, 1) * 255)
        got = imgs[v][py, px, :3].astype(np.float64)
        d = np.abs(got - want)
        ok = mg >= MARGIN
        assert d[ok].max() <= 1, f"frame {frame} eye {v}"
        far = ok[:, None] & (np.abs((np.clip(ref, 0, 1) * 255) % 1 - 0.5) > 0.3)
        assert np.array_equal(got[far], want[far]), f"frame {frame} eye {v}: far from a midpoint"
    r.close()


@pytest.mark.parametrize("fmt", ["f32", "rgba8"])
def test_pipelined_host_frames_equal_synchronous_frames(fmt):
    """Cached BF16 unified form over 8 frames of the path: pipelined host
    frames (from an empty cache) deliver the images of synchronous ones."""
    model, frames = gen.city_workload(n_frames=300)
    import paper_2502_14938_b300 as pkg
    kw = dict(precision="bf16", reuse="depth", stereo_unify=True, out_format=fmt)
    ch = 3 if fmt == "f32" else 4
    dt = torch.float32 if fmt == "f32" else torch.uint8
    L0, R0 = frames[0]
    res = {}
    for mode in ("sync", "async"):
        r = make_renderer(model, [L0, R0], partners=[1, 0], **kw)
        buf = [[torch.zeros((1080, 1920, ch), dtype=dt, pin_memory=True).numpy() for _ in range(2)] for _ in range(8)]
        r.render_frame_host(buf[0])  # grows the buffers
        r.cache_reset()
        for f in range(8):
            L, R = frames[10 * f]
            r.set_cameras([pkg.to_camera(L, partner=1, model_id=0), pkg.to_camera(R, partner=0, model_id=0)])
            if mode == "sync":
                r.render_frame_host(buf[f], stats=False)
            else:
                r.render_frame_host_async(buf[f])
        if mode == "async":
            r.wait_host()
        res[mode] = [np.stack(b) for b in buf]
        r.close()
    for f in range(8):
        assert np.array_equal(res["sync"][f], res["async"][f]), f"frame {f}"
    assert res["async"][7].any()


def test_pipelined_overflow_is_reported():
    import paper_2502_14938_b300 as pkg
    m, cam = gen.tiny_scene(), gen.tiny_camera()
    r = make_renderer(m, [cam], pair_capacity=64)
    out = [torch.zeros((cam.height, cam.width, 3), dtype=torch.float32, pin_memory=True).numpy()]
    r.render_frame_host_async(out)
    with pytest.raises(pkg.GscError) as e:
        r.wait_host()
    assert e.value.code == -4  # GSC_ERR_CAPACITY
    st = r.render_frame_host(out)  # a synchronous frame grows the buffer and renders
    assert st["error_flags"] == 0
    (ref, T, mg, nc), _ = oracle.render_view(m, cam)
    ok = mg >= MARGIN
    assert np.abs(out[0] - ref)[ok].max() < 1e-3
    r.close()

"""Edge cases through the C ABI against the oracle: the largest camera count,
an empty model, degenerate and ragged image sizes, a model that keeps no
Gaussian, and a multi-model frame where one model sees nothing."""
import dataclasses

import numpy as np
import pytest

import gen
import oracle
from test_gpu_parity import check_image, make_renderer, render

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def orbit_camera(i, n, w, h):
    """Camera i of n on a circle of radius 15 around the tiny scene, looking at its centre."""
    a = 2 * np.pi * i / n
    centre = np.array([15 * np.sin(a), 2.0 * np.cos(3 * a), -15 * np.cos(a)])
    f = -centre / np.linalg.norm(centre)
    right = np.cross(np.array([0.0, 1.0, 0.0]), f)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    return gen.pinhole(np.stack([right, down, f]), centre, w, h, 60.0)


def test_largest_camera_count():
    """32 cameras (the library's maximum) in one frame, every image against the oracle."""
    import paper_2502_14938_b300 as pkg
    m = gen.tiny_scene()
    cams = [orbit_camera(i, 32, 64 + 8 * (i % 3), 48 + 4 * (i % 5)) for i in range(pkg.native.MAX_VIEWS)]
    r = make_renderer(m, cams)
    imgs, st = render(r, cams)
    assert st["visible_anchors"] > 0
    for i, cam in enumerate(cams):
        (ref, T, mg, nc), _ = oracle.render_view(m, cam)
        check_image(imgs[i], ref, mg, f"camera {i}")
    with pytest.raises(pkg.GscError):
        pkg.Renderer(max_views=pkg.native.MAX_VIEWS + 1)
    r.close()


def empty_model():
    m = gen.tiny_scene()
    return dataclasses.replace(m, pos=m.pos[:0], feat=m.feat[:0], offs=m.offs[:0], scale=m.scale[:0],
                               level=m.level[:0])


@pytest.mark.parametrize("precision,reuse", [("fp32", "off"), ("bf16", "depth")])
def test_empty_model_renders_background(precision, reuse):
    m = empty_model()
    cam = gen.tiny_camera(100, 70)
    r = make_renderer(m, [cam], bg=(0.1, 0.2, 0.3), precision=precision, reuse=reuse)
    for _ in range(2):
        (img,), st = render(r, [cam])
        assert st["visible_anchors"] == 0 and st["records"] == 0 and st["pairs"] == 0
        assert np.array_equal(img, np.broadcast_to(np.array([0.1, 0.2, 0.3], np.float32), img.shape))
    r.close()


@pytest.mark.parametrize("w,h", [(1, 1), (17, 3), (3, 40), (1023, 9), (255, 257)])
def test_degenerate_and_ragged_image_sizes(w, h):
    m = gen.tiny_scene()
    cam = gen.tiny_camera(w, h)
    r = make_renderer(m, [cam])
    (img,), st = render(r, [cam])
    (ref, T, mg, nc), _ = oracle.render_view(m, cam)
    check_image(img, ref, mg, f"{w}x{h}")
    r.close()


def test_model_that_keeps_no_gaussian():
    """Opacity head biased to alpha <= 0 everywhere: every Gaussian is masked out."""
    m = gen.tiny_scene()
    b2 = [b.copy() for b in m.b2]
    b2[0][:] = -1e4
    m = dataclasses.replace(m, b2=b2)
    cam = gen.tiny_camera(128, 96)
    r = make_renderer(m, [cam], bg=(0.5, 0.5, 0.5))
    (img,), st = render(r, [cam])
    assert st["visible_anchors"] > 0 and st["valid_records"] == 0 and st["pairs"] == 0
    assert np.array_equal(img, np.full(img.shape, 0.5, np.float32))
    r.close()


def test_multi_model_frame_with_an_invisible_model():
    """Two models in one frame; the second model's camera looks away from it."""
    import paper_2502_14938_b300 as pkg
    m0 = gen.tiny_scene(seed=0)
    m1 = gen.tiny_scene(seed=3)
    c0 = gen.tiny_camera(96, 64)
    c1 = gen.tiny_camera(80, 56)
    c1.t = np.array([0, 0, -40.0], np.float32)  # its scene is behind it
    r = pkg.Renderer(max_views=2, bg=(0.0, 0.0, 0.0))
    a = r.load_model(m0)
    b = r.load_model(m1)
    r.set_cameras([pkg.to_camera(c0, model_id=a), pkg.to_camera(c1, model_id=b)])
    imgs, st = render(r, [c0, c1])
    (ref, T, mg, nc), _ = oracle.render_view(m0, c0)
    check_image(imgs[0], ref, mg, "visible model")
    assert not imgs[1].any()
    r.close()

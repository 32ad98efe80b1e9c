"""Octree-GS level selection on the GPU (per-anchor level offsets and the
level fade) against the oracle: visible sets bit-exact, derived attributes
within 1e-5, tile keys and sorted pairs exact, sampled pixels within 1e-3
(threshold-near pixels excepted); the cached unified form's decisions exact
and its images within the cache tolerance of the oracle's simulation."""
from dataclasses import replace

import numpy as np
import pytest

import gen
import oracle
from oracle.cache import CacheSim, cached_derive, project_view
from test_gpu_cache import CACHED_PIX_TOL, gpu_lines, set_cams
from test_gpu_parity import check_attrs, check_image, check_keygen_and_sort, make_renderer, render

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def city_octree():
    model, frames = gen.city_workload()
    return gen.with_level_offsets(model, sigma=0.5, beta=0.5), frames


def sample_pixels(rs, cam, n=20000):
    return rs.integers(0, cam.width, n), rs.integers(0, cam.height, n)


@pytest.mark.parametrize("frame", [0, 299])
def test_city_octree_stereo_frame(city_octree, frame):
    import paper_2502_14938_b300 as pkg
    model, frames = city_octree
    L, R = frames[frame]
    r = make_renderer(model, [L, R], partners=[1, 0], flags=pkg.FLAG_DEBUG_ATTRS)
    imgs, st = render(r, [L, R])
    plain = replace(model, level_offset=None, lod_blend=0.0)
    rs = np.random.default_rng(frame)
    for v, cam in enumerate((L, R)):
        ids = oracle.cull(model, cam)
        assert np.array_equal(r.debug_visible(v), ids), f"eye {v} visible set"
        assert not np.array_equal(ids, oracle.cull(plain, cam))  # the offsets change the set
        attrs, _ = oracle.derive(model, oracle.camera_center(cam), ids)
        check_attrs(r.debug_attrs(v), attrs, model.scale[ids], f"octree eye {v}")  # before the fade
        w = oracle.lod_weight(model, cam, ids)
        assert (w < 1).sum() > 100  # the fade is active on this frame
    check_keygen_and_sort(r, [L, R])
    for v, cam in enumerate((L, R)):
        px, py = sample_pixels(rs, cam)
        vr = oracle.view_gaussians(model, cam)
        ref, T, mg, nc = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, True, px, py)
        check_image(imgs[v][py, px], ref, mg, f"octree f{frame} eye {v}")
    r.close()


def test_zero_offsets_keep_the_plain_sets(city_octree):
    """Zero offsets with a fade take the radius path on the GPU; its visible
    set is the plain rule's, as the oracle's plain cull computes it."""
    model, frames = city_octree
    m0 = replace(model, level_offset=np.zeros(model.n, np.float32), lod_blend=0.25)
    L, R = frames[150]
    r = make_renderer(m0, [L, R], partners=[1, 0])
    render(r, [L, R])
    plain = replace(model, level_offset=None, lod_blend=0.0)
    for v, cam in enumerate((L, R)):
        assert np.array_equal(r.debug_visible(v), oracle.cull(plain, cam)), v
    r.close()


def test_cached_unified_octree_path(city_octree):
    """The fade is applied after the cache (it depends on this frame's
    distance): cached lines hold unfaded attributes and every frame's
    records fade them anew."""
    model, frames = city_octree
    L0, R0 = frames[0]
    r = make_renderer(model, [L0, R0], partners=[1, 0], reuse="depth", stereo_unify=True)
    sim = CacheSim(model.n, (4 << 20) // 10, max_depth=10)
    rs = np.random.default_rng(7)
    hits = 0
    for f in range(0, 27):
        L, R = frames[f]
        set_cams(r, [L, R], [1, 0])
        imgs, st = render(r, [L, R])
        U = oracle.unified_camera(L, R)
        ids, attrs, kept, hit, line, used = cached_derive(model, U, sim)
        assert np.array_equal(r.debug_visible(0), ids), f
        ghit, gline = gpu_lines(r.debug_cache(0)[0])
        assert np.array_equal(ghit, hit) and np.array_equal(gline, line), f
        hits += int(hit.sum())
        if f % 13 == 12:
            for v, cam in enumerate((L, R)):
                px, py = sample_pixels(rs, cam)
                vr = project_view(model, cam, ids, attrs, kept, derive_cam=U)
                ref, _, mg, _ = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, True, px, py)
                check_image(imgs[v][py, px], ref, mg, f"cached octree frame {f} eye {v}", CACHED_PIX_TOL)
    assert hits > 0
    r.close()


def test_cached_exact_stereo_octree_path(city_octree):
    """The exact stereo form with level offsets and the fade: each eye's own
    radius rule selects its anchors (masks bit-exact) and the fade of an eye
    is measured from that eye; decisions exact, images within the cache
    tolerance of the oracle's simulation."""
    model, frames = city_octree
    L0, R0 = frames[0]
    r = make_renderer(model, [L0, R0], partners=[1, 0], reuse="depth", stereo_unify="exact")
    sim = CacheSim(model.n, (4 << 20) // 10, max_depth=10)
    rs = np.random.default_rng(8)
    for f in range(0, 14):
        L, R = frames[f]
        set_cams(r, [L, R], [1, 0])
        imgs, st = render(r, [L, R])
        U = oracle.unified_camera(L, R)
        union, eyes = oracle.cull_pair(model, L, R)
        ids, attrs, kept, hit, line, used = cached_derive(model, U, sim, ids=union)
        assert np.array_equal(r.debug_visible(0), ids) and np.array_equal(r.debug_visible_eyes(0), eyes), f
        ghit, gline = gpu_lines(r.debug_cache(0)[0])
        assert np.array_equal(ghit, hit) and np.array_equal(gline, line), f
        if f % 13 in (0, 12):
            for v, cam in enumerate((L, R)):
                px, py = sample_pixels(rs, cam)
                vr = project_view(model, cam, ids, attrs, kept, mine=(eyes >> v) & 1)
                ref, _, mg, _ = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, True, px, py)
                check_image(imgs[v][py, px], ref, mg, f"cached exact octree frame {f} eye {v}", CACHED_PIX_TOL)
    r.close()


def test_invalid_level_offsets_are_rejected():
    import paper_2502_14938_b300 as pkg
    m = gen.tiny_scene(n=64)
    for bad in (np.full(64, np.nan, np.float32), np.full(64, 9.0, np.float32)):
        r = pkg.Renderer(max_views=1)
        with pytest.raises(pkg.GscError):
            r.load_model(replace(m, level_offset=bad))
        r.close()
    r = pkg.Renderer(max_views=1)
    with pytest.raises(pkg.GscError):
        r.load_model(replace(m, lod_blend=-1.0))
    r.close()

"""Batched multi-viewer frames on the GPU against the oracle.

Three city scenes and eight viewers (five stereo pairs and three mono views,
13 images) render as ONE frame: one cull over every derivation view, one
derivation, one projection, two sorts and one blend over all images.  Each
image must equal what the oracle gives for that image alone (the de-redundant
stereo form of Eq. 5-6 for the pairs), under every supported tile shape and
with the blend run one block per tile or as a persistent kernel.  The
full-size test runs the whole form (BF16 derivation, cache, unified stereo)
with the autotuned tiling and checks the visible sets and cache decisions of
every derivation view bit for bit against the oracle's simulation.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle.cache import CacheSim, cached_derive
from test_gpu_parity import check_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LINE_HIT = 0x80000000
LINE_NONE = 0x7FFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def batched_renderer(models, images, **kw):
    """One context holding every scene; cameras in frame order with their
    scene's model id, viewer and stereo partner."""
    import paper_2502_14938_b300 as pkg
    r = pkg.Renderer(max_views=len(images), **kw)
    mids = [r.load_model(m) for m in models]
    set_frame(r, mids, images)
    return r, mids


def set_frame(r, mids, images):
    import paper_2502_14938_b300 as pkg
    r.set_cameras([pkg.to_camera(c, partner=p, model_id=mids[s], viewer=v) for v, s, c, p in images])


def render_all(r, images):
    outs = [torch.zeros((c.height, c.width, 3), dtype=torch.float32, device="cuda") for _, _, c, _ in images]
    st = r.render_frame(outs)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], st


def derive_camera(images, i):
    """Camera whose anchors and view direction image i uses (unified for pairs)."""
    _, _, c, p = images[i]
    if p < 0:
        return c
    a, b = (i, p) if i < p else (p, i)
    return oracle.unified_camera(images[a][2], images[b][2])


def dview_images(r, images):
    """(derivation view index, first image) in the GPU's derivation-view order."""
    nd, first = r.debug_dviews()
    assert nd == len({v for v, _, _, _ in images})
    return list(enumerate(first))


def gpu_lines(vstat):
    hit = (vstat & LINE_HIT) != 0
    line = (vstat & ~np.uint32(LINE_HIT)).astype(np.int64)
    line[line == LINE_NONE] = -1
    return hit, line


# ------------------------------------------------------------------ reduced scale: whole images
@pytest.fixture(scope="module")
def small():
    models, viewers, frame_fn = gen.multiviewer_workload(scale=0.02, size_scale=0.25)
    images = frame_fn(40)
    refs = []
    for i, (v, s, c, p) in enumerate(images):
        vr = oracle.view_gaussians(models[s], c, derive_cam=derive_camera(images, i))
        ref, T, mg, nc = oracle.render(vr.rec, vr.depth32, vr.gid, c.width, c.height, True)
        refs.append((ref, mg))
    return models, images, refs


def test_batched_frame_every_image_matches_oracle(small):
    import paper_2502_14938_b300 as pkg
    models, images, refs = small
    r, mids = batched_renderer(models, images, stereo_unify=True, flags=pkg.FLAG_DEBUG_ATTRS)
    imgs, st = render_all(r, images)
    for d, first in dview_images(r, images):
        _, s, _, _ = images[first]
        U = derive_camera(images, first)
        ids = oracle.cull(models[s], U)
        assert np.array_equal(r.debug_visible(d), ids), f"derivation view {d} visible set"
    assert st["visible_anchors"] == sum(len(r.debug_visible(d)) for d, _ in dview_images(r, images))
    for i, (img, (ref, mg)) in enumerate(zip(imgs, refs)):
        check_image(img, ref, mg, f"batched image {i}")
    r.close()


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (16, 8), (8, 16), (32, 16), (16, 32), (32, 32), (8, 32),
                                  (16, 64), (8, 64), (8, 128)])
def test_batched_tilings_and_persistent_blend(small, tile):
    """Every tile shape, one block per tile and persistent: each image within
    tolerance of the oracle; persistent and per-tile blends bit-identical
    (same tile, same arithmetic, only the tile-to-block mapping differs)."""
    models, images, refs = small
    r, _ = batched_renderer(models, images, stereo_unify=True, tile=tile)
    per_tile, _ = render_all(r, images)
    for bps in (1, 4, 32):
        r.set_tiling(tile[0], tile[1], bps)
        pers, _ = render_all(r, images)
        for i in range(len(images)):
            assert np.array_equal(pers[i], per_tile[i]), f"tile {tile} bps {bps} image {i}"
    for i, (img, (ref, mg)) in enumerate(zip(per_tile, refs)):
        check_image(img, ref, mg, f"tile {tile} image {i}")
    r.close()


def test_set_tiling_rejects_unsupported_shapes(small):
    import paper_2502_14938_b300 as pkg
    models, images, _ = small
    r, _ = batched_renderer(models, images)
    for tw, th, bps in [(24, 16, 0), (16, 12, 0), (8, 8, 0), (32, 64, 0), (4, 64, 0), (16, 16, 33)]:
        with pytest.raises(pkg.GscError):
            r.set_tiling(tw, th, bps)
    r.set_tiling(16, 16, 0)  # still usable after the rejections
    render_all(r, images)
    r.close()


def test_autotuner_persists_its_choice(small, tmp_path):
    from paper_2502_14938_b300 import autotune
    models, images, refs = small
    r, _ = batched_renderer(models, images, stereo_unify=True)
    outs = [torch.zeros((c.height, c.width, 3), dtype=torch.float32, device="cuda") for _, _, c, _ in images]
    path = str(tmp_path / "tiling.json")
    best = autotune.tune(r, outs, path, shapes=[(16, 16), (32, 8)], blocks=[0, 4], reps=2)
    assert best["source"] == "sweep"
    again = autotune.tune(r, outs, path)
    assert again["source"] == "cache"
    assert (again["tile_w"], again["tile_h"], again["blocks_per_sm"]) == \
        (best["tile_w"], best["tile_h"], best["blocks_per_sm"])
    imgs, _ = render_all(r, images)
    for i, (img, (ref, mg)) in enumerate(zip(imgs, refs)):
        check_image(img, ref, mg, f"tuned image {i}")
    r.close()


# ------------------------------------------------------------------ full size, the whole form
@pytest.fixture(scope="module")
def full():
    return gen.multiviewer_workload()


def test_batched_full_size_cached_bf16_form(full):
    """3 scenes (0.5M / 2M / 4M anchors), 8 viewers, 13 images up to 1080p
    stereo; BF16 derivation, cache and unified stereo; persistent blend.
    Visible sets and cache hit / line / depth decisions bit-exact for every
    derivation view over four frames; every image >= 40 dB against the plain
    float64 oracle on sampled pixels."""
    models, viewers, frame_fn = full
    images = frame_fn(0)
    r, mids = batched_renderer(models, images, stereo_unify=True, precision="bf16", reuse="depth")
    r.set_tiling(16, 16, 8)
    quant = oracle.OrcQuant()
    quant.mode = 1
    sims = {}
    rs = np.random.default_rng(4)
    for t in range(4):
        images = frame_fn(t)
        set_frame(r, mids, images)
        imgs, st = render_all(r, images)
        derived = 0
        for d, first in dview_images(r, images):
            v, s, _, _ = images[first]
            sim = sims.setdefault(v, CacheSim(models[s].n, (4 << 20) // 10, max_depth=10))
            U = derive_camera(images, first)
            ids, attrs, kept, hit, line, used = cached_derive(models[s], U, sim, quant)
            assert np.array_equal(r.debug_visible(d), ids), f"frame {t} dview {d} visible"
            vstat, cst = r.debug_cache(d)
            ghit, gline = gpu_lines(vstat)
            assert np.array_equal(ghit, hit) and np.array_equal(gline, line), f"frame {t} dview {d} lines"
            assert cst["depth"] == sim.depth, f"frame {t} dview {d} depth"
            derived += int((~hit).sum())
        assert st["derived_anchors"] == derived
        if t == 3:
            assert derived < st["visible_anchors"]  # the cache is reused
            for i, (v, s, c, p) in enumerate(images):
                px = rs.integers(0, c.width, 4000)
                py = rs.integers(0, c.height, 4000)
                pv = oracle.view_gaussians(models[s], c)
                plain, _, _, _ = oracle.render(pv.rec, pv.depth32, pv.gid, c.width, c.height, True, px, py)
                q = oracle.psnr(imgs[i][py, px], plain)
                assert q >= 40.0, f"image {i}: {q:.2f} dB"
    r.close()


def test_batched_full_size_persistent_equals_per_tile(full):
    models, viewers, frame_fn = full
    images = frame_fn(150)
    r, _ = batched_renderer(models, images, stereo_unify=True, precision="bf16")
    a, _ = render_all(r, images)
    r.set_tiling(16, 16, 8)
    b, st = render_all(r, images)
    assert st["error_flags"] == 0
    for i in range(len(images)):
        assert np.array_equal(a[i], b[i]), f"image {i}"
    r.close()

"""The blend's work counters (GSC_FLAG_BLEND_WORK) against the oracle.

walk = the (pixel, Gaussian) evaluations of the method's front-to-back walk:
a pixel evaluates every Gaussian of its tile's list until the one at which it
stops (T would fall below 1e-4), that one included.  A pixel that never stops
walks its whole list, so where the oracle shows that no pixel stops, walk is
exactly sum over tiles of (list length x pixels of the tile in the image).
Where some pixels stop, the oracle says which (a stopped pixel ends with
T < 1e-2, since alpha <= 0.99; the brute-force walk confirms it), and the
count must lie between the walk with every stopped pixel ending at its first
Gaussian and the walk with none stopping.  issued = the pixel slots the
kernel ran (4 per lane of a warp per Gaussian whose box meets the warp's
rows) is a multiple of 128 and at most list length x tile pixels per tile.
The counting variant renders the image of the plain one, bit for bit."""
import dataclasses

import numpy as np
import pytest

import gen
import oracle
from test_gpu_parity import MARGIN, make_renderer, render

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILINGS = [(16, 16, 0), (16, 32, 0), (32, 8, 0), (16, 32, 8)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def tile_lengths(r, cam, tw, th):
    """GPU list length of each pixel's tile, [H, W], and the per-tile lengths."""
    lens = (lambda rg: (rg[:, 1].astype(np.int64) - rg[:, 0]))(r.debug_ranges())
    ntx = (cam.width + tw - 1) // tw
    ty = np.arange(cam.height) // th
    tx = np.arange(cam.width) // tw
    return lens[ty[:, None] * ntx + tx[None, :]], lens


def opacity_head(m, s, shift=0.0):
    """The opacity head's last layer scaled by s, its bias shifted by shift."""
    W2 = [w.copy() for w in m.W2]
    b2 = [b.copy() for b in m.b2]
    W2[0] *= s
    b2[0] = b2[0] * s + shift
    return dataclasses.replace(m, W2=W2, b2=b2)


def faint(m):
    """Every alpha at most ~0.7: no pixel of the tiny frame stops."""
    return opacity_head(m, 0.2)


def dense(m):
    """More and stronger Gaussians: some pixels of the tiny frame stop."""
    return opacity_head(m, 2.0, 1.0)


def render_counted(m, cam, tiling):
    import paper_2502_14938_b300 as pkg
    r = make_renderer(m, [cam], flags=pkg.FLAG_BLEND_WORK)
    r.set_tiling(*tiling)
    (img,), st = render(r, [cam])
    walk, issued = r.debug_blend_work()
    per_pix, lens = tile_lengths(r, cam, tiling[0], tiling[1])
    r0 = make_renderer(m, [cam])
    r0.set_tiling(*tiling)
    (img0,), _ = render(r0, [cam])
    r0.close()
    r.close()
    assert np.array_equal(img, img0), "the counting variant changed the image"
    assert issued % 128 == 0
    assert issued <= int(lens.sum()) * tiling[0] * tiling[1]
    return walk, issued, per_pix


@pytest.mark.parametrize("tiling", TILINGS)
def test_walk_is_the_whole_lists_when_no_pixel_stops(tiling):
    m, cam = faint(gen.tiny_scene()), gen.tiny_camera()
    (ref, T, mg, nc), _ = oracle.render_view(m, cam)
    assert T.min() > 1e-2  # no pixel stops
    walk, issued, per_pix = render_counted(m, cam, tiling)
    assert walk == int(per_pix.sum())
    assert 0 < issued


@pytest.mark.parametrize("tiling", TILINGS)
def test_walk_brackets_the_oracle_stops(tiling):
    m, cam = dense(gen.tiny_scene()), gen.tiny_camera()
    vr = oracle.view_gaussians(m, cam)
    ref, T, mg, nc = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, True,
                                   TW=tiling[0], TH=tiling[1])
    cand = np.argwhere(T < 1e-2)
    n_valid = int((vr.rec[:, 0] > 0).sum())
    stopped = np.zeros(T.shape, bool)
    if len(cand):
        _, _, _, _, wk = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, False,
                                       cand[:, 1], cand[:, 0], walk=True)
        stopped[cand[:, 0], cand[:, 1]] = wk < n_valid
    assert stopped.any(), "the tiny frame should have pixels that stop"
    walk, issued, per_pix = render_counted(m, cam, tiling)
    sure = (~stopped) & (mg >= MARGIN)
    lo = int(per_pix[sure].sum()) + int((per_pix[~sure] > 0).sum())
    hi = int(per_pix.sum())
    assert lo <= walk <= hi
    assert hi - walk > 0  # the stopped pixels walked less than their lists


def test_pipe_rates_are_plausible():
    """The unit-throughput probe returns rates within the device's reach:
    below SMs x clock x (32 exp2 | 128 FMA lanes) and not absurdly low."""
    import paper_2502_14938_b300 as pkg
    r = pkg.native.pipe_rates()
    p = torch.cuda.get_device_properties(0)
    clk = 2.2e9  # above any B300 SM clock
    n = p.multi_processor_count
    assert 0.1 * n * 16 * 1e9 < r["exp2_per_s"] <= n * 32 * clk
    assert 0.1 * n * 128 * 1e9 < r["ffma_lane_ops_per_s"] <= n * 128 * clk
    assert 0.1 * n * 128 * 1e9 < r["ffma2_lane_ops_per_s"] <= n * 128 * clk

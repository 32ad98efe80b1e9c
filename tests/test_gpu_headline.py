"""Parity of the exact configuration the frame-rate headline is measured on:
the city model, stereo 1920x1080, cached derivation shared by the two eyes
through the unified stereo camera (Sec. 4, Eq. 4-6) and BF16 tensor-core
MLPs, blended on 16x64 tiles (the tiling the autotuner picks for it).  Both
stereo readings are covered: "exact" (each eye filters its own anchors, the
union is derived once; the headline) and "unified" (Eq. 6's camera filters
for both eyes).

- Cache decisions (hit / line per visible anchor, next reuse depth) are
  bit-exact against the oracle's simulation of Alg. 1 over every rendered
  frame of the path.
- Tile counts, (tile, record) pairs in (tile, depth, Gaussian id) order and
  tile ranges are bit-exact, stage-isolated on the GPU's own float32 records
  through the oracle's float32 coverage at 16x64.
- Pixels: the float32 variant of the same form against the oracle's
  cached-form images within the float16 line tolerance (2e-3) on decided
  pixels; the BF16 headline against the oracle's BF16 cached-form images
  (inputs, weights and hidden values rounded to bf16, sums in float64) and
  >= 40 dB against the plain float64 oracle.
- The float32 mean position error of projected Gaussians stays inside the
  term the oracle's decision margin allows for it.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle.cache import CacheSim, cached_derive, project_view
from test_gpu_cache import CACHED_PIX_TOL, gpu_lines, set_cams
from test_gpu_parity import MARGIN, check_image, check_keygen_and_sort, make_renderer, render

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILING = (16, 64, 0)
LINES = (4 << 20) // 10  # cache capacity of the headline form: 4M Gaussians
# BF16 against the oracle's BF16 derivation: the two round hidden values from
# float32 and float64 sums, so an occasional bf16 rounding flips and moves
# the attributes it feeds by up to 1e-2 of their scale, which bounds every
# decided pixel; all but a rare few agree within the float16 line tolerance.
BF16_PIX_CLOSE = 2e-3
BF16_PIX_CLOSE_FRAC = 0.999
BF16_PIX_MAX = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def city():
    return gen.city_workload()


def bf16_quant():
    q = oracle.OrcQuant()
    q.mode = 1
    return q


def sample_pixels(rs, cam, n=20000):
    px = rs.integers(0, cam.width, n)
    py = rs.integers(0, cam.height, n)
    # plus the ragged bottom row of 16x64 tiles (1080 = 16 x 64 + 56) at the right edge
    tx, ty = np.meshgrid(np.arange(16), np.arange(1024, 1080))
    return np.r_[px, (cam.width - 16) + tx.ravel()], np.r_[py, ty.ravel()]


@pytest.mark.parametrize("stereo,precision,start,n", [("exact", "bf16", 0, 40), ("exact", "bf16", 150, 8),
                                                      ("exact", "bf16", 172, 10), ("exact", "bf16", 292, 8),
                                                      ("exact", "fp32", 0, 12), ("exact", "fp32", 292, 8),
                                                      ("unified", "bf16", 0, 12), ("unified", "fp32", 292, 8)])
def test_headline_form_at_16x64(city, stereo, precision, start, n):
    model, frames = city
    L0, R0 = frames[start]
    r = make_renderer(model, [L0, R0], partners=[1, 0], reuse="depth", stereo_unify=stereo, precision=precision)
    r.set_tiling(*TILING)
    sim = CacheSim(model.n, LINES, max_depth=10)
    quant = bf16_quant() if precision == "bf16" else None
    rs = np.random.default_rng(100 + start)
    hits = 0
    for f in range(start, start + n):
        L, R = frames[f]
        set_cams(r, [L, R], [1, 0])
        imgs, st = render(r, [L, R])
        U = oracle.unified_camera(L, R)
        eyes = None
        if stereo == "exact":
            union, eyes = oracle.cull_pair(model, L, R)
            ids, attrs, kept, hit, line, used = cached_derive(model, U, sim, quant, ids=union)
            assert np.array_equal(r.debug_visible_eyes(0), eyes), f
        else:
            ids, attrs, kept, hit, line, used = cached_derive(model, U, sim, quant)
        assert np.array_equal(r.debug_visible(0), ids), f
        ghit, gline = gpu_lines(r.debug_cache(0)[0])
        assert np.array_equal(ghit, hit) and np.array_equal(gline, line), f
        assert r.debug_cache(0)[1]["depth"] == sim.depth, f
        hits += int(hit.sum())
        if f not in (start, start + n - 1):
            continue
        n_pairs = check_keygen_and_sort(r, [L, R], TILING[0], TILING[1])
        assert n_pairs == st["pairs"] > 0
        for v, cam in enumerate((L, R)):
            px, py = sample_pixels(rs, cam)
            vr = project_view(model, cam, ids, attrs, kept, mine=None if eyes is None else (eyes >> v) & 1)
            ref, _, mg, _ = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, True, px, py)
            got = imgs[v][py, px]
            tag = f"{precision} cached {stereo} 16x64 frame {f} eye {v}"
            if precision == "fp32":
                check_image(got, ref, mg, tag, CACHED_PIX_TOL)
            else:
                ok = mg >= MARGIN
                err = np.abs(got.astype(np.float64) - ref)[ok].max(axis=-1)
                close = float(np.mean(err <= BF16_PIX_CLOSE))
                print(f"{tag}: {close:.5f} of decided pixels within {BF16_PIX_CLOSE}, worst {err.max():.3e}")
                assert close >= BF16_PIX_CLOSE_FRAC and err.max() <= BF16_PIX_MAX, tag
            pv = oracle.view_gaussians(model, cam)
            plain, _, _, _ = oracle.render(pv.rec, pv.depth32, pv.gid, cam.width, cam.height, True, px, py)
            p = oracle.psnr(got, plain)
            assert p >= 40.0, f"{tag}: {p:.2f} dB against the plain float64 oracle"
    assert hits > 0
    r.close()


def test_float32_mean_error_within_the_margin_term(city):
    """The oracle's decision margin for alpha >= 1/255 subtracts
    |grad_mean(q/2)|_1 x e_mean, e_mean (record slot 15) the distance a
    float32 projection can move the 2D mean.  Measured here: every valid
    record of three city frames (plain form, both eyes) has its GPU mean
    within e_mean of the oracle's float64 mean."""
    model, frames = city
    worst = 0.0
    for f in (0, 150, 299):
        L, R = frames[f]
        r = make_renderer(model, [L, R], partners=[1, 0])
        render(r, [L, R])
        rec, key, cnt = r.debug_records()
        base = 0
        for v, cam in enumerate((L, R)):
            ids = r.debug_visible(v)
            nv = len(ids) * model.k
            vr = oracle.view_gaussians(model, cam)
            assert np.array_equal(vr.ids, ids)
            g = slice(base, base + nv)
            ok = (key[g] != 0xFFFFFFFF) & (vr.rec[:, 0] != 0)
            mx, my = rec[g, 0][ok].astype(np.float64), rec[g, 1][ok].astype(np.float64)
            err = np.maximum(np.abs(mx - vr.rec[ok, 1]), np.abs(my - vr.rec[ok, 2]))
            ratio = err / vr.rec[ok, 15]
            worst = max(worst, float(ratio.max()))
            assert ok.sum() > 1000
            assert ratio.max() <= 1.0, (f"frame {f} eye {v}: mean error {ratio.max():.3f} x e_mean "
                                        f"at record {np.argmax(ratio)}")
            base += nv
        r.close()
    print(f"worst float32 mean error: {worst:.3f} x e_mean")

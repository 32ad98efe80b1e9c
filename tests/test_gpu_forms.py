"""The precision form of the derivation (tcgen05 tensor cores, BF16 inputs,
FP32 accumulation) against the oracle.

- Culling, keys, sort and ranges stay integer work: bit-exact as in the
  plain form (same checks, stage-isolated on the GPU's own records).
- Derived attributes against the oracle's BF16-quantised derivation (inputs,
  weights and hidden activations rounded to bf16, sums in float64): within
  1e-2 of each attribute's scale - the two round the hidden activations from
  float32 vs float64 sums, so an occasional bf16 rounding flips.
- Images against the plain float64 oracle: PSNR >= 40 dB (the form's
  quality bar) and the per-pixel error reported.
"""
import numpy as np
import pytest

import gen
import oracle
from test_gpu_parity import check_keygen_and_sort, make_renderer, render

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def bf16_quant():
    q = oracle.OrcQuant()
    q.mode = 1
    return q


def check_attrs_loose(got, ref, s_a, tol, tag):
    scale = np.ones(ref.shape, np.float64)
    scale[..., 4:7] = np.asarray(s_a, np.float64)[:, None, None]
    rel = np.abs(got.astype(np.float64) - ref) / scale
    assert rel.max() <= tol, f"{tag}: worst {rel.max():.3e} at {np.unravel_index(np.argmax(rel), rel.shape)}"
    return rel.max()


def test_bf16_tiny_scene():
    import paper_2502_14938_b300 as pkg
    m, cam = gen.tiny_scene(), gen.tiny_camera()
    r = make_renderer(m, [cam], flags=pkg.FLAG_DEBUG_ATTRS, precision="bf16")
    (img,), st = render(r, [cam])
    ids = oracle.cull(m, cam)
    assert np.array_equal(r.debug_visible(0), ids)
    attrs_q, _ = oracle.derive(m, oracle.camera_center(cam), ids, bf16_quant())
    check_attrs_loose(r.debug_attrs(0), attrs_q, m.scale[ids], 1e-2, "bf16 tiny")
    check_keygen_and_sort(r, [cam])
    (ref, T, mg, nc), _ = oracle.render_view(m, cam)
    assert oracle.psnr(img, ref) >= 40.0
    r.close()


@pytest.fixture(scope="module")
def city():
    return gen.city_workload()


@pytest.mark.parametrize("frame", [0, 299])
def test_bf16_city_stereo(city, frame):
    import paper_2502_14938_b300 as pkg
    model, frames = city
    L, R = frames[frame]
    r = make_renderer(model, [L, R], partners=[1, 0], flags=pkg.FLAG_DEBUG_ATTRS, precision="bf16")
    imgs, st = render(r, [L, R])
    for v, cam in enumerate((L, R)):
        ids = oracle.cull(model, cam)
        assert np.array_equal(r.debug_visible(v), ids)
        attrs_q, _ = oracle.derive(model, oracle.camera_center(cam), ids, bf16_quant())
        check_attrs_loose(r.debug_attrs(v), attrs_q, model.scale[ids], 1e-2, f"bf16 city eye {v}")
    check_keygen_and_sort(r, [L, R])
    rs = np.random.default_rng(frame + 1)
    for v, cam in enumerate((L, R)):
        px = rs.integers(0, cam.width, 30000)
        py = rs.integers(0, cam.height, 30000)
        vr = oracle.view_gaussians(model, cam)
        ref, _, _, _ = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, True, px, py)
        p = oracle.psnr(imgs[v][py, px], ref)
        assert p >= 40.0, f"bf16 city frame {frame} eye {v}: {p:.2f} dB"
    r.close()


def test_bf16_and_fp32_agree_on_integer_stages(city):
    """The precision form changes only derived values: visible sets are identical."""
    model, frames = city
    L, R = frames[150]
    r32 = make_renderer(model, [L, R], partners=[1, 0])
    r16 = make_renderer(model, [L, R], partners=[1, 0], precision="bf16")
    render(r32, [L, R])
    render(r16, [L, R])
    for v in range(2):
        assert np.array_equal(r32.debug_visible(v), r16.debug_visible(v))
    r32.close()
    r16.close()


# ------------------------------------------------------------------ FP8-E4M3
# One E4M3 step is 2^-3 relative: an input value that lies near an E4M3
# rounding midpoint rounds one way from the GPU's float32 and the other from
# the oracle's float64 (the inputs are one term), and moves the outputs it
# feeds by up to a few 1e-2; a hidden value's two-term expansion absorbs such
# a flip in its second term.  Most attributes agree to float32 accuracy; the
# test bounds the share that does not and the size of the rest.
FP8_CLOSE = 1e-4      # scale-relative agreement of an attribute
FP8_CLOSE_FRAC = 0.999  # share of attributes that must agree that closely
FP8_MAX = 1e-2        # bound on any attribute's scale-relative difference
FP8_PSNR = 40.0       # the form against the plain float64 oracle


def check_attrs_fp8(got, ref, s_a, tag):
    scale = np.ones(ref.shape, np.float64)
    scale[..., 4:7] = np.asarray(s_a, np.float64)[:, None, None]
    rel = np.abs(got.astype(np.float64) - ref) / scale
    close = np.mean(rel <= FP8_CLOSE)
    print(f"{tag}: {close:.4f} of attributes within {FP8_CLOSE}, worst {rel.max():.3e}")
    assert close >= FP8_CLOSE_FRAC and rel.max() <= FP8_MAX, f"{tag}: close {close:.3f}, worst {rel.max():.3e}"
    return close, rel.max()


def test_fp8_tiny_scene():
    import paper_2502_14938_b300 as pkg
    m, cam = gen.tiny_scene(), gen.tiny_camera()
    r = make_renderer(m, [cam], flags=pkg.FLAG_DEBUG_ATTRS, precision="fp8")
    (img,), st = render(r, [cam])
    ids = oracle.cull(m, cam)
    assert np.array_equal(r.debug_visible(0), ids)
    attrs_q, _ = oracle.derive(m, oracle.camera_center(cam), ids, oracle.fp8_scales(m))
    check_attrs_fp8(r.debug_attrs(0), attrs_q, m.scale[ids], "fp8 tiny")
    check_keygen_and_sort(r, [cam])
    (ref, T, mg, nc), _ = oracle.render_view(m, cam)
    assert oracle.psnr(img, ref) >= FP8_PSNR
    r.close()


@pytest.mark.parametrize("frame", [0, 150, 299])
def test_fp8_city_stereo(city, frame):
    import paper_2502_14938_b300 as pkg
    model, frames = city
    L, R = frames[frame]
    r = make_renderer(model, [L, R], partners=[1, 0], flags=pkg.FLAG_DEBUG_ATTRS, precision="fp8")
    imgs, st = render(r, [L, R])
    q = oracle.fp8_scales(model)
    for v, cam in enumerate((L, R)):
        ids = oracle.cull(model, cam)
        assert np.array_equal(r.debug_visible(v), ids)
        attrs_q, _ = oracle.derive(model, oracle.camera_center(cam), ids, q)
        check_attrs_fp8(r.debug_attrs(v), attrs_q, model.scale[ids], f"fp8 city eye {v}")
    check_keygen_and_sort(r, [L, R])
    rs = np.random.default_rng(frame + 7)
    for v, cam in enumerate((L, R)):
        px = rs.integers(0, cam.width, 30000)
        py = rs.integers(0, cam.height, 30000)
        vr = oracle.view_gaussians(model, cam)
        ref, _, _, _ = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, True, px, py)
        p = oracle.psnr(imgs[v][py, px], ref)
        print(f"fp8 city frame {frame} eye {v}: {p:.2f} dB")
        assert p >= FP8_PSNR, f"fp8 city frame {frame} eye {v}: {p:.2f} dB"
    r.close()

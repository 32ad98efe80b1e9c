"""Pins of the oracle's Octree-GS level selection (Sec. 2: octree levels of
detail chosen by distance; the per-anchor level offset and the level fade are
readings, stated in the oracle's cull and lod_weight).

- zero offsets give exactly the plain distance rule, and unit offsets the
  plain rule with d_max doubled (closed forms of d <= d_max 2^(Delta - l));
- the float32 decision equals the float64 predicate l <= log2(d_max / d) +
  Delta except within rounding of the boundary, on a city scene with offsets
  of both signs (a sign or level-direction slip fails here);
- the fade weight takes its special values: 0 at the switching distance, 1/2
  half a fade width inside it, 1 from a full width on, 1 at level 0.
"""
from dataclasses import replace

import numpy as np

import gen
import oracle


def city_cam():
    return gen.stereo_frames(gen.city_path(n_frames=3, seed=4, start=(-50.0, -80.0), h0=20.0, h1=30.0))[1][0]


def test_zero_and_unit_offsets_reduce_to_the_plain_rule():
    m = gen.city_scene(n=200_000, seed=3)
    cam = city_cam()
    plain = oracle.cull(m, cam)
    zero = oracle.cull(replace(m, level_offset=np.zeros(m.n, np.float32)), cam)
    assert np.array_equal(plain, zero) and len(plain) > 1000
    unit = oracle.cull(replace(m, level_offset=np.ones(m.n, np.float32)), cam)
    doubled = oracle.cull(replace(m, lod_dmax=2.0 * m.lod_dmax), cam)
    assert np.array_equal(unit, doubled) and len(unit) > len(plain)


def test_offset_rule_matches_fp64_levels():
    m = gen.with_level_offsets(gen.city_scene(n=200_000, seed=3), sigma=0.7, seed=9)
    cam = city_cam()
    ids = oracle.cull(m, cam)
    everything = oracle.cull(replace(m, level_offset=None, lod_dmax=1e30), cam)  # frustum only
    fr = np.zeros(m.n, bool)
    fr[everything] = True
    X = m.pos.astype(np.float64)
    d = np.linalg.norm(X - oracle.camera_center(cam), axis=1)
    lvl = m.level.astype(np.float64)
    delta = m.level_offset.astype(np.float64)
    u = np.log2(m.lod_dmax / d) + delta - lvl  # levels inside the switching distance
    ref = fr & ((lvl == 0) | (u >= 0))
    got = np.zeros(m.n, bool)
    got[ids] = True
    diff = np.nonzero(got != ref)[0]
    assert np.all(np.abs(u[diff]) < 1e-5)  # only rounding at the boundary
    assert got.sum() > 1000
    # the fade measures from the same radius and float32 distance as the cull:
    # kept anchors are at or inside their switch, dropped ones outside (w = 0)
    mb = replace(m, lod_blend=0.5)
    assert np.all(oracle.lod_weight(mb, cam, ids) >= 0.0)
    dropped = np.nonzero(fr & ~got & (m.level > 0))[0]
    assert len(dropped) > 1000 and np.all(oracle.lod_weight(mb, cam, dropped) == 0.0)
    # offsets move anchors across levels both ways
    plain = np.zeros(m.n, bool)
    plain[oracle.cull(replace(m, level_offset=None), cam)] = True
    assert (got & ~plain).sum() > 100 and (plain & ~got).sum() > 100


def test_fade_weight_special_values():
    beta, dmax = 0.5, 100.0
    levels = np.array([1, 1, 1, 1, 2, 3, 0], np.uint8)
    delta = np.array([0.0, 0.3, -0.4, 0.0, 0.25, -1.0, 0.0], np.float32)
    # distance of each anchor in units of its switching radius r = dmax 2^(Delta - l):
    # at r (u = 0), 2^-beta/2 r (u = beta/2), 2^-beta r (u = beta), 2^-2beta r, ...
    frac_u = np.array([0.0, 0.5, 1.0, 2.0, 0.25, 0.75, 5.0])
    r = dmax * 2.0 ** (delta.astype(np.float64) - levels)
    dist = r * 2.0 ** (-frac_u * beta)
    cam = gen.tiny_camera()
    p = oracle.camera_center(cam)
    pos = (p[None, :] + np.outer(dist, [0.0, 0.0, 1.0])).astype(np.float32)
    n = len(levels)
    m = replace(gen.tiny_scene(n=n), pos=pos, level=levels, n_levels=4, lod_dmax=dmax, level_offset=delta,
                lod_blend=beta)
    w = oracle.lod_weight(m, cam, np.arange(n))
    want = np.array([0.0, 0.5, 1.0, 1.0, 0.25, 0.75, 1.0])
    assert np.abs(w - want).max() < 1e-6  # float32 positions
    assert oracle.lod_weight(replace(m, lod_blend=0.0), cam, np.arange(n)).tolist() == [1.0] * n


def test_fade_scales_record_opacity_only():
    """Records with a fade equal those without it, opacity times the weight
    (tau = 2 ln(255 o) follows the opacity); positions and conics unchanged."""
    m0 = gen.with_level_offsets(gen.city_scene(n=100_000, seed=3), sigma=0.5, beta=0.0)
    m1 = replace(m0, lod_blend=0.75)
    cam = city_cam()
    v0 = oracle.view_gaussians(m0, cam)
    v1 = oracle.view_gaussians(m1, cam)
    assert np.array_equal(v0.ids, v1.ids)
    w = np.repeat(oracle.lod_weight(m1, cam, v1.ids), m1.k)
    ok = (v0.rec[:, 0] == 1) & (w > 0)
    assert ok.sum() > 1000 and (w < 1).sum() > 100
    assert np.array_equal(v1.rec[ok, 1:6], v0.rec[ok, 1:6])
    assert np.allclose(v1.rec[ok, 6], v0.rec[ok, 6] * w[ok], rtol=1e-15, atol=0)
    assert np.allclose(v1.rec[ok, 11], 2.0 * np.log(255.0 * v1.rec[ok, 6]), rtol=1e-12)
    assert not v1.rec[(v0.rec[:, 0] == 1) & (w == 0), 0].any()

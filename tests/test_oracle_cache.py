"""Pins of the oracle's cache policy (Sec. 4, Alg. 1, Eq. 4)."""
import numpy as np
import pytest

import gen
import oracle
from oracle.cache import CacheSim, cached_derive, next_depth, project_view


def test_linear_guide_values():
    """Eq. 4 with the linear guide: depth = round(D (1 - u)), clamped to [1, D]."""
    assert next_depth(10, 100, 15, 10) == 9      # 8.5 rounds up
    assert next_depth(10, 100, 14, 10) == 9      # 8.6
    assert next_depth(10, 100, 16, 10) == 8      # 8.4
    assert next_depth(10, 100, 100, 10) == 1     # u = 1 -> 0, clamped to 1
    assert next_depth(10, 100, 0, 10) == 10      # u = 0
    assert next_depth(7, 0, 0, 10) == 7          # nothing visible: unchanged
    for v in range(1, 60):
        for m in range(0, v + 1):
            d = next_depth(10, v, m, 10)
            exact = 10 * (v - m) / v
            assert 1 <= d <= 10
            assert d == min(max(int(np.floor(exact + 0.5)), 1), 10)


def test_branches_of_alg1_static_and_teleport():
    """First frame: decode all (0% duplicate); same view next frame: reuse all
    (100%); a disjoint view: decode all again."""
    sim = CacheSim(n_anchors=100, slots=100, max_depth=10)
    ids = np.arange(10, 40)
    hit, line, used = sim.step(ids)
    assert not hit.any() and np.all(line >= 0) and sim.depth == 1
    hit, line2, used = sim.step(ids)
    assert hit.all() and np.array_equal(line, line2) and sim.depth == 10
    hit, _, _ = sim.step(np.arange(60, 90))
    assert not hit.any()


def test_max_depth_invalidates_and_lines_recycle():
    sim = CacheSim(n_anchors=50, slots=20, max_depth=3)
    a = np.arange(0, 10)
    sim.step(a)                       # t=1: decode a into lines 0..9
    for _ in range(3):
        sim.step(np.arange(20, 30))   # t=2..4: b takes lines 10..19 at t=2, hits after
    # t=5: a's lines are 4 frames old (> D_max = 3): invalid, a is new again
    hit, line, _ = sim.step(a)
    assert not hit.any()
    # b's lines (decoded t=2, age 3 <= 3) are still valid, so the free lines are a's old ones
    assert set(line.tolist()) == set(range(10))


def test_free_lines_go_to_new_anchors_in_order_and_overflow_is_uncached():
    sim = CacheSim(n_anchors=100, slots=5, max_depth=10)
    hit, line, _ = sim.step(np.array([3, 7, 9, 20, 40, 41, 42]))
    assert list(line) == [0, 1, 2, 3, 4, -1, -1]
    assert sim.last["cached_new"] == 5 and sim.last["new"] == 7


def test_policy_against_per_anchor_history():
    """Random visible sequences: each anchor's status equals what its own
    decode history implies (an independent per-anchor formulation)."""
    rs = np.random.default_rng(0)
    N, S, D = 300, 120, 6
    sim = CacheSim(N, S, max_depth=D)
    owner = {}          # line -> anchor
    line_frame = {}     # line -> frame it was last written
    dec_frame = {}      # anchor -> frame of its last decode into a line
    line_of = {}
    depth = D
    for t in range(1, 120):
        centre = int(rs.integers(0, N))
        ids = np.unique((centre + rs.integers(-40, 40, 60)) % N)
        hit, line, used = sim.step(ids)
        assert used == depth
        free = sorted(l for l in range(S) if l not in owner or t - line_frame[l] > D)
        fi = 0
        misses = 0
        for a, h, l in zip(ids.tolist(), hit.tolist(), line.tolist()):
            ln = line_of.get(a)
            valid = ln is not None and owner.get(ln) == a and t - dec_frame[a] <= D
            exp_hit = valid and t - dec_frame[a] <= depth
            assert h == exp_hit, (t, a)
            if not valid:
                exp_line = free[fi] if fi < len(free) else -1
                fi += 1
                assert l == exp_line
            else:
                assert l == ln
            if not exp_hit:
                misses += 1
        for a, h, l in zip(ids.tolist(), hit.tolist(), line.tolist()):
            if not h and l >= 0:
                owner[l] = a
                line_frame[l] = t
                dec_frame[a] = t
                line_of[a] = l
        depth = next_depth(depth, len(ids), misses, D)


def test_view_independent_model_cached_equals_fp16_uncached():
    """With the view direction's weights zeroed, a hit's float16 line holds
    exactly the rounding of what a fresh decode would give, so the cached
    frame equals the plain frame rendered from float16-rounded attributes."""
    m = gen.tiny_scene(n=400)
    for h in range(3):
        m.W1[h][32:35, :] = 0.0
    cams = [gen.tiny_camera(160, 120)]
    R = gen.look_rotation(0.0, 0.0)
    sim = CacheSim(m.n, 4000, max_depth=10)
    for f in range(4):
        cam = gen.pinhole(np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1.0]]), np.array([0.02 * f, 0, -15.0]), 160, 120, 60)
        ids, attrs, kept, hit, line, used = cached_derive(m, cam, sim)
        vr = project_view(m, cam, ids, attrs, kept)
        img = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height)[0]
        fresh, _ = oracle.derive(m, oracle.camera_center(cam), ids)
        ref_attrs = np.where(hit[:, None, None], fresh.astype(np.float16).astype(np.float64), fresh)
        vr2 = project_view(m, cam, ids, ref_attrs, (ref_attrs[..., 0] > 0).astype(np.uint8))
        ref = oracle.render(vr2.rec, vr2.depth32, vr2.gid, cam.width, cam.height)[0]
        assert np.array_equal(img, ref)
        if f == 1:
            assert hit.all()


def test_guiding_functions_closed_forms():
    """Eq. 4 guides: all three give D at u = 0 and 1 at u = 1; the exponential
    one is D^(1-u) rounded (10^0.5 = 3.16 -> 3 at u = 1/2, 10^0.9 = 7.94 -> 8
    at u = 1/10); the staged one switches at u = 0.1 and u = 0.3; the
    exponential one never exceeds the linear one by more than rounding
    (D^(1-u) <= 1 + (D-1)(1-u) by convexity), so it reuses less under
    accelerating motion."""
    for g in ("linear", "exp", "staged"):
        assert next_depth(10, 100, 0, 10, g) == 10
        assert next_depth(10, 100, 100, 10, g) == 1
        assert next_depth(4, 0, 0, 10, g) == 4
    assert next_depth(10, 100, 50, 10, "exp") == 3
    assert next_depth(10, 100, 10, 10, "exp") == 8
    assert next_depth(10, 1000, 99, 10, "staged") == 10
    assert next_depth(10, 1000, 100, 10, "staged") == 5
    assert next_depth(9, 1000, 299, 9, "staged") == 5
    assert next_depth(10, 1000, 300, 10, "staged") == 1
    for v in (7, 100, 997):
        for m in range(0, v + 1, max(1, v // 50)):
            e, l = next_depth(10, v, m, 10, "exp"), next_depth(10, v, m, 10, "linear")
            assert e <= l + 1
            assert e == max(1, min(10, round(10 ** (1 - m / v))))
    for g in ("linear", "exp", "staged"):  # monotone non-increasing in the update rate
        ds = [next_depth(10, 500, m, 10, g) for m in range(0, 501)]
        assert all(a >= b for a, b in zip(ds, ds[1:]))
    with pytest.raises(ValueError):
        next_depth(10, 100, 5, 10, "cubic")

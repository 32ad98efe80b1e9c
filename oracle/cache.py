"""Cache-centric reuse of derived Gaussians (Sec. 4, Alg. 1, Eq. 4): the
oracle's plain simulation of the policy, one frame at a time.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Readings (the paper gives the algorithm's branches, not its data layout):
- A cache line holds the derived attributes of one anchor's k Gaussians in
  float16 (round to nearest even), the anchor id and the frame it was decoded
  in; anchors map to lines through a per-anchor index ("the anchor indices
  are translated to the cache indices by index mapping", Sec. 4).
- Reuse depth d: a line decoded `age` frames ago is reused iff age <= d
  ("results of the previous d frames").  Lines older than the maximum depth
  D_max are invalid (Alg. 1, "reach max cache reuse depth -> invalidate").
- A visible anchor is a hit (reuse), a refresh (valid line, too old for the
  current depth: decoded again into the same line) or new (no valid line:
  decoded, and given the next free line).  Free lines (never used, or past
  D_max) are handed out in ascending line order to new anchors in ascending
  anchor order; new anchors left without a line are decoded but not cached.
  The 0% / 100% duplicate branches of Alg. 1 are the cases "all new" and
  "all hits".
- Eq. 4 with the linear guiding function of the experiments: after a frame
  with V visible anchors of which m were decoded (the update rate u = m/V,
  equal to the miss rate), the next depth is round(D_max (1 - u)) clamped to
  [1, D_max], computed in integers as floor((2 D_max (V - m) + V) / (2 V)).
- In its own frame a decoded anchor is rendered with its fresh attributes;
  a hit is rendered with the cached float16 attributes.
- Learned form (an extension, see oracle.predictor): a valid line is reused
  iff the predictor says so; every decoded line also keeps the unit
  direction camera -> anchor it was decoded for (the predictor's input).
"""
from __future__ import annotations

import math

import numpy as np

ATTR = 11


GUIDES = ("linear", "exp", "staged")


def next_depth(depth: int, visible: int, misses: int, d_max: int, guide: str = "linear") -> int:
    """Guiding function H of Eq. 4, u = misses / visible, result in [1, d_max]:
    linear  round(d_max (1 - u)) (integer rounding, half up; the paper's
            experiments);
    exp     round(d_max ** (1 - u)) in float64 (the paper's "exponential
            response" for accelerating motion; its formula is this reading);
    staged  d_max for u < 0.1, ceil(d_max / 2) for u < 0.3, else 1 (the
            paper's "staged response"; thresholds are this reading)."""
    if visible <= 0:
        return depth
    v, m = int(visible), int(misses)
    if guide == "exp":
        d = int(math.floor(float(d_max) ** (1.0 - m / v) + 0.5))
    elif guide == "staged":
        d = d_max if 10 * m < v else ((d_max + 1) // 2 if 10 * m < 3 * v else 1)
    elif guide == "linear":
        d = (2 * d_max * (v - m) + v) // (2 * v)
    else:
        raise ValueError(guide)
    return int(min(max(d, 1), d_max))


class CacheSim:
    """Alg. 1 for one derivation view."""

    def __init__(self, n_anchors: int, slots: int, k: int = 10, max_depth: int = 10, guide: str = "linear"):
        self.k = k
        self.D = int(max_depth)
        self.guide = guide
        self.slot_of = np.full(n_anchors, -1, np.int64)
        self.slot_anchor = np.full(slots, -1, np.int64)
        self.slot_frame = np.zeros(slots, np.int64)
        self.slot_attr = np.zeros((slots, k, ATTR), np.float16)
        self.slot_dir = np.zeros((slots, 3), np.float32)
        self.t = 0
        self.depth = self.D

    def reset(self):
        self.slot_of[:] = -1
        self.slot_anchor[:] = -1
        self.slot_frame[:] = 0
        self.slot_dir[:] = 0
        self.t = 0
        self.depth = self.D

    def peek(self, ids: np.ndarray):
        """(valid mask, line or -1, age) of the visible ids as the next frame
        will find them, without changing the cache."""
        t = self.t + 1
        ids = np.asarray(ids, np.int64)
        s = self.slot_of[ids]
        valid = s >= 0
        sv = np.where(valid, s, 0)
        valid &= self.slot_anchor[sv] == ids
        age = t - self.slot_frame[sv]
        valid &= age <= self.D
        return valid, np.where(valid, s, -1), age

    def step(self, ids: np.ndarray, d_now=None, reuse=None):
        """Classify the ascending visible ids of one frame.  Returns
        (hit mask, line per anchor or -1, depth used this frame).
        d_now: unit directions camera -> anchor this frame (stored with the
        decoded lines); reuse: learned decision, a function of (valid mask,
        line) giving a mask, used instead of the depth rule."""
        valid, line, age = self.peek(ids)
        self.t += 1
        t = self.t
        ids = np.asarray(ids, np.int64)
        hit = valid & (age <= self.depth) if reuse is None else valid & reuse(valid, line)
        free = np.nonzero((self.slot_anchor < 0) | (t - self.slot_frame > self.D))[0]
        new_idx = np.nonzero(~valid)[0]
        n = min(len(new_idx), len(free))
        line[new_idx[:n]] = free[:n]
        # the lines of every decoded anchor now belong to it and to this frame
        dec = (~hit) & (line >= 0)
        self.slot_anchor[line[dec]] = ids[dec]
        self.slot_frame[line[dec]] = t
        self.slot_of[ids[dec]] = line[dec]
        if d_now is not None:
            self.slot_dir[line[dec]] = np.asarray(d_now, np.float32)[dec]
        used = self.depth
        self.last = dict(visible=len(ids), misses=int((~hit).sum()), hits=int(hit.sum()),
                         new=len(new_idx), cached_new=n, free=len(free))
        self.depth = next_depth(self.depth, len(ids), int((~hit).sum()), self.D, self.guide)
        return hit, line, used

    def store(self, line: np.ndarray, decoded: np.ndarray, attrs: np.ndarray):
        """Write fresh attributes [n,k,11] of the decoded anchors into their lines (float16)."""
        sel = decoded & (line >= 0)
        self.slot_attr[line[sel]] = attrs[sel].astype(np.float16)

    def cached_attrs(self, line: np.ndarray, hit: np.ndarray) -> np.ndarray:
        return self.slot_attr[line[hit]].astype(np.float64)


def cached_derive(model, dcam, sim: CacheSim, quant=None, theta=None, ids=None):
    """The derivation step of one frame in the cached form, for the derivation
    camera dcam: filtering (dcam's own, or the given ascending ids: the
    exact stereo form's union of both eyes' sets), the policy (the depth
    rule, or the predictor with parameters theta), fresh derivation of the
    decoded anchors, float16 lines for the hits.  Returns (ids, attrs
    [V,k,11], kept [V,k], hit mask, line per anchor, depth used)."""
    import oracle
    from oracle import predictor as P
    ids = oracle.cull(model, dcam) if ids is None else np.asarray(ids, np.uint32)
    d_now, dist = P.pinned_dir(model.pos[ids], oracle.camera_center(dcam))
    reuse = None
    if theta is not None:
        def reuse(valid, line):
            out = np.zeros(len(ids), bool)
            v = np.nonzero(valid)[0]
            if len(v):
                z = P.features(model.feat[ids[v]], d_now[v], sim.slot_dir[line[v]], dist[v])
                out[v] = P.decide(z, theta)
            return out
    hit, line, used = sim.step(ids, d_now, reuse)
    attrs = np.zeros((len(ids), model.k, ATTR), np.float64)
    miss = ~hit
    if miss.any():
        a_m, _ = oracle.derive(model, oracle.camera_center(dcam), ids[miss], quant)
        attrs[miss] = a_m
        sim.store(line[miss], np.ones(int(miss.sum()), bool), a_m)
    if hit.any():
        attrs[hit] = sim.cached_attrs(line, hit)
    kept = (attrs[..., 0] > 0).astype(np.uint8)
    return ids, attrs, kept, hit, line, used


def collect_samples(model, dcam, sim: CacheSim, quant=None, ids=None):
    """Predictor training samples of the coming frame (call before
    cached_derive for the same frame): for every visible anchor holding a
    valid line, its inputs z and its label (oracle.predictor.label of the
    float16 line against a fresh float64 derivation of this frame).  Returns
    (visible indices, z [n,36], labels [n], label margins [n]): the margin is
    how far the closest of the label's comparisons lies from its threshold."""
    import oracle
    from oracle import predictor as P
    ids = oracle.cull(model, dcam) if ids is None else np.asarray(ids, np.uint32)
    valid, line, _ = sim.peek(ids)
    v = np.nonzero(valid)[0]
    pc = oracle.camera_center(dcam)
    d_now, dist = P.pinned_dir(model.pos[ids[v]], pc)
    z = P.features(model.feat[ids[v]], d_now, sim.slot_dir[line[v]], dist)
    if len(v) == 0:
        return v, z, np.zeros(0, bool), np.zeros(0)
    fresh, _ = oracle.derive(model, pc, ids[v], quant)
    cached = sim.slot_attr[line[v]].astype(np.float64)
    return v, z, P.label(cached, fresh), P.label_margin(cached, fresh)


def project_view(model, cam, ids, attrs, kept, derive_cam=None, mine=None):
    """Records of one camera from attributes of the visible anchors (of the
    derivation camera `derive_cam`, which a level fade measures from).  In
    the exact stereo form `mine` marks the ids this camera keeps itself
    (bit of oracle.cull_pair's mask); the others' records are not kept and a
    level fade is measured from the camera."""
    import oracle
    if mine is not None:
        kept = np.asarray(kept, np.uint8) & np.asarray(mine, np.uint8)[:, None]
        derive_cam = cam
    rec, d32 = oracle.project_records(model, cam, ids, attrs, kept, derive_cam=derive_cam)
    gid = (np.asarray(ids, np.int64)[:, None] * model.k + np.arange(model.k)[None, :]).reshape(-1)
    return oracle.ViewResult(ids=ids, attrs=attrs, kept=kept, rec=rec, depth32=d32, gid=gid)

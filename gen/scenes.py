"""Seeded synthetic structured-3DGS scenes (anchors + decoder MLP weights).

The paper measures on MatrixCity with trained Scaffold-GS / Octree-GS models
(Sec. 7, Table 1).  Neither is available, so these generators stand in for
them with the same structure: anchors carrying a 32-d feature, k=10 offsets
and a scale; a level per anchor for distance LOD; and three two-layer decoder
MLPs (opacity, colour, covariance heads; hidden 32) with Glorot-uniform
weights and zero biases.  No content of the dataset is reproduced.

All values are drawn in float64 from `gen.rng` and cast to float32 once.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

from .rng import Stream

FEAT_DIM = 32
HIDDEN = 32
K_GAUSS = 10
IN_DIM = FEAT_DIM + 3          # feature + unit view direction (Eq. 3)


def head_out_dims(k: int = K_GAUSS):
    """Output widths of the opacity, colour and covariance heads."""
    return (k, 3 * k, 7 * k)


@dataclass
class Model:
    pos: np.ndarray            # float32 [N,3]  anchor positions (metres, world z up)
    feat: np.ndarray           # float32 [N,32] anchor features
    offs: np.ndarray           # float32 [N,k,3] per-Gaussian offsets (metres)
    scale: np.ndarray          # float32 [N]    per-anchor scale s_a
    level: np.ndarray          # uint8   [N]    LOD level (0 = coarsest)
    n_levels: int
    lod_dmax: float            # distance at which level 1 stops being drawn x2
    W1: List[np.ndarray] = field(default_factory=list)   # 3 x float32 [35,32]
    b1: List[np.ndarray] = field(default_factory=list)   # 3 x float32 [32]
    W2: List[np.ndarray] = field(default_factory=list)   # 3 x float32 [32,out_h]
    b2: List[np.ndarray] = field(default_factory=list)   # 3 x float32 [out_h]
    k: int = K_GAUSS
    name: str = ""
    level_offset: Optional[np.ndarray] = None  # float32 [N] per-anchor level offsets (Octree-GS), or None
    lod_blend: float = 0.0     # level fade width beta in levels (0: levels switch on at once)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def validate(self) -> None:
        n, k = self.n, self.k
        assert self.pos.shape == (n, 3) and self.pos.dtype == np.float32
        assert self.feat.shape == (n, FEAT_DIM) and self.feat.dtype == np.float32
        assert self.offs.shape == (n, k, 3) and self.offs.dtype == np.float32
        assert self.scale.shape == (n,) and self.scale.dtype == np.float32
        assert self.level.shape == (n,) and self.level.dtype == np.uint8
        if self.level_offset is not None:
            assert self.level_offset.shape == (n,) and self.level_offset.dtype == np.float32
        for h, od in enumerate(head_out_dims(k)):
            assert self.W1[h].shape == (IN_DIM, HIDDEN)
            assert self.b1[h].shape == (HIDDEN,)
            assert self.W2[h].shape == (HIDDEN, od)
            assert self.b2[h].shape == (od,)


def with_level_offsets(m: Model, sigma: float = 0.3, beta: float = 0.5, seed: int = 21) -> Model:
    """A copy of `m` with Octree-GS style per-anchor level offsets.  Trained
    offsets are not available; these are drawn N(0, sigma^2), clipped to
    [-3 sigma, 3 sigma], with fade width `beta` levels."""
    st = Stream(seed, "level_offset")
    d = np.clip(st.normal(m.n) * sigma, -3.0 * sigma, 3.0 * sigma).astype(np.float32)
    return replace(m, level_offset=d, lod_blend=float(beta), name=(m.name + "+octree") if m.name else "octree")


def glorot_mlps(seed: int, k: int = K_GAUSS):
    """Three Linear(35->32)-ReLU-Linear(32->out) heads, Glorot-uniform, zero bias."""
    st = Stream(seed, "mlp")
    W1, b1, W2, b2 = [], [], [], []
    for od in head_out_dims(k):
        a1 = np.sqrt(6.0 / (IN_DIM + HIDDEN))
        W1.append(st.uniform(IN_DIM * HIDDEN, -a1, a1).reshape(IN_DIM, HIDDEN).astype(np.float32))
        b1.append(np.zeros(HIDDEN, np.float32))
        a2 = np.sqrt(6.0 / (HIDDEN + od))
        W2.append(st.uniform(HIDDEN * od, -a2, a2).reshape(HIDDEN, od).astype(np.float32))
        b2.append(np.zeros(od, np.float32))
    return W1, b1, W2, b2


def tiny_scene(seed: int = 0, n: int = 2000, mlp_seed: int = 1, k: int = K_GAUSS) -> Model:
    """2,000 anchors uniform in a 10 m cube; one LOD level (LOD off)."""
    st = Stream(seed, "tiny")
    pos = st.uniform(n * 3, -5.0, 5.0).reshape(n, 3)
    feat = st.normal(n * FEAT_DIM).reshape(n, FEAT_DIM)
    offs = st.normal(n * k * 3, 0.0, 0.1).reshape(n, k, 3)
    scale = st.log_uniform(n, 0.01, 0.1)
    W1, b1, W2, b2 = glorot_mlps(mlp_seed, k)
    m = Model(pos=pos.astype(np.float32), feat=feat.astype(np.float32),
              offs=offs.astype(np.float32), scale=scale.astype(np.float32),
              level=np.zeros(n, np.uint8), n_levels=1, lod_dmax=0.0,
              W1=W1, b1=b1, W2=W2, b2=b2, k=k, name=f"tiny{n}_s{seed}")
    m.validate()
    return m


def city_scene(n: int = 2_000_000, seed: int = 10, mlp_seed: int = 1,
               extent: float = 2000.0, n_levels: int = 6, n_buildings: int = 4000,
               n_centres: int = 30, ground_frac: float = 0.55, size_mult: float = 4.0,
               keep_clear=None, k: int = K_GAUSS) -> Model:
    """City-like anchor set on a extent x extent metre plane (world z up).

    ~55% of anchors lie on the ground (z ~ N(0, 0.2 m)); the rest lie on the
    four facades and the roof of box buildings (footprint 15-60 m, height
    log-uniform 8-200 m) clustered around `n_centres` downtown centres.
    Level l in 0..n_levels-1 is drawn with P(l) proportional to 2^l; offsets
    and scales grow by 2^(n_levels-1-l) * size_mult so coarse levels carry
    large Gaussians.  `keep_clear` is an optional (x0, y0, x1, y1, margin)
    segment around which no building is placed (the camera path).
    """
    st = Stream(seed, "city")
    half = extent / 2.0
    n_ground = int(round(ground_frac * n))
    n_build = n - n_ground

    # --- buildings ---
    centres = st.uniform(n_centres * 2, -0.8 * half, 0.8 * half).reshape(n_centres, 2)
    which = np.minimum((st.uniform(n_buildings) * n_centres).astype(np.int64), n_centres - 1)
    bxy = centres[which] + st.normal(n_buildings * 2, 0.0, 150.0).reshape(n_buildings, 2)
    bxy = np.clip(bxy, -half + 40.0, half - 40.0)
    bw = st.uniform(n_buildings, 15.0, 60.0)
    bd = st.uniform(n_buildings, 15.0, 60.0)
    bh = st.log_uniform(n_buildings, 8.0, 200.0)
    if keep_clear is not None:
        x0, y0, x1, y1, margin = keep_clear
        seg = np.array([x1 - x0, y1 - y0])
        L2 = max(float(seg @ seg), 1e-9)
        rel = bxy - np.array([x0, y0])
        tpar = np.clip(rel @ seg / L2, 0.0, 1.0)
        dist = np.linalg.norm(rel - tpar[:, None] * seg[None, :], axis=1)
        ok = dist > margin + 0.75 * np.maximum(bw, bd)
        bxy, bw, bd, bh = bxy[ok], bw[ok], bd[ok], bh[ok]
    nb = bxy.shape[0]
    # faces: 0 x-, 1 x+, 2 y-, 3 y+, 4 roof
    areas = np.stack([bd * bh, bd * bh, bw * bh, bw * bh, bw * bd], axis=1).reshape(-1)
    cum = np.cumsum(areas)
    pick = np.searchsorted(cum, st.uniform(n_build) * cum[-1], side="right")
    pick = np.minimum(pick, 5 * nb - 1)
    b, face = pick // 5, pick % 5
    ua, ub = st.uniform(n_build), st.uniform(n_build)
    cx, cy = bxy[b, 0], bxy[b, 1]
    w, d, h = bw[b], bd[b], bh[b]
    px = np.where(face == 0, cx - w / 2, np.where(face == 1, cx + w / 2, cx + (ua - 0.5) * w))
    py = np.where(face == 2, cy - d / 2, np.where(face == 3, cy + d / 2,
                  np.where(face <= 1, cy + (ua - 0.5) * d, cy + (ub - 0.5) * d)))
    pz = np.where(face == 4, h, ub * h)
    bpos = np.stack([px, py, pz], axis=1)

    # --- ground ---
    gx = st.uniform(n_ground, -half, half)
    gy = st.uniform(n_ground, -half, half)
    gz = st.normal(n_ground, 0.0, 0.2)
    gpos = np.stack([gx, gy, gz], axis=1)

    pos = np.concatenate([gpos, bpos], axis=0)
    # shuffle so anchor ids are not spatially ordered by type
    perm = np.argsort(st.bits(n), kind="stable")
    pos = pos[perm]

    # --- levels, features, offsets, scales ---
    wl = 2.0 ** np.arange(n_levels)
    cl = np.cumsum(wl) / wl.sum()
    level = np.minimum(np.searchsorted(cl, st.uniform(n), side="right"), n_levels - 1).astype(np.uint8)
    mult = (2.0 ** (n_levels - 1 - level.astype(np.float64))) * size_mult
    feat = st.normal(n * FEAT_DIM).reshape(n, FEAT_DIM)
    offs = st.normal(n * k * 3, 0.0, 0.1).reshape(n, k, 3) * mult[:, None, None]
    scale = st.log_uniform(n, 0.01, 0.1) * mult
    W1, b1, W2, b2 = glorot_mlps(mlp_seed, k)
    m = Model(pos=pos.astype(np.float32), feat=feat.astype(np.float32),
              offs=offs.astype(np.float32), scale=scale.astype(np.float32),
              level=level, n_levels=n_levels, lod_dmax=float(np.float32(extent * np.sqrt(2.0))),
              W1=W1, b1=b1, W2=W2, b2=b2, k=k, name=f"city{n}_s{seed}")
    m.validate()
    return m


def reuse_mlp_init(seed: int = 7) -> np.ndarray:
    """Initial parameters of the 36 -> 64 -> 1 reuse predictor, flat float32
    [W1 (36x64, input-major), b1 (64), w2 (64), b2 (1)]: Glorot-uniform
    weights, zero biases."""
    st = Stream(seed, "reuse_mlp")
    a1 = np.sqrt(6.0 / (36 + 64))
    a2 = np.sqrt(6.0 / (64 + 1))
    return np.concatenate([st.uniform(36 * 64, -a1, a1), np.zeros(64), st.uniform(64, -a2, a2),
                           np.zeros(1)]).astype(np.float32)

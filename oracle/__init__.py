"""Plain CPU oracle of the structured-3DGS per-frame path (GS-Cache, arXiv 2502.14938).

TEST INFRASTRUCTURE.  Only tests/, `__graft_entry__.smoke()` and the bench's
CPU-baseline leg may import this package; the CUDA library never does and
shares no code with it.  The heavy loops live in `gsc_oracle.cpp` (float64,
-ffp-contract=off); this module marshals numpy arrays through ctypes and
strings the per-view steps together in the paper's order:

  anchor filtering (Alg. 1) -> derivation (Eq. 3) -> projection (Eq. 1-2,
  EWA) -> tile coverage, depth order and alpha blending (Sec. 3.1, Sec. 6).

The cache policy (Alg. 1, Eq. 4) and the reuse predictor live in
`oracle.cache` and `oracle.predictor`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsc_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
REC = 16            # doubles per projected record
ATTR = 11           # alpha, colour(3), scale(3), quaternion(4)


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (g++, float64, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
               "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrcCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("pad", C.c_int32)]


class OrcModel(C.Structure):
    _fields_ = [("n", C.c_int32), ("k", C.c_int32), ("n_levels", C.c_int32), ("pad0", C.c_int32),
                ("pos", C.c_void_p), ("feat", C.c_void_p), ("offs", C.c_void_p),
                ("scale", C.c_void_p), ("level", C.c_void_p), ("lod_dmax", C.c_float),
                ("pad1", C.c_int32), ("W1", C.c_void_p * 3), ("b1", C.c_void_p * 3),
                ("W2", C.c_void_p * 3), ("b2", C.c_void_p * 3),
                ("level_offset", C.c_void_p), ("lod_blend", C.c_float), ("pad2", C.c_int32)]


class OrcQuant(C.Structure):
    _fields_ = [("mode", C.c_int32), ("pad", C.c_int32), ("s_x", C.c_float),
                ("s_h", C.c_float * 3), ("s_w1", C.c_float * 3), ("s_w2", C.c_float * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        L.orc_camera_center.argtypes = [P, P]
        L.orc_unified_camera.argtypes = [P, P, P]
        L.orc_unified_camera.restype = C.c_int
        L.orc_cull.argtypes = [P, P, P, C.c_int64]
        L.orc_cull.restype = C.c_int64
        L.orc_lod_weight.argtypes = [P, P, P, C.c_int64, C.c_double, P]
        L.orc_lod_weight.restype = C.c_int
        L.orc_derive.argtypes = [P, P, P, C.c_int64, P, P, P, P]
        L.orc_derive.restype = C.c_int
        L.orc_quat_to_rot.argtypes = [P, P]
        L.orc_project_gaussian.argtypes = [P, P, P, P, P]
        L.orc_depth32.argtypes = [P, P, P]
        L.orc_depth32.restype = C.c_float
        L.orc_project_records.argtypes = [P, P, P, C.c_int64, P, P, P, P]
        L.orc_project_records.restype = C.c_int
        L.orc_cover_tiles64.argtypes = [C.c_double] * 6 + [C.c_int] * 4 + [P, C.c_int64]
        L.orc_cover_tiles64.restype = C.c_int64
        L.orc_keygen_f32.argtypes = [C.c_int64] + [P] * 8 + [C.c_int] * 4 + [P, P, P, C.c_int64]
        L.orc_keygen_f32.restype = C.c_int64
        L.orc_render.argtypes = [P, P, P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.c_int64, P, P, P, P, P, P, P, P]
        L.orc_render.restype = C.c_int
        L.orc_blend_trace.argtypes = [P, P, C.c_int64, P, P]
        L.orc_blend_trace.restype = C.c_int64
        L.orc_round_bf16.argtypes = [C.c_float]
        L.orc_round_bf16.restype = C.c_float
        L.orc_round_e4m3.argtypes = [C.c_double]
        L.orc_round_e4m3.restype = C.c_double
        L.orc_e4m3_two_term.argtypes = [C.c_double, C.c_double, P]
        L.orc_e4m3_two_term.restype = C.c_double
        L.orc_num_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (results do not depend on it)."""
    lib().orc_set_threads(int(n))


# ------------------------------------------------------------------ cameras
def to_cam(cam) -> OrcCamera:
    c = OrcCamera()
    R = np.ascontiguousarray(cam.R, np.float32).reshape(-1)
    t = np.ascontiguousarray(cam.t, np.float32).reshape(-1)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.znear = int(cam.width), int(cam.height), float(cam.znear)
    return c


@dataclass
class OCam:
    """Camera as plain float32 values (the oracle's own copy of the inputs)."""
    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float


def from_orc(c: OrcCamera) -> OCam:
    return OCam(R=np.array(c.R[:], np.float32).reshape(3, 3), t=np.array(c.t[:], np.float32),
                fx=c.fx, fy=c.fy, cx=c.cx, cy=c.cy, width=c.width, height=c.height, znear=c.znear)


def camera_center(cam) -> np.ndarray:
    out = np.zeros(3, np.float64)
    c = to_cam(cam)
    lib().orc_camera_center(C.byref(c), _p(out))
    return out


def unified_camera(left, right) -> OCam:
    """Eq. 5-6: one camera whose frustum covers both eyes (float32 result)."""
    a, b, o = to_cam(left), to_cam(right), OrcCamera()
    assert lib().orc_unified_camera(C.byref(a), C.byref(b), C.byref(o)) == 0
    return from_orc(o)


# ------------------------------------------------------------------ model
class ModelRef:
    """ctypes view of a gen.Model (keeps the arrays alive)."""

    def __init__(self, m):
        self.m = m
        self.keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dt)
            self.keep.append(a)
            return a.ctypes.data_as(C.c_void_p)

        s = OrcModel()
        s.n, s.k, s.n_levels = m.n, m.k, m.n_levels
        s.pos, s.feat, s.offs = arr(m.pos, np.float32), arr(m.feat, np.float32), arr(m.offs, np.float32)
        s.scale, s.level = arr(m.scale, np.float32), arr(m.level, np.uint8)
        s.lod_dmax = float(m.lod_dmax)
        lo = getattr(m, "level_offset", None)
        s.level_offset = arr(lo, np.float32) if lo is not None else None
        s.lod_blend = float(getattr(m, "lod_blend", 0.0))
        for h in range(3):
            s.W1[h], s.b1[h] = arr(m.W1[h], np.float32), arr(m.b1[h], np.float32)
            s.W2[h], s.b2[h] = arr(m.W2[h], np.float32), arr(m.b2[h], np.float32)
        self.s = s

    @property
    def ref(self):
        return C.byref(self.s)


_mref_cache = {}


def mref(m) -> ModelRef:
    key = id(m)
    r = _mref_cache.get(key)
    if r is None or r.m is not m:
        r = ModelRef(m)
        _mref_cache.clear()
        _mref_cache[key] = r
    return r


# ------------------------------------------------------------------ steps
def cull(model, cam) -> np.ndarray:
    """Ascending ids of anchors passing the frustum + LOD filter (decision-pinned fp32)."""
    mr = mref(model)
    c = to_cam(cam)
    n = lib().orc_cull(mr.ref, C.byref(c), None, 0)
    ids = np.zeros(max(n, 1), np.uint32)
    n2 = lib().orc_cull(mr.ref, C.byref(c), _p(ids), n)
    assert n2 == n
    return ids[:n]


def cull_pair(model, left, right):
    """The exact stereo form's filtering (a reading of Eq. 5-6, see below):
    the ascending union of the two eyes' own visible sets (each eye's
    frustum and LOD predicates, as `cull`), and per id a 2-bit mask of the
    eyes that keep it (bit 0 left, bit 1 right).  Derivation then runs once
    per id from the unified camera's centre, and each eye draws only its own
    ids, so every eye sees exactly the anchors the per-eye method selects."""
    a, b = cull(model, left), cull(model, right)
    ids = np.union1d(a, b).astype(np.uint32)
    eyes = np.isin(ids, a).astype(np.uint8) | (np.isin(ids, b).astype(np.uint8) << 1)
    return ids, eyes


def quant_none():
    return None


def derive(model, view_pos: np.ndarray, ids: np.ndarray, quant: Optional[OrcQuant] = None,
           want_raw: bool = False):
    """Eq. 3 in float64: attrs [n,k,11] (alpha, c, s, q), kept [n,k] (and raw head outputs)."""
    mr = mref(model)
    ids = np.ascontiguousarray(ids, np.uint32)
    n, k = ids.shape[0], model.k
    attrs = np.zeros((n, k, ATTR), np.float64)
    kept = np.zeros((n, k), np.uint8)
    raw = np.zeros((n, 11 * k), np.float64) if want_raw else None
    vp = np.ascontiguousarray(view_pos, np.float64)
    q = C.byref(quant) if quant is not None else None
    assert lib().orc_derive(mr.ref, _p(vp), _p(ids), n, q, _p(attrs), _p(kept), _p(raw)) == 0
    return (attrs, kept, raw) if want_raw else (attrs, kept)


def lod_weight(model, derive_cam, ids: np.ndarray) -> np.ndarray:
    """Octree-GS level fade per anchor (orc_lod_weight): w = clamp(u / beta,
    0, 1) with u = log2(r_a / d) the anchor's levels inside its switching
    distance, from the culling radius and the culling test's float32 d^2;
    level 0 and beta = 0 give w = 1."""
    ids = np.ascontiguousarray(ids, np.uint32)
    w = np.ones(ids.shape[0], np.float64)
    beta = float(getattr(model, "lod_blend", 0.0))
    if beta > 0.0 and ids.shape[0]:
        c = to_cam(derive_cam)
        assert lib().orc_lod_weight(mref(model).ref, C.byref(c), _p(ids), ids.shape[0], beta, _p(w)) == 0
    return w


def project_records(model, cam, ids: np.ndarray, attrs: np.ndarray, kept: Optional[np.ndarray], derive_cam=None):
    """Projected records [n*k, 16] and pinned float32 depths [n*k].  With a
    level fade (model.lod_blend > 0) the opacities are first scaled by
    lod_weight of the derivation camera `derive_cam` (default: `cam`)."""
    mr = mref(model)
    ids = np.ascontiguousarray(ids, np.uint32)
    n, k = ids.shape[0], model.k
    if float(getattr(model, "lod_blend", 0.0)) > 0.0:
        w = lod_weight(model, cam if derive_cam is None else derive_cam, ids)
        attrs = np.array(attrs, np.float64).reshape(n, k, -1)
        attrs[:, :, 0] *= w[:, None]
        if kept is not None:
            kept = (np.asarray(kept).reshape(n, k) != 0) & (w[:, None] > 0.0)
    rec = np.zeros((n * k, REC), np.float64)
    d32 = np.zeros(n * k, np.float32)
    c = to_cam(cam)
    attrs = np.ascontiguousarray(attrs, np.float64)
    kept = None if kept is None else np.ascontiguousarray(kept, np.uint8)
    assert lib().orc_project_records(mr.ref, C.byref(c), _p(ids), n, _p(attrs), _p(kept), _p(rec), _p(d32)) == 0
    return rec, d32


def project_gaussian(cam, mu, s, q) -> np.ndarray:
    out = np.zeros(11, np.float64)
    c = to_cam(cam)
    lib().orc_project_gaussian(C.byref(c), _p(np.ascontiguousarray(mu, np.float64)),
                               _p(np.ascontiguousarray(s, np.float64)),
                               _p(np.ascontiguousarray(q, np.float64)), _p(out))
    return out


def quat_to_rot(q) -> np.ndarray:
    R = np.zeros(9, np.float64)
    lib().orc_quat_to_rot(_p(np.ascontiguousarray(q, np.float64)), _p(R))
    return R.reshape(3, 3)


def cover_tiles64(mx, my, A, B, Cc, tau, W, H, TW=16, TH=16) -> np.ndarray:
    n = lib().orc_cover_tiles64(mx, my, A, B, Cc, tau, W, H, TW, TH, None, 0)
    out = np.zeros(max(n, 1), np.int32)
    lib().orc_cover_tiles64(mx, my, A, B, Cc, tau, W, H, TW, TH, _p(out), n)
    return out[:n]


def keygen_f32(mx, my, A, B, Cc, tau, view, valid, W, H, TW=16, TH=16):
    """Stage-isolated float32 key generation: (counts, keys, values) in record order."""
    f = lambda a: np.ascontiguousarray(a, np.float32)
    mx, my, A, B, Cc, tau = map(f, (mx, my, A, B, Cc, tau))
    view = np.ascontiguousarray(view, np.int32)
    valid = np.ascontiguousarray(valid, np.uint8)
    n = mx.shape[0]
    counts = np.zeros(n, np.uint32)
    L = lib()
    args = [_p(x) for x in (mx, my, A, B, Cc, tau, view, valid)]
    P = L.orc_keygen_f32(n, *args, W, H, TW, TH, _p(counts), None, None, 0)
    keys = np.zeros(max(P, 1), np.uint32)
    vals = np.zeros(max(P, 1), np.uint32)
    P2 = L.orc_keygen_f32(n, *args, W, H, TW, TH, _p(counts), _p(keys), _p(vals), P)
    assert P2 == P
    return counts, keys[:P], vals[:P]


def render(rec: np.ndarray, depth32: np.ndarray, gid: np.ndarray, W: int, H: int, tiled: bool = True,
           px: Optional[np.ndarray] = None, py: Optional[np.ndarray] = None, bg=(0.0, 0.0, 0.0),
           TW: int = 16, TH: int = 16, walk: bool = False):
    """Alpha-blend the records.  Returns rgb, final T, decision margin, contributor count
    (per listed pixel, or [H,W,...] images when no pixel list is given), and with
    walk=True also the walk length: how many Gaussians of its list each pixel
    evaluated (all, or up to and including the one at which it stops)."""
    rec = np.ascontiguousarray(rec, np.float64)
    depth32 = np.ascontiguousarray(depth32, np.float32)
    gid = np.ascontiguousarray(gid, np.int64)
    n = rec.shape[0]
    if px is None:
        npix = -1
        NP = W * H
    else:
        px = np.ascontiguousarray(px, np.int32)
        py = np.ascontiguousarray(py, np.int32)
        npix = NP = px.shape[0]
    rgb = np.zeros((NP, 3), np.float64)
    T = np.zeros(NP, np.float64)
    mg = np.zeros(NP, np.float64)
    nc = np.zeros(NP, np.int32)
    wk = np.zeros(NP, np.int32) if walk else None
    bgv = np.ascontiguousarray(bg, np.float64)
    assert lib().orc_render(_p(rec), _p(depth32), _p(gid), n, W, H, 1 if tiled else 0, TW, TH, npix,
                            _p(px), _p(py), _p(bgv), _p(rgb), _p(T), _p(mg), _p(nc), _p(wk)) == 0
    if px is None:
        out = (rgb.reshape(H, W, 3), T.reshape(H, W), mg.reshape(H, W), nc.reshape(H, W))
        return out + (wk.reshape(H, W),) if walk else out
    return (rgb, T, mg, nc, wk) if walk else (rgb, T, mg, nc)


def blend_trace(alpha_raw: np.ndarray, colour: np.ndarray):
    a = np.ascontiguousarray(alpha_raw, np.float64)
    c = np.ascontiguousarray(colour, np.float64).reshape(-1, 3)
    tr = np.zeros((a.shape[0], 3), np.float64)
    out = np.zeros(4, np.float64)
    u = lib().orc_blend_trace(_p(a), _p(c), a.shape[0], _p(tr), _p(out))
    return tr[:u], out[:3], out[3]


def round_bf16(x: float) -> float:
    return float(lib().orc_round_bf16(float(x)))


def round_e4m3(x: float) -> float:
    return float(lib().orc_round_e4m3(float(x)))


def e4m3_two_term(v: float, s: float):
    """(hi + lo, hi): the FP8 form's two-term E4M3 expansion of v at scale s."""
    hi = C.c_double()
    tot = lib().orc_e4m3_two_term(float(v), float(s), C.byref(hi))
    return float(tot), float(hi.value)


E4M3_MAX = 448.0


def pow2_ceil(v: float) -> float:
    """Smallest power of two >= v (v > 0); 1 for v <= 0."""
    if not v > 0:
        return 1.0
    m, e = np.frexp(v)  # v = m 2^e, m in [0.5, 1)
    return float(np.ldexp(1.0, int(e) - 1 if m == 0.5 else int(e)))


def fp8_scales(model) -> OrcQuant:
    """Per-tensor scales of the FP8-E4M3 form (a reading of "per-tensor
    scales" with amax / 448, rounded up to a power of two so that scaling is
    exact):
      s_x     from max(amax of the anchor features, 1) (the unit view
              direction shares the input tensor),
      s_w1[h], s_w2[h] from amax of each head's weight matrices,
      s_h[h]  from a bound on the head's hidden activations that holds for
              every anchor and view direction:
              max_o sum_c |W1[c,o]| amax_c + |b1[o]|, with amax_c the
              largest |feature c| over the anchors and 1 for a direction
              component."""
    q = OrcQuant()
    q.mode = 2
    feat = np.abs(np.asarray(model.feat, np.float64))
    amax_c = feat.max(axis=0) if feat.size else np.zeros(feat.shape[1])
    q.s_x = pow2_ceil(max(float(amax_c.max()) if amax_c.size else 0.0, 1.0) / E4M3_MAX)
    xb = np.concatenate([amax_c, np.ones(3)])
    for h in range(3):
        W1 = np.asarray(model.W1[h], np.float64)
        W2 = np.asarray(model.W2[h], np.float64)
        q.s_w1[h] = pow2_ceil(float(np.abs(W1).max()) / E4M3_MAX)
        q.s_w2[h] = pow2_ceil(float(np.abs(W2).max()) / E4M3_MAX)
        hb = (np.abs(W1) * xb[:, None]).sum(axis=0) + np.abs(np.asarray(model.b1[h], np.float64))
        q.s_h[h] = pow2_ceil(float(hb.max()) / E4M3_MAX)
    return q


# ------------------------------------------------------------------ one view / one frame
@dataclass
class ViewResult:
    ids: np.ndarray            # visible anchor ids (of the derivation camera)
    attrs: np.ndarray          # [V,k,11]
    kept: np.ndarray           # [V,k]
    rec: np.ndarray            # [V*k,16]
    depth32: np.ndarray        # [V*k]
    gid: np.ndarray            # [V*k] global Gaussian id a*k + j


def view_gaussians(model, cam, derive_cam=None, quant=None, attrs_override=None, pair=None) -> ViewResult:
    """Visible anchors, derived attributes and projected records of one view.
    `derive_cam` (default: `cam`) selects the anchors and the view direction
    (the unified camera of Eq. 5-6 in the de-redundant stereo form).  With
    pair = (left, right) (cam one of them) the anchors are instead the
    exact stereo form's (`cull_pair`): the union of the eyes' own sets,
    derived from derive_cam's centre, of which `cam` draws only its own
    (records of the other eye's anchors are not kept); a level fade is then
    measured from `cam`, whose distances selected its anchors."""
    dc = cam if derive_cam is None else derive_cam
    if pair is not None:
        ids, eyes = cull_pair(model, *pair)
        mine = (eyes >> (0 if cam is pair[0] else 1)) & 1
    else:
        ids = cull(model, dc)
    if attrs_override is not None:
        attrs, kept = attrs_override(ids)
    else:
        attrs, kept = derive(model, camera_center(dc), ids, quant)
    if pair is not None:
        kept = np.asarray(kept, np.uint8) & mine[:, None]
    rec, d32 = project_records(model, cam, ids, attrs, kept, derive_cam=cam if pair is not None else dc)
    gid = (ids.astype(np.int64)[:, None] * model.k + np.arange(model.k)[None, :]).reshape(-1)
    return ViewResult(ids=ids, attrs=attrs, kept=kept, rec=rec, depth32=d32, gid=gid)


def render_view(model, cam, derive_cam=None, quant=None, tiled=True, px=None, py=None, bg=(0, 0, 0)):
    vr = view_gaussians(model, cam, derive_cam, quant)
    out = render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, tiled, px, py, bg)
    return out, vr


def psnr(img: np.ndarray, ref: np.ndarray) -> float:
    """PSNR for images in [0,1]: 10 log10(1 / MSE) over all values."""
    mse = float(np.mean((np.asarray(img, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)

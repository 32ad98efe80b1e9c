"""ctypes binding of the C ABI in include/gsc.h and include/gsc_debug.h.

Argument marshalling only: every step of a frame runs in the library's CUDA
kernels.  The library is loaded from this package directory; a missing or
unloadable libgsc.so raises at import of `lib()` - there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# GSC_LIBRARY selects another build of the library for this process (the
# bounds-checked libgsc_checked.so), read when the library is first loaded.
LIB_PATH = os.environ.get("GSC_LIBRARY") or os.path.join(HERE, "libgsc.so")

MAX_VIEWS = 32
K = 10

GSC_OK = 0
STATUS = {0: "GSC_OK", -1: "GSC_ERR_INVALID_ARG", -2: "GSC_ERR_OOM", -3: "GSC_ERR_CUDA",
          -4: "GSC_ERR_CAPACITY", -5: "GSC_ERR_TIMEOUT", -6: "GSC_ERR_STATE",
          -7: "GSC_ERR_UNIMPLEMENTED", -8: "GSC_ERR_INTERNAL"}
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}
OUT_FORMAT = {"f32": 0, "rgba8": 1}
DEPTH_GUIDE = {"linear": 0, "exp": 1, "staged": 2}
REUSE = {"off": 0, "depth": 1, "learned": 2}
# stereo_unify: False / "off"; True / "unified" (Eq. 5-6's camera filters for
# both eyes); "exact" (the union of the eyes' own filters, each eye drawing
# its own anchors); the derivation is shared in both
STEREO = {False: 0, "off": 0, True: 1, "unified": 1, "exact": 2}
FLAG_DEBUG_ATTRS = 0x1
FLAG_DEBUG_T = 0x2
FLAG_TIMING = 0x4
FLAG_REUSE_COLLECT = 0x8
FLAG_BLEND_WORK = 0x10
FLAG_UNFUSED = 0x20
REUSE_NPARAM = 2433


class GscError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("max_views", C.c_uint32), ("precision", C.c_uint32), ("reuse", C.c_uint32),
                ("stereo_unify", C.c_uint32), ("cache_gaussians", C.c_uint32), ("max_depth", C.c_uint32),
                ("tile_w", C.c_uint32), ("tile_h", C.c_uint32), ("pair_capacity", C.c_uint64),
                ("bg", C.c_float * 3), ("use_graph", C.c_uint32), ("flags", C.c_uint32),
                ("blocks_per_sm", C.c_uint32), ("out_format", C.c_uint32), ("depth_guide", C.c_uint32),
                ("reserved", C.c_uint32 * 5)]


class ModelDesc(C.Structure):
    _fields_ = [("n_anchors", C.c_uint32), ("feat_dim", C.c_uint32), ("k", C.c_uint32),
                ("hidden", C.c_uint32), ("n_levels", C.c_uint32), ("lod_dmax", C.c_float),
                ("pos", C.c_void_p), ("feat", C.c_void_p), ("offset", C.c_void_p), ("scale", C.c_void_p),
                ("level", C.c_void_p), ("W1", C.c_void_p * 3), ("b1", C.c_void_p * 3),
                ("W2", C.c_void_p * 3), ("b2", C.c_void_p * 3),
                ("level_offset", C.c_void_p), ("lod_blend", C.c_float), ("reserved0", C.c_uint32)]


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32),
                ("znear", C.c_float), ("stereo_partner", C.c_int32), ("model_id", C.c_uint32),
                ("viewer", C.c_uint32)]


class FrameStats(C.Structure):
    _fields_ = [("visible_anchors", C.c_uint64), ("derived_anchors", C.c_uint64), ("records", C.c_uint64),
                ("valid_records", C.c_uint64), ("pairs", C.c_uint64), ("cache_depth", C.c_uint32),
                ("error_flags", C.c_uint32), ("ms_stage", C.c_float * 8)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "ms_stage"}
        d["ms_stage"] = list(self.ms_stage)
        return d


_lib = None


def lib():
    """The loaded libgsc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libgsc.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, U32, U64, I = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
        sig = {
            "gsc_default_config": (None, [P]),
            "gsc_version": (I, []),
            "gsc_create": (I, [P, P, P]),
            "gsc_destroy": (None, [P]),
            "gsc_last_error": (C.c_char_p, [P]),
            "gsc_load_model": (I, [P, P, P]),
            "gsc_set_cameras": (I, [P, P, U32]),
            "gsc_render_frame": (I, [P, P, P]),
            "gsc_render_frame_host": (I, [P, P, P]),
            "gsc_cache_reset": (I, [P]),
            "gsc_synchronize": (I, [P]),
            "gsc_debug_visible": (I, [P, U32, P, U64, P]),
            "gsc_debug_visible_eyes": (I, [P, U32, P, U64, P]),
            "gsc_debug_dviews": (I, [P, P, P]),
            "gsc_debug_attrs": (I, [P, U32, P, U64, P]),
            "gsc_debug_records": (I, [P, P, P, P, U64, P]),
            "gsc_debug_pairs": (I, [P, P, P, U64, P]),
            "gsc_debug_depth_order": (I, [P, P, U64, P]),
            "gsc_debug_ranges": (I, [P, P, U64, P]),
            "gsc_debug_final_T": (I, [P, U32, P, U64, P]),
            "gsc_debug_blend_work": (I, [P, P]),
            "gsc_debug_pipe_rates": (I, [P]),
            "gsc_debug_set_spin_limit": (I, [P, U32]),
            "gsc_debug_sort_pairs": (I, [P, P, P, U64, U32]),
            "gsc_debug_scan": (I, [P, P, U64, P]),
            "gsc_debug_wait_timeout": (I, [P, U32]),
            "gsc_scan_u32_noalloc": (I, [P, P, U64, P, P]),
            "gsc_debug_cache": (I, [P, U32, P, U64, P, P]),
            "gsc_set_tiling": (I, [P, U32, U32, U32]),
            "gsc_render_frame_host_async": (I, [P, P]),
            "gsc_wait_host": (I, [P]),
            "gsc_debug_frame_upload_bytes": (I, []),
            "gsc_reuse_set_weights": (I, [P, P, U32]),
            "gsc_reuse_get_weights": (I, [P, P, U32]),
            "gsc_reuse_collect": (I, [P, U32, P, P, P, U64, P]),
            "gsc_reuse_train": (I, [P, P, P, U64, U32, U32, C.c_float, U64, P, P]),
            "gsc_debug_reuse_grad": (I, [P, P, P, U64, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> List[str]:
    """Names declared in include/*.h (the C ABI)."""
    import re
    root = os.path.dirname(HERE)
    names = []
    for h in ("gsc.h", "gsc_debug.h"):
        txt = open(os.path.join(root, "include", h)).read()
        names += re.findall(r"^\s*(?:GSC_API\s+)?(?:int|void|const char\*)\s+(gsc_\w+)\s*\(", txt, re.M)
    return names


def _p(a) -> C.c_void_p:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(int(a))


def scan_u32_noalloc(d_in: int, d_out: int, n: int, d_total: int = 0, stream: int = 0) -> None:
    """gsc_scan_u32_noalloc on caller-owned device buffers (pointers as ints).

    For callers that cannot allocate device memory where they scan; the
    library uses a fixed internal device array as working memory.  Raises
    GscError on a non-zero status."""
    rc = lib().gsc_scan_u32_noalloc(C.c_void_p(d_in or None), C.c_void_p(d_out or None), int(n),
                                    C.c_void_p(d_total or None), C.c_void_p(stream or None))
    if rc != GSC_OK:
        raise GscError(rc, "gsc_scan_u32_noalloc failed")


def pipe_rates() -> dict:
    """Measured unit throughputs of the current device (per second): exp2
    results, scalar FP32 FMA lane ops, packed FP32x2 FMA lane ops."""
    r = np.zeros(3, np.float64)
    code = lib().gsc_debug_pipe_rates(_p(r))
    if code:
        raise GscError(code, "gsc_debug_pipe_rates failed")
    return {"exp2_per_s": float(r[0]), "ffma_lane_ops_per_s": float(r[1]), "ffma2_lane_ops_per_s": float(r[2])}


def default_config() -> Config:
    c = Config()
    lib().gsc_default_config(C.byref(c))
    return c


def to_camera(cam, partner: int = -1, model_id: int = 0, viewer: int = 0) -> Camera:
    c = Camera()
    R = np.ascontiguousarray(cam.R, np.float32).reshape(-1)
    t = np.ascontiguousarray(cam.t, np.float32).reshape(-1)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.znear = int(cam.width), int(cam.height), float(cam.znear)
    c.stereo_partner, c.model_id, c.viewer = int(partner), int(model_id), int(viewer)
    return c


class Renderer:
    """One gsc_ctx: load_model / set_cameras / render_frame / cache_reset."""

    def __init__(self, max_views: int = 2, precision: str = "fp32", reuse: str = "off",
                 stereo_unify=False, tile: tuple = (16, 16), pair_capacity: int = 0,
                 bg=(0.0, 0.0, 0.0), use_graph: bool = True, flags: int = 0, stream=None,
                 cache_gaussians: int = 0, max_depth: int = 0, blocks_per_sm: int = 0, out_format: str = "f32",
                 depth_guide: str = "linear"):
        cfg = default_config()
        cfg.max_views = max_views
        cfg.precision = PREC[precision]
        cfg.reuse = REUSE[reuse]
        cfg.stereo_unify = STEREO[stereo_unify]
        cfg.tile_w, cfg.tile_h = tile
        cfg.pair_capacity = pair_capacity
        for i in range(3):
            cfg.bg[i] = float(bg[i])
        cfg.use_graph = 1 if use_graph else 0
        cfg.flags = flags
        cfg.cache_gaussians = cache_gaussians
        cfg.max_depth = max_depth
        cfg.blocks_per_sm = blocks_per_sm
        cfg.out_format = OUT_FORMAT[out_format]
        cfg.depth_guide = DEPTH_GUIDE[depth_guide]
        self.cfg = cfg
        self.out_format = out_format
        self.ctx = C.c_void_p()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:
                stream = 0
        self._keep = []
        rc = lib().gsc_create(C.byref(self.ctx), C.byref(cfg), C.c_void_p(int(stream)))
        if rc != GSC_OK:
            raise GscError(rc, "gsc_create failed")
        self.cams: List[Camera] = []

    def _check(self, rc: int):
        if rc != GSC_OK:
            raise GscError(rc, lib().gsc_last_error(self.ctx).decode())

    def close(self):
        if self.ctx:
            lib().gsc_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- the four calls
    def load_model(self, m) -> int:
        keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dt)
            keep.append(a)
            return a.ctypes.data_as(C.c_void_p)

        d = ModelDesc()
        d.n_anchors, d.feat_dim, d.k, d.hidden = m.n, m.feat.shape[1], m.k, m.W1[0].shape[1]
        d.n_levels, d.lod_dmax = m.n_levels, float(m.lod_dmax)
        d.pos, d.feat, d.offset = arr(m.pos, np.float32), arr(m.feat, np.float32), arr(m.offs, np.float32)
        d.scale, d.level = arr(m.scale, np.float32), arr(m.level, np.uint8)
        for h in range(3):
            d.W1[h], d.b1[h] = arr(m.W1[h], np.float32), arr(m.b1[h], np.float32)
            d.W2[h], d.b2[h] = arr(m.W2[h], np.float32), arr(m.b2[h], np.float32)
        lo = getattr(m, "level_offset", None)
        d.level_offset = arr(lo, np.float32) if lo is not None else None
        d.lod_blend = float(getattr(m, "lod_blend", 0.0))
        mid = C.c_uint32()
        self._check(lib().gsc_load_model(self.ctx, C.byref(d), C.byref(mid)))
        return int(mid.value)

    def set_cameras(self, cams: Sequence[Camera]):
        arr = (Camera * len(cams))(*cams)
        self._check(lib().gsc_set_cameras(self.ctx, arr, len(cams)))
        self.cams = list(cams)

    def render_frame(self, outs, stats: bool = True) -> Optional[dict]:
        """outs: list of device pointers or CUDA tensors, one per camera: [H,W,3]
        float32 (out_format "f32") or [H,W,4] uint8 ("rgba8")."""
        ptrs = (C.c_void_p * MAX_VIEWS)()
        for i, o in enumerate(outs):
            ptrs[i] = o.data_ptr() if hasattr(o, "data_ptr") else int(o)
        if stats:
            st = FrameStats()
            self._check(lib().gsc_render_frame(self.ctx, ptrs, C.byref(st)))
            return st.as_dict()
        self._check(lib().gsc_render_frame(self.ctx, ptrs, None))
        return None

    def _host_ptrs(self, outs):
        want = np.float32 if self.out_format == "f32" else np.uint8
        ptrs = (C.c_void_p * MAX_VIEWS)()
        for i, o in enumerate(outs):
            assert o.dtype == want and o.flags.c_contiguous
            ptrs[i] = o.ctypes.data
        return ptrs

    def render_frame_host(self, outs: Sequence[np.ndarray], stats: bool = True) -> Optional[dict]:
        """outs: host arrays [H,W,3] float32 or [H,W,4] uint8 per camera."""
        ptrs = self._host_ptrs(outs)
        st = FrameStats()
        self._check(lib().gsc_render_frame_host(self.ctx, ptrs, C.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def render_frame_host_async(self, outs: Sequence[np.ndarray]):
        """Pipelined host frame: the images land in outs (keep them alive,
        preferably pinned) by the time wait_host() returns."""
        self._check(lib().gsc_render_frame_host_async(self.ctx, self._host_ptrs(outs)))

    def wait_host(self):
        self._check(lib().gsc_wait_host(self.ctx))

    def set_tiling(self, tile_w: int, tile_h: int, blocks_per_sm: int = 0):
        """Blend tiling of this context (the autotuner's knob)."""
        self._check(lib().gsc_set_tiling(self.ctx, tile_w, tile_h, blocks_per_sm))

    # ---------------------------------------------------------------- reuse predictor
    def reuse_set_weights(self, theta):
        t = np.ascontiguousarray(theta, np.float32)
        assert t.shape == (REUSE_NPARAM,)
        self._check(lib().gsc_reuse_set_weights(self.ctx, _p(t), REUSE_NPARAM))

    def reuse_get_weights(self) -> np.ndarray:
        t = np.zeros(REUSE_NPARAM, np.float32)
        self._check(lib().gsc_reuse_get_weights(self.ctx, _p(t), REUSE_NPARAM))
        return t

    def reuse_collect(self, d: int):
        """(z [n,36], label [n], visible index [n]) of derivation view d's last frame."""
        n = C.c_uint64()
        self._check(lib().gsc_reuse_collect(self.ctx, d, None, None, None, 0, C.byref(n)))
        m = n.value
        z = np.zeros((max(m, 1), 36), np.float32)
        y = np.zeros(max(m, 1), np.uint8)
        vi = np.zeros(max(m, 1), np.uint32)
        self._check(lib().gsc_reuse_collect(self.ctx, d, _p(z), _p(y), _p(vi), m, C.byref(n)))
        return z[:m], y[:m], vi[:m]

    def reuse_train(self, z, y, epochs: int, batch: int, lr: float, seed: int = 0, order=None) -> np.ndarray:
        """Train on the GPU; returns the mean loss of each epoch."""
        z = np.ascontiguousarray(z, np.float32)
        y = np.ascontiguousarray(y, np.uint8)
        n = z.shape[0]
        assert z.shape == (n, 36) and y.shape == (n,)
        o = None if order is None else np.ascontiguousarray(order, np.uint32)
        if o is not None:
            assert o.size == n * epochs
        loss = np.zeros(epochs, np.float32)
        self._check(lib().gsc_reuse_train(self.ctx, _p(z), _p(y), n, epochs, batch, float(lr), int(seed),
                                          _p(o), _p(loss)))
        return loss

    def debug_reuse_grad(self, z, y):
        z = np.ascontiguousarray(z, np.float32)
        y = np.ascontiguousarray(y, np.uint8)
        g = np.zeros(REUSE_NPARAM, np.float32)
        loss = np.zeros(1, np.float32)
        self._check(lib().gsc_debug_reuse_grad(self.ctx, _p(z), _p(y), z.shape[0], _p(g), _p(loss)))
        return g, float(loss[0])

    def cache_reset(self):
        self._check(lib().gsc_cache_reset(self.ctx))

    def synchronize(self):
        self._check(lib().gsc_synchronize(self.ctx))

    # ---------------------------------------------------------------- debug read-backs
    def debug_visible(self, d: int) -> np.ndarray:
        n = C.c_uint64()
        self._check(lib().gsc_debug_visible(self.ctx, d, None, 0, C.byref(n)))
        out = np.zeros(max(n.value, 1), np.uint32)
        self._check(lib().gsc_debug_visible(self.ctx, d, _p(out), n.value, C.byref(n)))
        return out[: n.value]

    def debug_visible_eyes(self, d: int) -> np.ndarray:
        """Exact stereo views: per visible anchor of view d, bit e = camera e of the pair keeps it."""
        n = C.c_uint64()
        self._check(lib().gsc_debug_visible_eyes(self.ctx, d, None, 0, C.byref(n)))
        out = np.zeros(max(n.value, 1), np.uint8)
        self._check(lib().gsc_debug_visible_eyes(self.ctx, d, _p(out), n.value, C.byref(n)))
        return out[: n.value]

    def debug_dviews(self):
        n = C.c_uint32()
        first = (C.c_int32 * MAX_VIEWS)()
        self._check(lib().gsc_debug_dviews(self.ctx, C.byref(n), first))
        return int(n.value), list(first)[: n.value]

    def debug_attrs(self, d: int) -> np.ndarray:
        n = C.c_uint64()
        self._check(lib().gsc_debug_attrs(self.ctx, d, None, 0, C.byref(n)))
        out = np.zeros((max(n.value, 1), K, 11), np.float32)
        self._check(lib().gsc_debug_attrs(self.ctx, d, _p(out), n.value, C.byref(n)))
        return out[: n.value]

    def debug_records(self):
        n = C.c_uint64()
        self._check(lib().gsc_debug_records(self.ctx, None, None, None, 0, C.byref(n)))
        m = max(n.value, 1)
        rec = np.zeros((m, 12), np.float32)
        key = np.zeros(m, np.uint32)
        cnt = np.zeros(m, np.uint32)
        self._check(lib().gsc_debug_records(self.ctx, _p(rec), _p(key), _p(cnt), n.value, C.byref(n)))
        k = n.value
        return rec[:k], key[:k], cnt[:k]

    def debug_pairs(self):
        n = C.c_uint64()
        self._check(lib().gsc_debug_pairs(self.ctx, None, None, 0, C.byref(n)))
        k = np.zeros(max(n.value, 1), np.uint32)
        v = np.zeros(max(n.value, 1), np.uint32)
        self._check(lib().gsc_debug_pairs(self.ctx, _p(k), _p(v), n.value, C.byref(n)))
        return k[: n.value], v[: n.value]

    def debug_depth_order(self) -> np.ndarray:
        n = C.c_uint64()
        self._check(lib().gsc_debug_depth_order(self.ctx, None, 0, C.byref(n)))
        v = np.zeros(max(n.value, 1), np.uint32)
        self._check(lib().gsc_debug_depth_order(self.ctx, _p(v), n.value, C.byref(n)))
        return v[: n.value]

    def debug_ranges(self) -> np.ndarray:
        n = C.c_uint64()
        self._check(lib().gsc_debug_ranges(self.ctx, None, 0, C.byref(n)))
        r = np.zeros((max(n.value, 1), 2), np.uint32)
        self._check(lib().gsc_debug_ranges(self.ctx, _p(r), n.value, C.byref(n)))
        return r[: n.value]

    def debug_final_T(self, v: int) -> np.ndarray:
        n = C.c_uint64()
        self._check(lib().gsc_debug_final_T(self.ctx, v, None, 0, C.byref(n)))
        T = np.zeros(max(n.value, 1), np.float32)
        self._check(lib().gsc_debug_final_T(self.ctx, v, _p(T), n.value, C.byref(n)))
        return T[: n.value]

    def debug_blend_work(self) -> tuple:
        """(walk, issued) pixel evaluations of the last frame's blend (needs FLAG_BLEND_WORK):
        walk = the front-to-back walk of every pixel up to its stop; issued = pixel
        slots run through the inner loop after the warp-band box test."""
        w = np.zeros(2, np.uint64)
        self._check(lib().gsc_debug_blend_work(self.ctx, _p(w)))
        return int(w[0]), int(w[1])

    def debug_cache(self, d: int):
        """(line status per visible anchor, state dict) of derivation view d's cache."""
        n = C.c_uint64()
        st = (C.c_uint32 * 8)()
        self._check(lib().gsc_debug_cache(self.ctx, d, None, 0, C.byref(n), st))
        v = np.zeros(max(n.value, 1), np.uint32)
        self._check(lib().gsc_debug_cache(self.ctx, d, _p(v), n.value, C.byref(n), st))
        keys = ["t", "depth", "misses", "new", "free", "visible", "d_max", "lines"]
        return v[: n.value], dict(zip(keys, list(st)))

    def debug_set_spin_limit(self, limit: int):
        self._check(lib().gsc_debug_set_spin_limit(self.ctx, limit))

    def debug_sort_pairs(self, keys: np.ndarray, vals: np.ndarray, bits: int):
        k = np.ascontiguousarray(keys, np.uint32).copy()
        v = np.ascontiguousarray(vals, np.uint32).copy()
        self._check(lib().gsc_debug_sort_pairs(self.ctx, _p(k), _p(v), k.shape[0], bits))
        return k, v

    def debug_wait_timeout(self, spin_limit: int) -> int:
        """Status code of the timeout probe (GSC_ERR_TIMEOUT = -5 expected)."""
        return int(lib().gsc_debug_wait_timeout(self.ctx, spin_limit))

    def debug_scan(self, vals: np.ndarray):
        a = np.ascontiguousarray(vals, np.uint32).copy()
        tot = C.c_uint64()
        self._check(lib().gsc_debug_scan(self.ctx, _p(a), a.shape[0], C.byref(tot)))
        return a, int(tot.value)

"""Learned reuse predictor: training-data collection, GPU training and the
comparison with the depth rule, all through the C ABI.

collect()   renders camera paths in the cached form with label collection
            on (GSC_FLAG_REUSE_COLLECT) and gathers (inputs, label) of every
            anchor that held a valid line, subsampled to a fixed count
train()     gsc_reuse_train from an initial parameter vector
evaluate()  renders a path with the depth rule or with the predictor (label
            collection on, so every reuse decision can be scored) and
            reports reuse and wrong-reuse rates and PSNR against the same
            form without the cache (so only the reuse error is measured);
            it also returns the rendered values at given pixels of given
            frames, for a caller that judges them against reference images
save() / load()  the flat float32 parameter vector, with a small header
"""
from __future__ import annotations

import struct
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .native import FLAG_REUSE_COLLECT, REUSE_NPARAM, Renderer, to_camera

MAGIC = b"GSCR"
VERSION = 1


def _pair(r: Renderer, mid: int, L, R):
    r.set_cameras([to_camera(L, partner=1, model_id=mid), to_camera(R, partner=0, model_id=mid)])


def _outs(L):
    import torch
    return [torch.empty((L.height, L.width, 3), dtype=torch.float32, device="cuda") for _ in range(2)]


def collect(model, paths: Sequence[Sequence[Tuple]], n_samples: int = 100_000, seed: int = 0,
            precision: str = "bf16") -> Tuple[np.ndarray, np.ndarray, Dict]:
    """Samples from stereo paths [(L, R), ...] (unified derivation camera,
    depth-rule cache, each path from an empty cache).  Returns (z [n,36],
    label [n] uint8, stats)."""
    rs = np.random.default_rng(seed)
    r = Renderer(max_views=2, precision=precision, reuse="depth", stereo_unify=True, flags=FLAG_REUSE_COLLECT)
    mid = r.load_model(model)
    outs = _outs(paths[0][0][0])
    per_frame = []
    total = 0
    for path in paths:
        r.cache_reset()
        for L, R in path:
            _pair(r, mid, L, R)
            r.render_frame(outs, stats=False)
            z, y, _ = r.reuse_collect(0)
            total += len(y)
            per_frame.append((z, y))
    r.close()
    # an equal share of every frame's candidates (uniform over the pooled set)
    keep = min(1.0, n_samples / max(total, 1))
    Z, Y = [], []
    for z, y in per_frame:
        sel = rs.uniform(size=len(y)) < keep
        Z.append(z[sel])
        Y.append(y[sel])
    Z = np.concatenate(Z) if Z else np.zeros((0, 36), np.float32)
    Y = np.concatenate(Y) if Y else np.zeros(0, np.uint8)
    if len(Y) > n_samples:
        idx = np.sort(rs.choice(len(Y), n_samples, replace=False))
        Z, Y = Z[idx], Y[idx]
    return Z, Y, {"candidates": total, "samples": int(len(Y)), "positive_frac": float(Y.mean()) if len(Y) else 0.0}


def train(z: np.ndarray, y: np.ndarray, theta0: np.ndarray, epochs: int = 40, batch: int = 4096,
          lr: float = 2e-3, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """GPU training; returns (trained parameters, mean loss per epoch)."""
    r = Renderer(max_views=1)
    r.reuse_set_weights(theta0)
    losses = r.reuse_train(z, y, epochs, batch, lr, seed)
    theta = r.reuse_get_weights()
    r.close()
    return theta, losses


def evaluate(model, path: Sequence[Tuple], theta: Optional[np.ndarray] = None, precision: str = "bf16",
             psnr_every: int = 1, sample: Optional[Dict[int, Tuple[np.ndarray, np.ndarray]]] = None) -> Dict:
    """Render a stereo path from an empty cache with the depth rule (theta
    None) or the predictor; score every reuse by its label (a reuse of a
    line whose label is 0 is wrong) and the images by PSNR against the same
    form (precision, unified stereo) without the cache, every `psnr_every`
    frames.  sample: {frame: (px, py)}; the result's "samples" then holds,
    per listed frame, the two eyes' rendered values at those pixels
    ([2, n, 3] float32)."""
    import torch
    mode = "depth" if theta is None else "learned"
    r = Renderer(max_views=2, precision=precision, reuse=mode, stereo_unify=True, flags=FLAG_REUSE_COLLECT)
    mid = r.load_model(model)
    if theta is not None:
        r.reuse_set_weights(theta)
    ref = Renderer(max_views=2, precision=precision, stereo_unify=True)
    rmid = ref.load_model(model)
    outs, routs = _outs(path[0][0]), _outs(path[0][0])
    vis = hits = wrong = cand = good = 0
    psnrs = []
    samples = {}
    for f, (L, R) in enumerate(path):
        _pair(r, mid, L, R)
        st = r.render_frame(outs)
        if sample and f in sample:
            px, py = sample[f]
            ix, iy = torch.as_tensor(px, device="cuda").long(), torch.as_tensor(py, device="cuda").long()
            samples[f] = np.stack([o[iy, ix].cpu().numpy() for o in outs])
        z, y, vi = r.reuse_collect(0)
        vstat, _ = r.debug_cache(0)
        hit = (vstat & 0x80000000) != 0
        lab = np.zeros(len(vstat), np.int8) - 1
        lab[vi] = y
        vis += len(vstat)
        hits += int(hit.sum())
        wrong += int((hit & (lab == 0)).sum())
        cand += len(vi)
        good += int((lab == 1).sum())
        if psnr_every and f % psnr_every == 0:
            _pair(ref, rmid, L, R)
            ref.render_frame(routs, stats=False)
            torch.cuda.synchronize()
            mse = sum(float(torch.mean((a - b) ** 2)) for a, b in zip(outs, routs)) / 2
            psnrs.append(10 * np.log10(1.0 / max(mse, 1e-10)))  # identical images count as 100 dB
    r.close()
    ref.close()
    return {"mode": mode, "frames": len(path), "reuse_frac": hits / max(vis, 1),
            "wrong_reuse_frac": wrong / max(hits, 1), "wrong_per_visible": wrong / max(vis, 1),
            "reusable_frac": good / max(vis, 1), "candidates_frac": cand / max(vis, 1),
            "psnr_db_min": min(psnrs) if psnrs else None, "psnr_db_mean": float(np.mean(psnrs)) if psnrs else None,
            "samples": samples}


def save(path: str, theta: np.ndarray) -> None:
    t = np.ascontiguousarray(theta, "<f4")
    assert t.shape == (REUSE_NPARAM,)
    with open(path, "wb") as f:
        f.write(MAGIC + struct.pack("<II", VERSION, REUSE_NPARAM) + t.tobytes())


def load(path: str) -> np.ndarray:
    with open(path, "rb") as f:
        head = f.read(12)
        if head[:4] != MAGIC:
            raise ValueError(f"{path}: not a reuse-predictor file")
        ver, n = struct.unpack("<II", head[4:])
        if ver != VERSION or n != REUSE_NPARAM:
            raise ValueError(f"{path}: version {ver}, {n} parameters")
        return np.frombuffer(f.read(4 * n), "<f4").astype(np.float32)

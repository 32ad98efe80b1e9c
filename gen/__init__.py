"""Seeded synthetic inputs shared by the oracle tests, the CUDA path and the bench.

Holds random-number streams, scenes and camera paths only; none of the
rendering method's arithmetic lives here.
"""
import numpy as np

from .rng import Stream, splitmix64, stream_seed
from .scenes import (FEAT_DIM, HIDDEN, IN_DIM, K_GAUSS, Model, city_scene,
                     glorot_mlps, head_out_dims, reuse_mlp_init, tiny_scene, with_level_offsets)
from .cameras import (Camera, HeadPose, city_path, look_rotation, path_extent,
                      pinhole, reuse_path, stereo_frames, stereo_pair, tiny_camera)


def city_workload(n_anchors: int = 2_000_000, seed: int = 10, path_seed: int = 11,
                  n_frames: int = 300, width: int = 1920, height: int = 1080):
    """The city-scale stereo workload: scene plus the ascending stereo path."""
    poses = city_path(n_frames=n_frames, seed=path_seed)
    x0, y0, x1, y1 = path_extent(poses)
    model = city_scene(n=n_anchors, seed=seed, keep_clear=(x0, y0, x1, y1, 30.0))
    frames = stereo_frames(poses, width=width, height=height)
    return model, frames


__all__ = [
    "Stream", "splitmix64", "stream_seed", "FEAT_DIM", "HIDDEN", "IN_DIM", "K_GAUSS",
    "Model", "city_scene", "glorot_mlps", "head_out_dims", "reuse_mlp_init", "tiny_scene", "Camera",
    "HeadPose", "city_path", "look_rotation", "path_extent", "pinhole", "stereo_frames",
    "stereo_pair", "tiny_camera", "with_level_offsets", "city_workload", "reuse_path", "multiviewer_workload", "MV_SCENES", "MV_VIEWERS",
]


# Batched multi-viewer workload: three city scenes and eight viewers whose
# images all render in one frame.  Each entry of VIEWERS is
# (scene index, width, height, stereo, frame offset along the scene's path,
#  yaw offset in degrees).
MV_SCENES = ((500_000, 40, 42), (2_000_000, 10, 11), (4_000_000, 41, 43))  # (anchors, scene seed, path seed)
MV_VIEWERS = (
    (1, 1920, 1080, True, 0, 0.0),
    (1, 1920, 1080, True, 60, 20.0),
    (2, 1920, 1080, True, 30, 0.0),
    (0, 1600, 900, True, 0, 0.0),
    (2, 1280, 720, True, 120, -25.0),
    (1, 1920, 1080, False, 150, 0.0),
    (0, 1280, 720, False, 90, 30.0),
    (2, 1280, 720, False, 200, 10.0),
)


def multiviewer_workload(scale: float = 1.0, size_scale: float = 1.0, n_frames: int = 300):
    """Three scenes (0.5M / 2M / 4M anchors x `scale`) generated like the city
    scene, each with its own ascending path, and eight viewers riding those
    paths at different frame offsets and yaw offsets (13 images: five stereo
    pairs and three mono views, 1280x720 up to 1920x1080, x `size_scale`).

    Returns (models, viewers, frame_fn): frame_fn(t) gives, for each image,
    (viewer, scene, Camera, stereo partner index within the frame or -1)."""
    models, paths = [], []
    for n, seed, pseed in MV_SCENES:
        poses = city_path(n_frames=n_frames, seed=pseed)
        x0, y0, x1, y1 = path_extent(poses)
        models.append(city_scene(n=max(int(n * scale), 1000), seed=seed, keep_clear=(x0, y0, x1, y1, 30.0)))
        paths.append(poses)

    def frame_fn(t: int):
        out = []
        for v, (s, w, h, stereo, off, dyaw) in enumerate(MV_VIEWERS):
            p = paths[s][(t + off) % n_frames]
            R = look_rotation(p.yaw + np.deg2rad(dyaw), p.pitch)
            W = max(int(round(w * size_scale)), 16)
            H = max(int(round(h * size_scale)), 8)
            if stereo:
                L, Rr = stereo_pair(R, p.pos, W, H, 60.0)
                i = len(out)
                out.append((v, s, L, i + 1))
                out.append((v, s, Rr, i))
            else:
                out.append((v, s, pinhole(R, p.pos, W, H, 60.0), -1))
        return out

    return models, MV_VIEWERS, frame_fn
